"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/diffrestore.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "diffrestore.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dr_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["dr_create", "dr_destroy", "dr_scene_upload", "dr_chains_init", "dr_step", "dr_splat",
                     "dr_resolve", "dr_readback_state", "dr_eval_logp", "dr_get_counters"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2605_08916_gb300 import _lib
    L = _lib.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(_lib.EXPORTS) == _declared()
    assert L.dr_version() >= 100


def test_library_is_built_for_sm103a():
    from paper_2605_08916_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.build())


def test_calls_fail_cleanly_without_a_context():
    from paper_2605_08916_gb300 import _lib
    L = _lib.load()
    assert L.dr_step(None, 1) == _lib.DR_ERR_INVALID_ARG
    assert "NULL" in _lib.last_error()
    assert L.dr_destroy(None) == _lib.DR_OK
    assert L.dr_create(None, 0, None) == _lib.DR_ERR_INVALID_ARG
    # the hierarchy and instancing entry points check their context first
    assert L.dr_scene_upload_instanced(None, None, 0, None, 0, None, 0, None, 1, 1) == _lib.DR_ERR_INVALID_ARG
    assert L.dr_two_level_info(None, None, None, None) == _lib.DR_ERR_INVALID_ARG
    assert L.dr_bvh8_info(None, None, None) == _lib.DR_ERR_INVALID_ARG
    assert L.dr_bvh4_sah(None, None, None) == _lib.DR_ERR_INVALID_ARG
    assert L.dr_set_option(None, _lib.DR_OPT_TWO_LEVEL, 1) == _lib.DR_ERR_INVALID_ARG


def test_create_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2605_08916_gb300 import _lib
    h = ctypes.c_void_p()
    assert _lib.load().dr_create(ctypes.byref(h), 0, None) == _lib.DR_ERR_CUDA
    assert not h.value


def test_oracle_and_library_share_no_code():
    """The oracle (test infrastructure) and the CUDA library include nothing
    from each other."""
    csrc = os.path.join(ROOT, "paper_2605_08916_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    orc = open(os.path.join(ROOT, "oracle", "oracle.cpp")).read()
    assert "#include \"" not in orc
    for f in ["renderer.py", "_lib.py", "build.py", "__init__.py"]:
        txt = open(os.path.join(ROOT, "paper_2605_08916_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f
