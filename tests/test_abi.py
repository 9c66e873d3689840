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


# --- the Python binding against the header --------------------------------

_SCALARS = {"int": ctypes.c_int, "int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32,
            "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64, "size_t": ctypes.c_size_t,
            "uint8_t": ctypes.c_uint8, "float": ctypes.c_float, "double": ctypes.c_double}


def _header_src():
    src = open(os.path.join(ROOT, "include", "diffrestore.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"//[^\n]*", "", src)


def _prototypes():
    """{name: (return type, [parameter types])} parsed from the header."""
    out = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\b(dr_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", _header_src()):
        params = [p.strip() for p in m.group(3).split(",")]
        types = [] if params == ["void"] else [re.sub(r"\s*\w+$", "", p) for p in params]
        out[m.group(2)] = (m.group(1).strip(), types)
    return out


def _is_pointer(ct):
    return ct in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(ct, type) and issubclass(ct, ctypes._Pointer))


def _check_param(ctype_decl, ct, _lib):
    t = ctype_decl.replace("const ", "").replace(" ", "")
    stars = t.count("*")
    base = t.rstrip("*")
    if stars == 0:
        return ct is _SCALARS[base]
    if not _is_pointer(ct):
        return False
    if ct is ctypes.c_void_p:                      # untyped pointer: any pointee
        return True
    pointee = ct._type_
    if stars > 1:
        return _is_pointer(pointee)
    if base in _SCALARS:
        return pointee is _SCALARS[base]
    return getattr(_lib, base, None) is pointee


def test_binding_signatures_match_the_header():
    """Every argtype and restype of the ctypes binding has the width, signedness
    and pointer-ness of the header's prototype, argument by argument."""
    from paper_2605_08916_gb300 import _lib
    protos, sigs = _prototypes(), _lib.signatures()
    assert sorted(protos) == _declared() == sorted(sigs)
    for name, (ret, params) in protos.items():
        args, res = sigs[name]
        assert len(args) == len(params), name
        for i, (decl, ct) in enumerate(zip(params, args)):
            assert _check_param(decl, ct, _lib), f"{name} argument {i}: {decl} vs {ct}"
        assert res is (ctypes.c_char_p if ret == "const char*" else _SCALARS[ret]), name


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """The ctypes structs have the C compiler's member order, offsets and sizes,
    and every DR_* constant of the binding has the header's value."""
    import shutil
    import subprocess
    from paper_2605_08916_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = _header_src()
    structs = {m.group(2): m.group(1) for m in
               re.finditer(r"typedef struct[^{]*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S)}
    assert set(structs) == {"dr_params", "dr_scene_desc", "dr_mesh_desc", "dr_instance_desc"}
    lines = []
    for sname, body in structs.items():
        members = []
        for decl in body.split(";"):
            decl = re.sub(r"\[\d+\]", "", decl).strip()
            if decl:
                first, *rest = decl.split(",")
                members.append(re.findall(r"\w+", first)[-1])
                members += [r.strip() for r in rest]
        cls = getattr(_lib, sname)
        assert [f[0] for f in cls._fields_] == members, sname
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for f in members:
            lines.append(f'printf("{sname} {f} %zu\\n", offsetof({sname}, {f}));')
    consts = {k: v for k, v in vars(_lib).items() if re.fullmatch(r"DR_[A-Z0-9_]+", k) and isinstance(v, int)}
    for k in consts:
        lines.append(f'printf("const {k} %lld\\n", (long long){k});')
    prog = tmp_path / "probe.c"
    prog.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"diffrestore.h\"\n"
                    "int main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(prog),
                    "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for sname in structs:
        cls = getattr(_lib, sname)
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert got[(sname, f)] == getattr(cls, f).offset, (sname, f)
    for k, v in consts.items():
        assert got[("const", k)] == v, k
