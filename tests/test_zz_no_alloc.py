"""dr_splat_records_noalloc: the splat for callers that cannot call
cudaMalloc (a render loop held to a fixed device-memory budget, code running
where another framework owns the allocator, code that must not trigger the
synchronisation cudaMalloc / cudaFree can cause).  Its scratch is a fixed
array inside the library, so it must give exactly what the allocating entry
point dr_splat_records gives, call after call.

This file is collected last on purpose: it also has to pass after every other
test has run in the same process (the shared scratch keeps the previous
call's contents)."""
import ctypes

import numpy as np
import pytest

from paper_2605_08916_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _records(rng, M, n_pix):
    pix = (rng.zipf(1.4, M) % n_pix).astype(np.uint32)
    val = (rng.normal(size=(M, 3)) * 1e-3).astype(np.float32)
    rec = np.zeros((M, 4), np.int32)
    rec[:, 0] = pix.view(np.int32)
    rec[:, 1:] = val.view(np.int32)
    return rec


def test_noalloc_splat_matches_allocating_splat_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_08916_gb300 import _lib
    from paper_2605_08916_gb300 import renderer as R
    L = _lib.load()
    W, H = 40, 30
    n_pix = W * H
    rng = np.random.default_rng(11)
    batches = [_records(rng, 50000, n_pix), _records(rng, 65536, n_pix)]

    # the existing, allocating entry point on a context
    r = R.Renderer()
    r.set_mixture(S.constant_target(d=2, value=1.0, width=W, height=H))
    r.init_chains(16, 1, R.make_params(L=1, drift="none", k0=1.0))
    r.clear_image()

    # the allocation-free entry point, on a plain device buffer
    accum = torch.zeros((n_pix, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for rec in batches:
        d_rec = torch.from_numpy(rec).cuda()
        r.splat_records(d_rec)
        code = L.dr_splat_records_noalloc(ctypes.c_void_p(d_rec.data_ptr()), rec.shape[0], n_pix,
                                          ctypes.c_void_p(accum.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert code == _lib.DR_OK, _lib.last_error()
        torch.cuda.synchronize()
        # same records, same stable sort, same FP64 sums: identical images
        assert np.array_equal(accum.cpu().numpy(), r.readback_accum())
    r.close()


def test_noalloc_splat_rejects_oversized_batches():
    import torch
    from paper_2605_08916_gb300 import _lib
    L = _lib.load()
    accum = torch.zeros((16, 3), dtype=torch.float64, device="cuda")
    big = torch.zeros((_lib.DR_NOALLOC_MAX_RECORDS + 1, 4), dtype=torch.int32, device="cuda")
    code = L.dr_splat_records_noalloc(ctypes.c_void_p(big.data_ptr()), big.shape[0], 16,
                                      ctypes.c_void_p(accum.data_ptr()), None)
    assert code == _lib.DR_ERR_INVALID_ARG
    assert "DR_NOALLOC_MAX_RECORDS" in _lib.last_error()
    assert float(accum.abs().sum()) == 0.0


def test_noalloc_splat_skips_bad_pixel_indices_and_reports_them():
    """A record whose pixel index is >= n_pix is skipped without touching
    the other pixels' sums (it sorts after every valid record), and
    dr_splat_records_noalloc_status reports it; an empty batch is a no-op
    that clears the report."""
    import torch
    from paper_2605_08916_gb300 import _lib
    from paper_2605_08916_gb300 import renderer as R
    L = _lib.load()
    W, H = 40, 30
    n_pix = W * H
    rng = np.random.default_rng(12)
    rec = _records(rng, 30000, n_pix)
    bad = rng.choice(rec.shape[0], 7, replace=False)
    # indices whose low bits alias valid pixels: n_pix + 5, 2^11 + 3, and the largest
    rec[bad[:3], 0] = np.array([n_pix + 5, (1 << 11) + 3, 0x7fffffff], np.int64).astype(np.int32)
    rec[bad[3:], 0] = np.array([0xffffffff, n_pix, n_pix + 1, 1 << 20], np.uint32).view(np.int32)
    good = np.ones(rec.shape[0], bool)
    good[bad] = False

    r = R.Renderer()
    r.set_mixture(S.constant_target(d=2, value=1.0, width=W, height=H))
    r.init_chains(16, 1, R.make_params(L=1, drift="none", k0=1.0))
    r.clear_image()
    r.splat_records(torch.from_numpy(np.ascontiguousarray(rec[good])).cuda())
    expect = r.readback_accum()
    r.close()

    stream = torch.cuda.current_stream()
    s = ctypes.c_void_p(stream.cuda_stream)
    accum = torch.zeros((n_pix, 3), dtype=torch.float64, device="cuda")
    d_rec = torch.from_numpy(rec).cuda()
    assert L.dr_splat_records_noalloc(ctypes.c_void_p(d_rec.data_ptr()), rec.shape[0], n_pix,
                                      ctypes.c_void_p(accum.data_ptr()), s) == _lib.DR_OK
    assert L.dr_splat_records_noalloc_status(s) == _lib.DR_ERR_DEVICE_CHECK
    assert "n_pix" in _lib.last_error()
    assert np.array_equal(accum.cpu().numpy(), expect)
    # an empty batch adds nothing and clears the report
    assert L.dr_splat_records_noalloc(None, 0, n_pix, ctypes.c_void_p(accum.data_ptr()), s) == _lib.DR_OK
    assert L.dr_splat_records_noalloc_status(s) == _lib.DR_OK
    torch.cuda.synchronize()
    assert np.array_equal(accum.cpu().numpy(), expect)
