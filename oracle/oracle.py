"""ctypes front end of the FP64 CPU oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  It
shares no code with the CUDA library; both receive the same seeded inputs from
``paper_2605_08916_gb300.scenes``.

Parity pins of every function here live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

INFO_MAXV = 20


class Params(C.Structure):
    """Restore parameters (all of Sec. 5.3 / Sec. 6 "Parameter choices")."""
    _fields_ = [("L", C.c_int32), ("drift_mode", C.c_int32), ("rb_weight", C.c_int32), ("pad", C.c_int32),
                ("stddev", C.c_double), ("dt", C.c_double), ("gamma_tilde", C.c_double), ("eps", C.c_double),
                ("fd_h", C.c_double), ("m", C.c_double), ("k0", C.c_double)]


DRIFT = {"none": 0, "fd": 1, "exact": 2, "adjoint": 2, "mala": 3}


def make_params(L=4, drift="exact", rb=True, stddev=5e-3, dt=1e-5, gamma_tilde=None, eps=1e-8, fd_h=1e-3,
                m=64.0, k0=1.0):
    if gamma_tilde is None:
        gamma_tilde = 0.5 * stddev * stddev
    return Params(int(L), DRIFT[drift] if isinstance(drift, str) else int(drift), int(bool(rb)), 0,
                  float(stddev), float(dt), float(gamma_tilde), float(eps), float(fd_h), float(m), float(k0))


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        fp = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        up = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        L.orc_philox.argtypes = [up, up, up, C.c_int64]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_scene_create.restype = P
        L.orc_scene_create.argtypes = [fp, C.c_int, ip, P, C.c_int, ip, fp, C.c_int, fp, C.c_int, C.c_int, C.c_int]
        L.orc_scene_destroy.argtypes = [P]
        L.orc_scene_num_lights.argtypes = [P]
        L.orc_mixture_create.restype = P
        L.orc_mixture_create.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int, C.c_double]
        L.orc_mixture_destroy.argtypes = [P]
        L.orc_step_create.restype = P
        L.orc_step_create.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
        L.orc_step_destroy.argtypes = [P]
        L.orc_lstar_over_p.restype = C.c_int
        L.orc_lstar_over_p.argtypes = [P, C.c_int, dp, dp, C.c_int64, C.c_double, C.c_int, dp]
        L.orc_trace.argtypes = [P, dp, dp, C.c_int64, C.c_int, ip, dp, P]
        L.orc_info_stride.restype = C.c_int
        L.orc_eval.argtypes = [P, C.c_int, C.c_int, dp, C.c_int64, C.c_double, P, P, P, P, P]
        L.orc_fd_score.argtypes = [P, C.c_int, C.c_int, dp, C.c_int64, C.c_double, C.c_double, dp]
        L.orc_bsdf_sample.argtypes = [fp, dp, dp, C.c_double, C.c_double, dp, dp, dp, ip]
        L.orc_bsdf_sample.restype = C.c_int
        L.orc_bsdf_eval.argtypes = [fp, dp, dp, dp, dp, dp]
        L.orc_fresnel_dielectric.restype = C.c_double
        L.orc_fresnel_dielectric.argtypes = [C.c_double] * 3
        L.orc_fresnel_conductor.restype = C.c_double
        L.orc_fresnel_conductor.argtypes = [C.c_double] * 3
        L.orc_local_dynamics.argtypes = [dp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, dp, dp, dp]
        L.orc_restore_run.argtypes = [P, C.c_int, C.POINTER(Params), C.c_uint64, C.c_uint32, up, C.c_int64,
                                      C.c_int, P, P, P, P, P, P, P, P, P, P]
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L.orc_restore_tours.argtypes = [P, C.c_int, C.POINTER(Params), C.c_uint64, C.c_uint32, up, C.c_int64,
                                        C.c_int64, dp, dp, dp, i64p, u8p, P]
        L.orc_pt_image.argtypes = [P, C.c_int, C.c_int, C.c_uint64, dp, dp]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def set_threads(n):
    lib().orc_set_threads(int(n))


def num_threads():
    return lib().orc_num_threads()


def philox4x32_10(ctr, key):
    """ctr: uint32 [n, 4]; key: uint32 [n, 2] -> uint32 [n, 4]."""
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    lib().orc_philox(ctr.ravel(), key.ravel(), out.ravel(), ctr.shape[0])
    return out


class OracleScene:
    kind = 0

    def __init__(self, scene, use_bvh=None):
        self.scene = scene
        if use_bvh is None:
            use_bvh = scene.n_tris > 64
        L = lib()
        self._keep = (np.ascontiguousarray(scene.verts, np.float32), np.ascontiguousarray(scene.tris, np.int32),
                      None if scene.normals is None else np.ascontiguousarray(scene.normals, np.float32),
                      np.ascontiguousarray(scene.tri_mat, np.int32),
                      np.ascontiguousarray(scene.materials, np.float32), np.ascontiguousarray(scene.camera,
                                                                                             np.float32))
        v, t, n, tm, m, cam = self._keep
        self.h = L.orc_scene_create(v.ravel(), v.shape[0], t.ravel(), _ptr(n), t.shape[0], tm, m.ravel(),
                                    m.shape[0], cam, scene.width, scene.height, int(bool(use_bvh)))
        self.width, self.height = scene.width, scene.height

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_destroy(self.h)
            self.h = None

    @property
    def n_lights(self):
        return lib().orc_scene_num_lights(self.h)

    def trace(self, o, d, exclude=-1, count_tests=False):
        o = np.ascontiguousarray(o, np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
        n = o.shape[0]
        tri = np.zeros(n, np.int32)
        t = np.zeros(n, np.float64)
        tests = np.zeros(n, np.int64) if count_tests else None
        lib().orc_trace(self.h, o.ravel(), d.ravel(), n, int(exclude), tri, t, _ptr(tests))
        return (tri, t, tests) if count_tests else (tri, t)


class OracleMixture:
    kind = 1

    def __init__(self, mix):
        self.mix = mix
        self.d = mix.d
        self._keep = (np.ascontiguousarray(mix.w, np.float64).reshape(-1), np.ascontiguousarray(mix.mu,
                                                                                               np.float64).reshape(-1),
                      np.ascontiguousarray(mix.sig, np.float64).reshape(-1))
        w, mu, sig = self._keep
        if w.size == 0:
            w = mu = sig = np.zeros(1)
        self.h = lib().orc_mixture_create(mix.d, mix.K, w, mu, sig, mix.width, mix.height, float(mix.const))
        self.width, self.height = mix.width, mix.height

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_mixture_destroy(self.h)
            self.h = None


class OracleStep:
    """The jump density of ``scenes.StepDensity``."""
    kind = 2

    def __init__(self, st):
        self.st = st
        self.d = st.d
        self.h = lib().orc_step_create(st.d, float(st.c1), float(st.c2), float(st.w), st.width, st.height)
        self.width, self.height = st.width, st.height

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_step_destroy(self.h)
            self.h = None


def target(obj, **kw):
    from paper_2605_08916_gb300 import scenes as S
    if isinstance(obj, S.Scene):
        return OracleScene(obj, **kw)
    if isinstance(obj, S.Mixture):
        return OracleMixture(obj)
    if isinstance(obj, S.StepDensity):
        return OracleStep(obj)
    return obj


def lstar_over_p(tgt, y, stddev=5e-3, dt=1e-5, gamma_tilde=None, eps=1e-8, radius=8.0, n=129):
    """(L* p / p)(y) of App. C for a 2-D target at points y [M, 2]: the bias
    term of the modified killing rate (Sec. 5.2) for the Euler-Maruyama local
    dynamics with holding rate 1 / dt, by quadrature."""
    if gamma_tilde is None:
        gamma_tilde = 0.5 * stddev * stddev
    y = np.ascontiguousarray(y, np.float64).reshape(-1, 2)
    out = np.zeros(y.shape[0])
    rc = lib().orc_lstar_over_p(tgt.h, tgt.kind, np.array([stddev, dt, gamma_tilde, eps], np.float64), y.ravel(),
                                y.shape[0], float(radius), int(n), out)
    if rc != 0:
        raise ValueError("lstar_over_p needs a 2-D analytic target")
    return out


def dim(tgt, L):
    return 2 + 4 * (L - 1) if tgt.kind == 0 else tgt.d


def evaluate(tgt, x, L=4, eps=1e-8, grad=False, info=False):
    """f [M,3], log p [M], pixel [M], optional grad log p [M,d], optional
    path info [M, stride]."""
    d = dim(tgt, L)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, d)
    M = x.shape[0]
    f = np.zeros((M, 3))
    lp = np.zeros(M)
    pix = np.zeros(M, np.int32)
    g = np.zeros((M, d)) if grad else None
    inf = np.zeros((M, lib().orc_info_stride()), np.int32) if info else None
    lib().orc_eval(tgt.h, tgt.kind, int(L), x.ravel(), M, float(eps), _ptr(f), _ptr(lp), _ptr(g), _ptr(pix),
                   _ptr(inf))
    out = {"f": f, "logp": lp, "pix": pix}
    if grad:
        out["grad"] = g
    if info:
        out["info"] = inf
    return out


def fd_score(tgt, x, L=4, eps=1e-8, h=1e-3):
    d = dim(tgt, L)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, d)
    s = np.zeros_like(x)
    lib().orc_fd_score(tgt.h, tgt.kind, int(L), x.ravel(), x.shape[0], float(eps), float(h), s.ravel())
    return s


def bsdf_sample(mat, n, wo, u1, u2):
    wi = np.zeros(3)
    w = np.zeros(3)
    pdf = np.zeros(1)
    lobe = np.zeros(1, np.int32)
    ok = lib().orc_bsdf_sample(np.ascontiguousarray(mat, np.float32), np.ascontiguousarray(n, np.float64),
                               np.ascontiguousarray(wo, np.float64), float(u1), float(u2), wi, w, pdf, lobe)
    return bool(ok), wi, w, float(pdf[0]), int(lobe[0])


def bsdf_eval(mat, n, wo, wi):
    fs = np.zeros(3)
    pdf = np.zeros(1)
    lib().orc_bsdf_eval(np.ascontiguousarray(mat, np.float32), np.ascontiguousarray(n, np.float64),
                        np.ascontiguousarray(wo, np.float64), np.ascontiguousarray(wi, np.float64), fs, pdf)
    return fs, float(pdf[0])


def local_dynamics(x, score, stddev, gamma_tilde, seed, frame, step, chain):
    x = np.ascontiguousarray(x, np.float64)
    score = np.ascontiguousarray(score, np.float64)
    out = np.zeros_like(x)
    lib().orc_local_dynamics(np.array([stddev, gamma_tilde], np.float64), int(seed), int(frame), int(step),
                             int(chain), x.size, x, score, out)
    return out


def restore_run(tgt, params, seed, chain_ids, n_steps, frame=0, record=True, info=False, accum=True):
    """Runs Alg. 1 + n_steps x Alg. 2 for the given chains.  Returns a dict of
    per-step arrays ([n_steps + 1, M, ...]) when ``record``, plus the FP64
    accumulation image, tour count and the init-pass sum of p."""
    d = dim(tgt, params.L)
    ids = np.ascontiguousarray(chain_ids, np.uint32)
    M = ids.size
    T = n_steps + 1
    out = {}
    if record:
        out["x"] = np.zeros((T, M, d))
        out["logp"] = np.zeros((T, M))
        out["score"] = np.zeros((T, M, d))
        out["killed"] = np.zeros((T, M), np.uint8)
        out["pix"] = np.zeros((T, M), np.int32)
        out["val"] = np.zeros((T, M, 3))
    if info:
        out["info"] = np.zeros((T, M, lib().orc_info_stride()), np.int32)
    acc = np.zeros((tgt.width * tgt.height, 3)) if accum else None
    tc = np.zeros(1, np.uint64)
    ps = np.zeros(1, np.float64)
    g = out.get
    lib().orc_restore_run(tgt.h, tgt.kind, C.byref(params), int(seed), int(frame), ids, M, int(n_steps),
                          _ptr(g("x")), _ptr(g("logp")), _ptr(g("score")), _ptr(g("killed")), _ptr(g("pix")),
                          _ptr(g("val")), _ptr(g("info")), _ptr(acc), _ptr(tc), _ptr(ps))
    out["accum"] = acc
    out["tour_count"] = int(tc[0])
    out["p_init_sum"] = float(ps[0])
    return out


def restore_tours(tgt, params, seed, chain_ids, max_steps=1 << 20, frame=0, image=False):
    """One complete tour per chain id (start at a regeneration, run until the
    first kill).  Returns per-tour I1, Ix, Ixx, steps, truncated and, with
    ``image``, the FP64 sum of weight * f / p over all tours."""
    d = dim(tgt, params.L)
    ids = np.ascontiguousarray(chain_ids, np.uint32)
    M = ids.size
    I1 = np.zeros(M)
    Ix = np.zeros((M, d))
    Ixx = np.zeros((M, d, d))
    steps = np.zeros(M, np.int64)
    tr = np.zeros(M, np.uint8)
    acc = np.zeros((tgt.width * tgt.height, 3)) if image else None
    lib().orc_restore_tours(tgt.h, tgt.kind, C.byref(params), int(seed), int(frame), ids, M, int(max_steps),
                            I1, Ix.ravel(), Ixx.ravel(), steps, tr, _ptr(acc))
    return {"I1": I1, "Ix": Ix, "Ixx": Ixx, "steps": steps, "truncated": tr, "accum": acc}


def resolve(accum, k0, tour_count):
    """Alg. 3: out = k0 / tourCount * accum."""
    if tour_count == 0:
        return np.zeros_like(accum)
    return accum * (k0 / tour_count)


def pt_image(scene_tgt, L, spp, seed=7):
    n = scene_tgt.width * scene_tgt.height
    mean = np.zeros((n, 3))
    var = np.zeros((n, 3))
    lib().orc_pt_image(scene_tgt.h, int(L), int(spp), int(seed), mean, var)
    return mean, var


def rel_mse(img, ref, floor=1e-2):
    """relMSE = mean over pixels and channels of (I - R)^2 / (R^2 + floor)."""
    img = np.asarray(img, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.mean((img - ref) ** 2 / (ref ** 2 + floor)))
