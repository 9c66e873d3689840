"""Torch-facing wrapper of the C ABI: device tensors in, device tensors out.

PyTorch provides device memory and the CUDA stream; all computation runs in
``libdiffrestore.so``.  ``LogPFunction`` exposes x -> log p as an autograd
function whose backward uses the library's hand-written adjoint kernel.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import call, dr_params

DRIFT = {"none": _lib.DR_DRIFT_NONE, "fd": _lib.DR_DRIFT_FD, "adjoint": _lib.DR_DRIFT_ADJOINT,
         "mala": _lib.DR_DRIFT_MALA}


def make_params(L=4, drift="adjoint", rb=True, stddev=5e-3, dt=1e-5, gamma_tilde=None, eps=1e-8, fd_h=1e-3, m=64.0,
                k0=0.0, steps_per_splat=16):
    """Diffusion Restore parameters (Sec. 5.3 and Sec. 6).  gamma_tilde
    defaults to stddev^2 / 2 (gamma = sigma^2); k0 <= 0 means estimate
    p_lambda from the initial samples and set k0 = p_lambda / (m dt)."""
    if gamma_tilde is None:
        gamma_tilde = 0.5 * stddev * stddev
    return dr_params(int(L), DRIFT[drift] if isinstance(drift, str) else int(drift), int(bool(rb)),
                     int(steps_per_splat), float(stddev), float(dt), float(gamma_tilde), float(eps), float(fd_h),
                     float(m), float(k0))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data_as(C.c_void_p)
    assert t.is_contiguous()
    return C.c_void_p(t.data_ptr())


class Renderer:
    """One library context on one CUDA device."""

    def __init__(self, device=0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("Renderer needs a CUDA device (the library has no CPU path)")
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = C.c_void_p()
        call("dr_create", C.byref(h), int(device), C.c_void_p(stream.cuda_stream))
        self.h = h
        self.width = self.height = 0
        self.d = 0
        self.N = 0
        self.L = 0

    def close(self):
        if getattr(self, "h", None):
            _lib.load().dr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- inputs
    def set_option(self, option, value):
        """option: "wavefront" (-1 auto / 0 / 1), "work_order" (0/1), "profile" (0/1) or
        "bvh_width" (0 automatic / 2 / 4 / 8; 8 before the upload), "traverse_blocks" (0 = all resident),
        "refill" (1..32), "ray_order" (-1 automatic / 0 / 1), "tail_bounce" (-1 automatic, 0 off, k) or
        "two_level" (1: walk an instanced scene's two-level BVH, 0: its flattened BVH)."""
        code = {"work_order": _lib.DR_OPT_WORK_ORDER, "wavefront": _lib.DR_OPT_WAVEFRONT,
                "profile": _lib.DR_OPT_PROFILE, "bvh_width": _lib.DR_OPT_BVH_WIDTH,
                "traverse_blocks": _lib.DR_OPT_TRAVERSE_BLOCKS, "refill": _lib.DR_OPT_REFILL,
                "ray_order": _lib.DR_OPT_RAY_ORDER, "tail_bounce": _lib.DR_OPT_TAIL_BOUNCE,
                "two_level": _lib.DR_OPT_TWO_LEVEL}[option]
        call("dr_set_option", self.h, code, int(value))

    def set_bvh_builder(self, builder="ploc", radius=16):
        call("dr_set_bvh_builder", self.h, _lib.DR_BVH_PLOC if builder == "ploc" else _lib.DR_BVH_LBVH, int(radius))

    def upload_scene(self, scene):
        v = np.ascontiguousarray(scene.verts, np.float32)
        t = np.ascontiguousarray(scene.tris, np.int32)
        n = None if scene.normals is None else np.ascontiguousarray(scene.normals, np.float32)
        tm = np.ascontiguousarray(scene.tri_mat, np.int32)
        m = np.ascontiguousarray(scene.materials, np.float32)
        cam = np.ascontiguousarray(scene.camera, np.float32)
        call("dr_scene_upload", self.h, _ptr(v), v.shape[0], _ptr(t), _ptr(n), t.shape[0], _ptr(tm), _ptr(m),
             m.shape[0], _ptr(cam), int(scene.width), int(scene.height))
        self.width, self.height = int(scene.width), int(scene.height)
        self.kind = 0

    def upload_instanced(self, iscene):
        """An instanced scene (scenes.InstancedScene): meshes placed by affine
        maps; the library flattens it (the scene it renders) and, with two or
        more instances, builds a two-level BVH as well."""
        keep = []
        meshes = (_lib.dr_mesh_desc * len(iscene.meshes))()
        for i, mesh in enumerate(iscene.meshes):
            v = np.ascontiguousarray(mesh.verts, np.float32)
            t = np.ascontiguousarray(mesh.tris, np.int32)
            nr = None if mesh.normals is None else np.ascontiguousarray(mesh.normals, np.float32)
            tm = np.ascontiguousarray(mesh.tri_mat, np.int32)
            keep += [v, t, nr, tm]
            meshes[i] = _lib.dr_mesh_desc(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0],
                                          None if nr is None else nr.ctypes.data, tm.ctypes.data)
        insts = (_lib.dr_instance_desc * len(iscene.instances))()
        for i, (mesh, mat, xf) in enumerate(iscene.instances):
            insts[i] = _lib.dr_instance_desc(int(mesh), int(mat),
                                             (C.c_float * 12)(*np.asarray(xf, np.float32).ravel().tolist()))
        m = np.ascontiguousarray(iscene.materials, np.float32)
        cam = np.ascontiguousarray(iscene.camera, np.float32)
        call("dr_scene_upload_instanced", self.h, meshes, len(iscene.meshes), insts, len(iscene.instances),
             _ptr(m), m.shape[0], _ptr(cam), int(iscene.width), int(iscene.height))
        self.width, self.height = int(iscene.width), int(iscene.height)
        self.kind = 0
        del keep

    def two_level_info(self):
        """Instances, TLAS nodes and BLAS nodes of the two-level BVH, or None."""
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        r = _lib.load().dr_two_level_info(self.h, C.byref(a), C.byref(b), C.byref(c))
        if r == _lib.DR_ERR_STATE:
            return None
        _lib.check(r, "dr_two_level_info")
        return {"n_instances": a.value, "n_tlas_nodes": b.value, "n_blas_nodes": c.value}

    def upload_scenes(self, items):
        """A multi-scene batch: items = [(scene, max_path_len, n_chains), ...].
        Afterwards init_chains(sum of n_chains, ...) with adjoint drift, step /
        frame as usual, and resolve_scene(s) per scene."""
        keep = []
        descs = (_lib.dr_scene_desc * len(items))()
        for i, (scene, L, n) in enumerate(items):
            v = np.ascontiguousarray(scene.verts, np.float32)
            t = np.ascontiguousarray(scene.tris, np.int32)
            nr = None if scene.normals is None else np.ascontiguousarray(scene.normals, np.float32)
            tm = np.ascontiguousarray(scene.tri_mat, np.int32)
            m = np.ascontiguousarray(scene.materials, np.float32)
            cam = np.ascontiguousarray(scene.camera, np.float32)
            keep += [v, t, nr, tm, m, cam]
            descs[i] = _lib.dr_scene_desc(v.ctypes.data, v.shape[0], t.ctypes.data,
                                          None if nr is None else nr.ctypes.data, t.shape[0], tm.ctypes.data,
                                          m.ctypes.data, m.shape[0], cam.ctypes.data, int(scene.width),
                                          int(scene.height), int(L), int(n))
        call("dr_scenes_upload_batch", self.h, descs, len(items))
        self.batch = [(int(sc.width), int(sc.height), int(L), int(n)) for sc, L, n in items]
        self.width, self.height = sum(w * h for w, h, _, _ in self.batch), 1  # the shared accumulator
        self.kind = 2
        del keep

    def resolve_scene(self, s, out=None):
        w, h = self.batch[s][0], self.batch[s][1]
        if out is None:
            out = torch.empty((h, w, 3), dtype=torch.float32, device=self.device)
        call("dr_resolve_scene", self.h, int(s), _ptr(out))
        return out

    def scene_counters(self, s):
        tc, k0 = C.c_uint64(), C.c_double()
        call("dr_get_scene_counters", self.h, int(s), C.byref(tc), C.byref(k0))
        return {"tour_count": tc.value, "k0": k0.value}

    def set_mixture(self, mix):
        w = np.ascontiguousarray(mix.w, np.float32).reshape(-1)
        mu = np.ascontiguousarray(mix.mu, np.float32).reshape(-1)
        sig = np.ascontiguousarray(mix.sig, np.float32).reshape(-1)
        call("dr_target_mixture", self.h, int(mix.d), int(mix.K), _ptr(w) if w.size else None,
             _ptr(mu) if mu.size else None, _ptr(sig) if sig.size else None, float(mix.const), int(mix.width),
             int(mix.height))
        self.width, self.height = int(mix.width), int(mix.height)
        self.kind = 1
        self.mix_d = int(mix.d)

    # ---------------------------------------------------------------- chains
    def init_chains(self, n_chains, seed, params, frame=0):
        self.params = params
        call("dr_chains_init", self.h, int(n_chains), int(seed), int(frame), C.byref(params))
        self._sync_shape()

    def step(self, n=1):
        call("dr_step", self.h, int(n))

    def splat(self):
        call("dr_splat", self.h)

    def frame(self, n_steps):
        """n_steps steps + splat as one replayed CUDA graph (needs a renderer
        created on a non-default torch stream)."""
        call("dr_frame", self.h, int(n_steps))

    def bounce_profile(self, n_bounces):
        """Per-bounce milliseconds of the trace / shade / shadow passes, and the
        closest-hit and shadow rays of each bounce, since the last profile()
        call: dict of five lists of n_bounces values."""
        ms = (C.c_double * (3 * n_bounces))()
        call("dr_get_bounce_profile", self.h, ms, int(n_bounces))
        v = list(ms)
        rays = (C.c_uint64 * (2 * n_bounces))()
        call("dr_get_bounce_rays", self.h, rays, int(n_bounces))
        n = list(rays)
        return {"trace": v[:n_bounces], "shade": v[n_bounces:2 * n_bounces], "shadow": v[2 * n_bounces:],
                "rays": n[:n_bounces], "shadow_rays": n[n_bounces:]}

    def profile(self):
        """Per-phase device milliseconds since the last call (DR_OPT_PROFILE)."""
        ms = (C.c_double * _lib.DR_PHASES)()
        cnt = (C.c_uint64 * _lib.DR_PHASES)()
        call("dr_get_profile", self.h, ms, cnt, _lib.DR_PHASES)
        return {n: (ms[i], cnt[i]) for i, n in enumerate(_lib.PHASE_NAMES)}

    def resolve(self, out=None):
        if out is None:
            out = torch.empty((self.height, self.width, 3), dtype=torch.float32, device=self.device)
        call("dr_resolve", self.h, _ptr(out))
        return out

    def clear_image(self):
        call("dr_clear_image", self.h)

    def readback_state(self, fields=("x", "score", "killed", "logp", "pix", "val")):
        N, d = self.N, self.d
        out = {}
        bufs = {
            "x": np.zeros((N, d), np.float32) if "x" in fields else None,
            "score": np.zeros((N, d), np.float32) if "score" in fields else None,
            "killed": np.zeros(N, np.uint8) if "killed" in fields else None,
            "logp": np.zeros(N, np.float32) if "logp" in fields else None,
            "pix": np.zeros(N, np.int32) if "pix" in fields else None,
            "val": np.zeros((N, 3), np.float32) if "val" in fields else None,
        }
        call("dr_readback_state", self.h, *[_ptr(bufs[k]) for k in ("x", "score", "killed", "logp", "pix", "val")])
        for k, v in bufs.items():
            if v is not None:
                out[k] = v
        return out

    def readback_accum(self):
        a = np.zeros((self.width * self.height, 3), np.float64)
        call("dr_readback_accum", self.h, _ptr(a))
        return a

    def p_sum(self):
        """(sum of p over the initial samples, their count) of the last
        init that estimated p_lambda."""
        ps, n = C.c_double(), C.c_uint64()
        call("dr_get_p_sum", self.h, C.byref(ps), C.byref(n))
        return ps.value, n.value

    def k0_from_p_sum(self, p_sum, n, params):
        return k0_from_p_sum(p_sum, n, params)

    def counters(self):
        tc, st, rays = C.c_uint64(), C.c_uint64(), C.c_uint64()
        k0, pl = C.c_double(), C.c_double()
        call("dr_get_counters", self.h, C.byref(tc), C.byref(k0), C.byref(st), C.byref(rays), C.byref(pl))
        return {"tour_count": tc.value, "k0": k0.value, "steps": st.value, "rays": rays.value, "p_lambda": pl.value}

    def set_stats(self, enable=True):
        call("dr_set_stats", self.h, int(bool(enable)))

    def traversal_stats(self):
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        call("dr_get_traversal_stats", self.h, C.byref(a), C.byref(b), C.byref(c))
        return {"node_visits": a.value, "tri_tests": b.value, "rays": c.value}

    def bvh_info(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        call("dr_bvh_info", self.h, C.byref(a), C.byref(b), C.byref(c))
        return {"n_nodes": a.value, "n_tris": b.value, "max_depth": c.value}

    def bvh4_info(self):
        """The 4-wide BVH's node count, depth and traversal-stack need, or None when the scene has none."""
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        r = _lib.load().dr_bvh4_info(self.h, C.byref(a), C.byref(b), C.byref(c))
        if r == _lib.DR_ERR_STATE:
            return None
        _lib.check(r, "dr_bvh4_info")
        return {"n_nodes": a.value, "max_depth": b.value, "stack_need": c.value}

    def bvh4_sah(self):
        """SAH cost of the 4-wide BVH: expected node steps and triangle tests of a ray hitting the root box."""
        a, b = C.c_double(), C.c_double()
        r = _lib.load().dr_bvh4_sah(self.h, C.byref(a), C.byref(b))
        if r == _lib.DR_ERR_STATE:
            return None
        _lib.check(r, "dr_bvh4_sah")
        return {"node_steps": a.value, "tri_tests": b.value}

    def bvh8_info(self):
        """The 8-wide compressed BVH's node count and depth, or None when the scene has none."""
        a, b = C.c_int32(), C.c_int32()
        r = _lib.load().dr_bvh8_info(self.h, C.byref(a), C.byref(b))
        if r == _lib.DR_ERR_STATE:
            return None
        _lib.check(r, "dr_bvh8_info")
        return {"n_nodes": a.value, "max_depth": b.value}

    def launch_count(self):
        n = C.c_uint64()
        call("dr_get_launch_count", self.h, C.byref(n))
        return n.value

    def state_save(self):
        n = C.c_size_t(0)
        call("dr_state_save", self.h, None, C.byref(n))
        buf = np.zeros(n.value, np.uint8)
        call("dr_state_save", self.h, _ptr(buf), C.byref(n))
        return buf

    def state_load(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        call("dr_state_load", self.h, _ptr(buf), buf.size)
        self._sync_shape()

    def _sync_shape(self):
        n, d, L = C.c_uint64(), C.c_int32(), C.c_int32()
        call("dr_get_chain_shape", self.h, C.byref(n), C.byref(d), C.byref(L))
        self.N, self.d, self.L = n.value, d.value, L.value

    # ---------------------------------------------------------------- queries
    def eval_logp(self, x, L=None, grad=False, want_f=False):
        """x: float32 CUDA tensor [M, d]. Returns (logp [M], grad [M, d] or
        None, pix [M], f [M, 3] or None)."""
        L = self.L if L is None else int(L)
        x = x.contiguous()
        M = x.shape[0]
        logp = torch.empty(M, dtype=torch.float32, device=x.device)
        g = torch.empty_like(x) if grad else None
        pix = torch.empty(M, dtype=torch.int32, device=x.device)
        f = torch.empty((M, 3), dtype=torch.float32, device=x.device) if want_f else None
        call("dr_eval_logp", self.h, int(L), _ptr(x), int(M), _ptr(logp), _ptr(g), _ptr(pix), _ptr(f))
        return logp, g, pix, f

    def lstar_over_p(self, y, params, radius=8.0, n=129):
        """(L* p / p)(y) of the 2-D mixture target at query points y (float32
        CUDA tensor [M, 2]); FP64 CUDA tensor [M]."""
        y = y.contiguous()
        out = torch.empty(y.shape[0], dtype=torch.float64, device=y.device)
        call("dr_lstar_over_p", self.h, C.byref(params), _ptr(y), int(y.shape[0]), float(radius), int(n), _ptr(out))
        return out

    def pt_render(self, L, spp, seed=7):
        """Stratified path-traced image [H, W, 3] (FP64 CUDA tensor) of the
        uploaded scene, in the units of resolve()."""
        out = torch.empty((self.height, self.width, 3), dtype=torch.float64, device=self.device)
        call("dr_pt_render", self.h, int(L), int(spp), int(seed), _ptr(out))
        return out

    def trace_closest(self, rays, exclude=-1):
        rays = rays.contiguous()
        n = rays.shape[0]
        tri = torch.empty(n, dtype=torch.int32, device=rays.device)
        t = torch.empty(n, dtype=torch.float32, device=rays.device)
        call("dr_trace_closest", self.h, _ptr(rays), int(n), int(exclude), _ptr(tri), _ptr(t))
        return tri, t

    def trace_closest_counted(self, rays, exclude=-1):
        """trace_closest plus each ray's node steps and triangle tests."""
        rays = rays.contiguous()
        n = rays.shape[0]
        tri = torch.empty(n, dtype=torch.int32, device=rays.device)
        t = torch.empty(n, dtype=torch.float32, device=rays.device)
        nodes = torch.empty(n, dtype=torch.int32, device=rays.device)
        tests = torch.empty(n, dtype=torch.int32, device=rays.device)
        call("dr_trace_closest_counted", self.h, _ptr(rays), int(n), int(exclude), _ptr(tri), _ptr(t), _ptr(nodes),
             _ptr(tests))
        return tri, t, nodes, tests

    def bvh4_download(self):
        """The 4-wide BVH on the host: nodes float32 [n, 28] and triangles
        float32 [n_tris, 12] (layouts in the C header)."""
        import numpy as np
        n4 = self.bvh4_info()["n_nodes"]
        nt = self.bvh_info()["n_tris"]
        nodes = np.empty((n4, 28), np.float32)
        tris = np.empty((nt, 12), np.float32)
        call("dr_bvh4_download", self.h, nodes.ctypes.data, tris.ctypes.data)
        return nodes, tris

    def splat_records(self, recs):
        """recs: CUDA tensor of 16-byte records viewed as int32 [M, 4] (pixel
        index, then float bits of r, g, b)."""
        recs = recs.contiguous()
        call("dr_splat_records", self.h, _ptr(recs), int(recs.shape[0]))


def k0_from_p_sum(p_sum, n, params):
    """k0 = (p_sum / n) / (m dt) computed by the library (Eq.
    killing-rate-constant)."""
    k0 = C.c_double()
    call("dr_k0_from_p_sum", float(p_sum), int(n), C.byref(params), C.byref(k0))
    return k0.value


def resolve_accum(accum, tour_count, k0, stream=None):
    """Resolve (Alg. 3) of an FP64 CUDA tensor by the library: k0 /
    tour_count * accum as FP32 (zeros when tour_count is 0)."""
    accum = accum.contiguous()
    out = torch.empty(accum.shape, dtype=torch.float32, device=accum.device)
    s = stream if stream is not None else torch.cuda.current_stream(accum.device)
    code = _lib.load().dr_resolve_accum(_ptr(accum), int(accum.numel()), int(tour_count), float(k0), _ptr(out),
                                        C.c_void_p(s.cuda_stream))
    if not (code == _lib.DR_ERR_STATE and int(tour_count) == 0):
        _lib.check(code, "dr_resolve_accum")
    return out


def philox(ctr, key, stream=None):
    """ctr uint32 [n, 4], key uint32 [n, 2] as int32 CUDA tensors -> [n, 4]."""
    out = torch.empty_like(ctr)
    s = stream if stream is not None else torch.cuda.current_stream(ctr.device)
    call("dr_philox", _ptr(ctr.contiguous()), _ptr(key.contiguous()), _ptr(out), int(ctr.shape[0]),
         C.c_void_p(s.cuda_stream))
    return out


class LogPFunction(torch.autograd.Function):
    """x [M, d] (CUDA float32) -> log p(x) [M] through the library; the
    backward recomputes the paths and applies the hand-written adjoint
    (grad log p), scaled by the incoming gradient."""

    @staticmethod
    def forward(ctx, x, renderer, L):
        logp, _, _, _ = renderer.eval_logp(x.detach(), L=L, grad=False)
        ctx.save_for_backward(x)
        ctx.renderer = renderer
        ctx.L = L
        return logp

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        _, grad, _, _ = ctx.renderer.eval_logp(x.detach(), L=ctx.L, grad=True)
        return grad * g.unsqueeze(1), None, None
