"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle
on the same seeded inputs and the same Philox4x32-10 streams.

Tolerances (FP32 kernels vs FP64 oracle):
* Philox, splat reduction (same records): bit-exact.
* Closest-hit triangle ids: identical except on edge/tie cases, where the
  two distances must agree to 1e-4 relative.
* Chain state over 16-step horizons: torus distance of x <= 1e-4,
  |log p difference| <= 1e-4 max(1, |log p|), splat values within 1e-4
  relative, kill flags and pixels identical.  A chain whose discrete choices
  differ (kill, pixel, or an x jump beyond tolerance after an edge crossing)
  is counted as divergent from that step on; the divergent fraction is
  bounded.
* grad log p (hand-written adjoint, FP32) vs the oracle's dual-number
  gradient: relative L2 error <= 1e-4 on >= 99% of points with f > 0 whose
  log p agrees; vs FP64 central differences (h = 1e-6, discrete choices held
  equal): <= 1e-4 relative on >= 99% of such points.
* The stored score of surviving chains: 1e-4 relative for the exact drift;
  for FP32 finite differences, plus the rounding of log p divided by h.
"""
import math

import numpy as np
import pytest

from paper_2605_08916_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    return T


@pytest.fixture(scope="module")
def R(torch):
    from paper_2605_08916_gb300 import renderer
    return renderer


def torus_dist(a, b):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return np.abs(d - np.round(d))


def test_philox_bit_exact(torch, R, oracle):
    rng = np.random.default_rng(1)
    n = 8192
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    g = R.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), torch.from_numpy(key.view(np.int32)).cuda())
    torch.cuda.synchronize()
    mine = g.cpu().numpy().view(np.uint32)
    assert np.array_equal(mine, oracle.philox4x32_10(ctr, key))


def hit_scene(which):
    if which == "cornell":
        return S.cornell_box(1, 16, 16)
    if which == "caustic":
        return S.caustic_scene(1, 16, 16, n_theta=40, n_phi=40)
    return S.procedural_scene(1, 32, 18, target_tris=30000, n_objects=40)


def random_rays(scene, n, seed):
    lo, hi = scene.verts.min(0), scene.verts.max(0)
    rng = np.random.default_rng(seed)
    o = (lo + (hi - lo) * rng.uniform(0.05, 0.95, (n, 3))).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


@pytest.mark.parametrize("width", [2, 4, 8])
@pytest.mark.parametrize("builder", ["ploc", "lbvh"])
@pytest.mark.parametrize("which", ["cornell", "caustic", "procedural"])
def test_closest_hit_matches_oracle(torch, R, oracle, which, builder, width):
    scene = hit_scene(which)
    r = R.Renderer()
    r.set_bvh_builder(builder)
    r.set_option("bvh_width", width)
    r.upload_scene(scene)
    info = r.bvh_info()
    assert info["n_tris"] == scene.n_tris and info["max_depth"] < 48
    info4 = r.bvh4_info()
    assert info4 is not None and info4["stack_need"] <= 48
    assert info4["n_nodes"] < info["n_nodes"] and info4["max_depth"] < info["max_depth"]
    info8 = r.bvh8_info()
    if width == 8:
        assert info8 is not None and info8["n_nodes"] < info4["n_nodes"] and info8["max_depth"] <= info4["max_depth"]
    else:
        assert info8 is None
    tgt = oracle.OracleScene(scene)
    n = 20000
    o, d = random_rays(scene, n, 2)
    rays = torch.from_numpy(np.concatenate([o, d], 1)).cuda()
    tri_g, t_g = r.trace_closest(rays)
    torch.cuda.synchronize()
    tri_g, t_g = tri_g.cpu().numpy(), t_g.cpu().numpy()
    tri_o, t_o = tgt.trace(o.astype(np.float64), d.astype(np.float64))
    same = tri_g == tri_o
    assert same.mean() > 0.999, same.mean()
    bad = ~same
    both = bad & (tri_g >= 0) & (tri_o >= 0)
    assert np.all(np.abs(t_g[both] - t_o[both]) <= 1e-4 * np.maximum(1.0, t_o[both]))
    hit = same & (tri_o >= 0)
    assert np.allclose(t_g[hit], t_o[hit], rtol=1e-4, atol=1e-5)
    r.close()


@pytest.mark.parametrize("which", ["cornell", "caustic", "procedural"])
def test_bvh_widths_return_the_same_hits(torch, R, which):
    """The 4-wide and 8-wide BVHs regroup the binary one's boxes (the 8-wide
    widened to its 8-bit grid) and triangles: the closest hit (ties to the
    smaller id) and its distance come from the same triangle test on the
    same data, so they agree bitwise."""
    scene = hit_scene(which)
    o, d = random_rays(scene, 50000, 3)
    rays = torch.from_numpy(np.concatenate([o, d], 1)).cuda()
    out = []
    for width in (2, 4, 8):
        r = R.Renderer()
        r.set_option("bvh_width", width)
        r.upload_scene(scene)
        tri, t = r.trace_closest(rays)
        torch.cuda.synchronize()
        out.append((tri.cpu().numpy(), t.cpu().numpy()))
        r.close()
    (a, ta) = out[0]
    for b, tb in out[1:]:
        assert (a == b).mean() >= 0.9999
        same = a == b
        assert np.array_equal(ta[same], tb[same])


def test_bvh4_sah_cost_closed_form(torch, R):
    """Two unit right triangles 5 apart in the z = 0 plane: the 4-wide root
    holds the two one-triangle leaves, so the SAH cost is one node step and
    (2 + 2) / 12 triangle tests (leaf box areas 2 over a 6 x 1 root box).
    A large scene's cost is finite, positive and consistent with its tree."""
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [5, 0, 0], [6, 0, 0], [5, 1, 0]], np.float32)
    tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    mats = np.stack([S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))])
    cam = np.array([3, 0.5, 5, 3, 0.5, 0, 0, 1, 0, 40], np.float32)
    r = R.Renderer()
    r.upload_scene(S.Scene(verts, tris, np.zeros(2, np.int32), mats, cam, 8, 8))
    sah = r.bvh4_sah()
    assert abs(sah["node_steps"] - 1.0) < 1e-12
    assert abs(sah["tri_tests"] - 4.0 / 12.0) < 1e-7
    r.upload_scene(hit_scene("procedural"))
    sah = r.bvh4_sah()
    info = r.bvh4_info()
    assert 1.0 < sah["node_steps"] < info["n_nodes"] and 0.0 < sah["tri_tests"] < 4.0 * info["n_nodes"]
    r.close()


def test_one_triangle_scene_keeps_the_binary_bvh(torch, R):
    scene = S.cornell_box(1, 8, 8)
    keep = np.zeros(scene.n_tris, bool)
    keep[0] = True
    one = S.Scene(verts=scene.verts, tris=np.ascontiguousarray(scene.tris[keep]),
                  tri_mat=np.ascontiguousarray(scene.tri_mat[keep]), materials=scene.materials,
                  camera=scene.camera, width=8, height=8, normals=scene.normals).check()
    r = R.Renderer()
    r.upload_scene(one)
    assert r.bvh4_info() is None
    v = scene.verts[scene.tris[0]].astype(np.float64)
    centre = v.mean(0)
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    nrm /= np.linalg.norm(nrm)
    o = centre + nrm
    rays = torch.tensor([np.concatenate([o, -nrm])], dtype=torch.float32).cuda()
    tri, t = r.trace_closest(rays)
    torch.cuda.synchronize()
    assert int(tri.cpu()[0]) == 0 and abs(float(t.cpu()[0]) - 1.0) < 1e-4
    r.close()


def _soup(tri_verts, seed):
    """A scene of the given triangles ([nt, 3, 3]) under one diffuse material."""
    nt = len(tri_verts)
    verts = np.ascontiguousarray(tri_verts.reshape(-1, 3), dtype=np.float32)
    tris = np.arange(3 * nt, dtype=np.int32).reshape(nt, 3)
    mats = np.stack([S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))])
    cam = np.array([0.5, 0.5, 4, 0.5, 0.5, 0, 0, 1, 0, 40], np.float32)
    return S.Scene(verts, tris, np.zeros(nt, np.int32), mats, cam, 8, 8, name=f"soup{seed}")


@pytest.mark.parametrize("builder", ["ploc", "lbvh"])
def test_bvh_builds_on_tiny_and_degenerate_scenes(torch, R, oracle, builder):
    """Both builders make a tree over every triangle of tiny scenes (2, 3 and
    5 triangles) and of scenes full of exact ties: 300 copies of one
    triangle beside 20 others, and a grid of equal triangles.  On the
    copies, clustering finds every cluster's nearest neighbour in the same
    cluster, merges one pair per pass and would build a chain some 300
    levels tall: the builder then falls back to the linear BVH, so the tree
    stays within the traversal stack.  Closest hits match the oracle's brute
    force (ties to the smaller id on both sides)."""
    rng = np.random.default_rng(11)

    def rand_tris(n):
        c = rng.uniform(0.0, 1.0, (n, 1, 3))
        return c + rng.uniform(-0.08, 0.08, (n, 3, 3))

    one = np.array([[0.2, 0.2, 0.3], [0.8, 0.25, 0.35], [0.4, 0.8, 0.3]])
    gx, gy = np.meshgrid(np.arange(40) / 40.0, np.arange(40) / 40.0)
    cell = np.array([[0.0, 0.0, 0.0], [0.02, 0.0, 0.0], [0.0, 0.02, 0.0]])
    grid = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 0.5)], 1)[:, None, :] + cell[None]
    cases = [rand_tris(2), rand_tris(3), rand_tris(5),
             np.concatenate([np.repeat(one[None], 300, 0), rand_tris(20)]), grid]
    r = R.Renderer()
    r.set_bvh_builder(builder)
    for k, tv in enumerate(cases):
        scene = _soup(tv, k)
        # 3000 rays aimed at random points of random triangles, 1000 random
        n_aim = 3000
        w = rng.dirichlet(np.ones(3), n_aim)
        target = np.einsum("nk,nkc->nc", w, tv[rng.integers(0, len(tv), n_aim)])
        o = rng.uniform(-0.5, 1.5, (n_aim + 1000, 3))
        d = np.concatenate([target - o[:n_aim], rng.normal(size=(1000, 3))])
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        o, d = o.astype(np.float32), d.astype(np.float32)
        rays = torch.from_numpy(np.concatenate([o, d], 1)).cuda()
        r.upload_scene(scene)
        info = r.bvh_info()
        assert info["n_tris"] == scene.n_tris and info["max_depth"] <= 49, (k, info)
        tri_g, t_g = r.trace_closest(rays)
        torch.cuda.synchronize()
        tri_g, t_g = tri_g.cpu().numpy(), t_g.cpu().numpy()
        tri_o, t_o = oracle.OracleScene(scene).trace(o.astype(np.float64), d.astype(np.float64))
        same = tri_g == tri_o
        assert same.mean() > 0.999, (k, same.mean())
        assert (tri_o >= 0).sum() > 1000, k
        # distances of hits that are not grazing (an FP32 hit distance loses
        # relative accuracy as 1 / |cos| of the angle to the plane)
        hit = same & (tri_o >= 0)
        nrm = np.cross(tv[:, 1] - tv[:, 0], tv[:, 2] - tv[:, 0])
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        steep = hit.copy()
        steep[hit] = np.abs(np.einsum("ij,ij->i", d[hit], nrm[tri_o[hit]])) >= 0.05
        assert steep.sum() > 0.8 * hit.sum(), k
        assert np.allclose(t_g[steep], t_o[steep], rtol=1e-4, atol=1e-5), k
    r.close()


EVAL_CASES = {
    "cornell-L4": (lambda: S.cornell_box(1, 64, 64), 4),
    "glossy-L8": (lambda: S.cornell_box(1, 256, 256, glossy=True), 8),
    "conductor-L8": (lambda: S.cornell_box(1, 256, 256, metal=True), 8),
    "caustic-L6": (lambda: S.caustic_scene(1, 64, 64, n_theta=24, n_phi=24), 6),
}


@pytest.mark.parametrize("case", list(EVAL_CASES))
def test_eval_logp_and_adjoint_match_oracle(torch, R, oracle, case):
    make, L = EVAL_CASES[case]
    scene = make()
    d = S.pss_dim(L)
    r = R.Renderer()
    r.upload_scene(scene)
    rng = np.random.default_rng(3)
    M = 3000
    x = rng.random((M, d)).astype(np.float32)
    lp, g, pix, f = r.eval_logp(torch.from_numpy(x).cuda(), L=L, grad=True, want_f=True)
    torch.cuda.synchronize()
    lp, g, pix, f = lp.cpu().numpy(), g.cpu().numpy(), pix.cpu().numpy(), f.cpu().numpy()
    ro = oracle.evaluate(oracle.OracleScene(scene), x.astype(np.float64), L, grad=True)
    assert np.array_equal(pix, ro["pix"])
    lit = ro["f"].sum(1) > 0
    assert lit.mean() > 0.03
    ok_lp = np.abs(lp - ro["logp"]) <= 1e-4 * np.maximum(1.0, np.abs(ro["logp"]))
    assert ok_lp.mean() > 0.995, ok_lp.mean()
    go = ro["grad"]
    rel = np.linalg.norm(g - go, axis=1) / np.maximum(np.linalg.norm(go, axis=1), 1e-6)
    # the dual gradient is the derivative of the smooth piece the oracle's
    # path lies in, which is what the adjoint differentiates wherever the
    # FP32 path made the same discrete choices (log p agreeing)
    good = rel[lit & ok_lp] <= 1e-4
    q = np.quantile(rel[lit & ok_lp], [0.5, 0.99, 0.999])
    print(f"{case}: rel grad err quantiles 50/99/99.9% {q}, frac<=1e-4 {good.mean():.4f}")
    assert good.mean() >= 0.99, good.mean()
    r.close()


def _fd_gradient_fp64(oracle, tgt, x, L, h=1e-6):
    """FP64 central differences of the oracle's log p at every coordinate,
    and whether every x +- h e_i keeps the discrete choices (triangles,
    lobes, light visibility and pixel) of x, as Sec. 6's autodiff
    derivative of the smooth piece requires."""
    M, d = x.shape
    base = oracle.evaluate(tgt, x, L, info=True)
    idx = np.tile(np.arange(d), M)
    rows = np.arange(M * d)
    lp = []
    same = np.ones(M, bool)
    for sgn in (1.0, -1.0):
        xx = np.repeat(x, d, 0)
        xx[rows, idx] += sgn * h
        rr = oracle.evaluate(tgt, xx, L, info=True)
        ok = np.all(rr["info"] == np.repeat(base["info"], d, 0), 1) & (rr["pix"] == np.repeat(base["pix"], d, 0))
        same &= ok.reshape(M, d).all(1)
        lp.append(rr["logp"].reshape(M, d))
    return (lp[0] - lp[1]) / (2 * h), same, base


@pytest.mark.parametrize("case", list(EVAL_CASES))
def test_adjoint_matches_fp64_central_differences(torch, R, oracle, case):
    """The CUDA adjoint (FP32 reverse mode) against FP64 central differences
    of the oracle's f at h = 1e-6 with every discrete choice held equal: on
    lit points where the GPU's log p agrees with the oracle's, the gradient
    vector agrees to 1e-4 relative (scale max(|grad|, 1)) on >= 99% of
    them.  Points whose choices change within +-h sit on an edge of the
    piecewise-smooth f, where the derivative of the smooth piece is not
    what a difference measures; they are excluded and counted."""
    make, L = EVAL_CASES[case]
    scene = make()
    d = S.pss_dim(L)
    r = R.Renderer()
    r.upload_scene(scene)
    M = 1500
    x = np.random.default_rng(17).random((M, d)).astype(np.float32)
    lp, g, _, _ = r.eval_logp(torch.from_numpy(x).cuda(), L=L, grad=True)
    torch.cuda.synchronize()
    lp, g = lp.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    r.close()
    tgt = oracle.OracleScene(scene)
    fd, stable, base = _fd_gradient_fp64(oracle, tgt, x.astype(np.float64), L)
    lit = base["f"].sum(1) > 0
    agree = np.abs(lp - base["logp"]) <= 1e-4 * np.maximum(1.0, np.abs(base["logp"]))
    use = lit & agree & stable
    rel = np.linalg.norm(g - fd, axis=1) / np.maximum(np.linalg.norm(fd, axis=1), 1.0)
    q = np.quantile(rel[use], [0.5, 0.9, 0.99, 0.999]) if use.any() else []
    print(f"{case}: lit {lit.sum()}, on an edge within h {(lit & ~stable).sum()}, log p disagreeing "
          f"{(lit & ~agree).sum()}, compared {use.sum()}; rel err quantiles 50/90/99/99.9% {q}; "
          f"frac <= 1e-4 {np.mean(rel[use] <= 1e-4):.4f}")
    assert use.sum() >= 60
    assert np.mean(rel[use] <= 1e-4) >= 0.99


def test_lstar_over_p_matches_oracle(torch, R, oracle):
    """The App. C diagnostic L* p / p (Sec. 5.2, Eq. bias) on a 2-D mixture,
    on the device (FP64 quadrature, one block per point) against the
    oracle's quadrature with the same nodes: both are FP64 sums of the same
    terms in different orders, so they agree to a relative 1e-13 of K* p / p,
    i.e. 1e-8 after the factor h = 1 / dt; the constant density gives 0 (the
    kernel's mass is 1)."""
    f32 = lambda v: np.asarray(v, np.float32).astype(np.float64)
    mix = S.Mixture(2, f32([0.3, 0.7]), f32([[0.35, 0.45], [0.62, 0.58]]), f32([0.05, 0.08]), 8, 8)
    stddev, dt, gt, eps = (float(np.float32(v)) for v in (5e-3, 1e-5, 1.25e-5, 1e-8))
    prm = R.make_params(L=1, drift="adjoint", stddev=stddev, dt=dt, gamma_tilde=gt, eps=eps)
    y = np.random.default_rng(21).random((2048, 2)).astype(np.float32)
    y[:1024] = (mix.mu[np.arange(1024) % 2] + np.random.default_rng(22).normal(size=(1024, 2)) * 0.06).astype(
        np.float32) % 1.0
    r = R.Renderer()
    r.set_mixture(mix)
    yd = torch.from_numpy(y).cuda()
    r.lstar_over_p(yd, prm)                  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    got = r.lstar_over_p(yd, prm)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    got = got.cpu().numpy()
    ref = oracle.lstar_over_p(oracle.target(mix), y.astype(np.float64), stddev=stddev, dt=dt, gamma_tilde=gt,
                              eps=eps, radius=8.0, n=129)
    err = np.abs(got - ref)
    print(f"L*p/p on {len(y)} points in {ms:.2f} ms ({len(y) * 129 * 129 / ms / 1e6:.2f} G nodes/s); max |dev - "
          f"oracle| {err.max():.2e}, range of values {np.abs(ref).max():.3g}")
    assert np.abs(ref).max() > 1.0
    assert np.all(err <= 1e-8 * (1.0 + np.abs(ref)) + 1e-7)
    r.set_mixture(S.constant_target(d=2, value=2.0, width=8, height=8))
    flat = r.lstar_over_p(yd[:64], prm).cpu().numpy()
    assert np.all(np.abs(flat) < 1e-6), np.abs(flat).max()
    r.close()


@pytest.mark.parametrize("inside", [True, False], ids=["camera-in-glass", "camera-in-air"])
def test_dielectric_radiance_scaling_on_gpu(torch, R, oracle, inside):
    """The CUDA dielectric branch against optics directly (the oracle's pins
    D1 and D2): in a room of black walls emitting Le every path that reaches
    a wall carries n^2 Le from a camera inside a glass body and Le from one
    in air (FP32: within 1e-5 relative); and path for path the device's f
    equals the oracle's."""
    n, Le, L = 1.5, 1.0, 8
    scene = S.glass_furnace(camera_inside=inside, emission=Le, ior=n)
    d = S.pss_dim(L)
    x = np.random.default_rng(23).random((20000, d)).astype(np.float32)
    r = R.Renderer()
    r.upload_scene(scene)
    _, _, _, f = r.eval_logp(torch.from_numpy(x).cuda(), L=L, want_f=True)
    torch.cuda.synchronize()
    f = f.cpu().numpy().astype(np.float64) / (scene.width * scene.height)
    r.close()
    reached = f[:, 0] > 0
    expect = n * n * Le if inside else Le
    assert reached.mean() > 0.9
    assert np.allclose(f[reached], expect, rtol=1e-5, atol=0.0), np.unique(np.round(f[reached, 0], 6))[:8]
    fo = oracle.evaluate(oracle.OracleScene(scene), x.astype(np.float64), L)["f"] / (scene.width * scene.height)
    same = np.abs(f - fo).max(1) <= 1e-5 * np.maximum(fo.max(1), 1e-12)
    assert same.mean() > 0.995, same.mean()


def test_logp_autograd_function(torch, R, oracle):
    """LogPFunction: x -> log p as a torch autograd node; its backward runs
    the adjoint kernel, scaled by the incoming gradient, and matches the
    oracle's dual-number gradient on lit points."""
    scene, L = S.cornell_box(1, 64, 64, glossy=True), 6
    d = S.pss_dim(L)
    r = R.Renderer()
    r.upload_scene(scene)
    rng = np.random.default_rng(8)
    M = 600
    x0 = rng.random((M, d)).astype(np.float32)
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.normal(size=M).astype(np.float32)).cuda()
    y = R.LogPFunction.apply(x, r, L)
    (y * w).sum().backward()
    # the forward is the value-only evaluation, the backward the one with the
    # adjoint (two kernel instantiations: log p agrees to the last bits)
    lp, _, _, _ = r.eval_logp(torch.from_numpy(x0).cuda(), L=L, grad=False)
    lp_g, g, _, _ = r.eval_logp(torch.from_numpy(x0).cuda(), L=L, grad=True)
    torch.cuda.synchronize()
    assert torch.equal(y.detach(), lp)
    assert torch.allclose(lp, lp_g, rtol=1e-5, atol=1e-5)
    assert torch.equal(x.grad, g * w[:, None])
    ro = oracle.evaluate(oracle.OracleScene(scene), x0.astype(np.float64), L, grad=True)
    lit = ro["f"].sum(1) > 0
    go = ro["grad"] * w.cpu().numpy()[:, None].astype(np.float64)
    gg = x.grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(gg - go, axis=1) / np.maximum(np.linalg.norm(go, axis=1), 1e-6)
    print(f"LogPFunction: lit {lit.sum()}, frac rel <= 1e-4 {np.mean(rel[lit] <= 1e-4):.4f}")
    assert lit.mean() > 0.05 and np.mean(rel[lit] <= 1e-4) >= 0.97
    r.close()


def score_tolerance(params_orc, loosen=1.0):
    """Per-chain test of |score_gpu - score_oracle| for a chain whose discrete
    choices agree.  Exact drift (the adjoint / the mixture's gradient): 1e-4
    relative to the oracle's score vector (floor 1), the bound the per-point
    adjoint tests hold on >= 99% of points.  Finite differences in FP32: log
    p at x +- h carries a rounding error of about 1e-6 max(1, |log p|), which
    the difference divides by h, so the bound adds 2e-6 max(1, |log p|) / h
    (2e-3 max(1, |log p|) at h = 1e-3).  ``loosen`` scales the bound."""
    if params_orc.drift_mode == 1:
        h = params_orc.fd_h

        def ok(sg, so, lo):
            lim = loosen * (1e-4 * np.abs(so) + 2e-6 * np.maximum(1.0, np.abs(lo))[:, None] / h)
            return np.all(np.abs(sg - so) <= lim, axis=1)
    else:
        def ok(sg, so, lo):
            return np.linalg.norm(sg - so, axis=1) <= loosen * 1e-4 * np.maximum(np.linalg.norm(so, axis=1), 1.0)
    return ok


def _chain_parity(torch, R, oracle, target_obj, params_gpu, params_orc, N, M, T, seed, x_tol=1e-4):
    r = R.Renderer()
    if isinstance(target_obj, S.Scene):
        r.upload_scene(target_obj)
    else:
        r.set_mixture(target_obj)
    r.init_chains(N, seed, params_gpu)
    tgt = oracle.target(target_obj)
    ro = oracle.restore_run(tgt, params_orc, seed=seed, chain_ids=np.arange(M), n_steps=T)
    alive = np.ones(M, bool)
    first_div = np.full(M, -1)
    n_cmp = 0
    n_score = 0
    n_score_bad = 0
    n_score_bad10 = 0
    causes = {}
    score_ok = score_tolerance(params_orc)
    score_ok10 = score_tolerance(params_orc, 10.0)
    for s in range(T + 1):
        if s > 0:
            r.step(1)
        st = r.readback_state()
        xg, lg, kg, pg, vg = st["x"][:M], st["logp"][:M], st["killed"][:M], st["pix"][:M], st["val"][:M]
        xo, lo_, ko, po, vo = ro["x"][s], ro["logp"][s], ro["killed"][s], ro["pix"][s], ro["val"][s]
        xerr = torus_dist(xg, xo).max(1)
        checks = {"killed": kg == ko, "pix": pg == po, "x": xerr <= x_tol,
                  "logp": np.abs(lg - lo_) <= 1e-4 * np.maximum(1.0, np.abs(lo_)),
                  "val": np.linalg.norm(vg - vo, axis=1) <= 1e-4 * np.linalg.norm(vo, axis=1) + 1e-12}
        # the stored score (used by the next LocalDynamics) of surviving,
        # agreeing chains, counted per (chain, step): like the per-point
        # adjoint tests, FP32 leaves a small tail above 1e-4 (a chain meets
        # it once in a while over 16 steps; it grows with the path length,
        # to about 1.2% of comparisons at L = 16), so the score is held to
        # the bound on >= 98% of comparisons and to ten times it on >= 99.8%
        cmp_ = alive & np.logical_and.reduce(list(checks.values())) & (kg == 0) & (ko == 0)
        sg_, so_ = st["score"][:M][cmp_], ro["score"][s][cmp_]
        n_score += int(cmp_.sum())
        n_score_bad += int((~score_ok(sg_, so_, lo_[cmp_])).sum())
        n_score_bad10 += int((~score_ok10(sg_, so_, lo_[cmp_])).sum())
        ok = np.logical_and.reduce(list(checks.values()))
        newly = alive & ~ok
        for j in np.nonzero(newly)[0]:
            failed = ",".join(k for k, v in checks.items() if not v[j])
            causes[failed] = causes.get(failed, 0) + 1
            if len(causes) <= 6:
                print(f"  chain {j} step {s}: {failed}; xerr {xerr[j]:.2e} logp {lg[j]:.6g}/{lo_[j]:.6g} "
                      f"killed {kg[j]}/{ko[j]} pix {pg[j]}/{po[j]}")
        first_div[newly] = s
        alive &= ok
        n_cmp += alive.sum()
    frac_div = 1.0 - alive.mean()
    print(f"  divergence causes: {causes}; scores compared {n_score}, beyond the bound {n_score_bad}, "
          f"beyond ten times it {n_score_bad10}")
    r.close()
    assert n_score >= min(100, M), n_score
    assert n_score_bad <= 0.02 * n_score and n_score_bad10 <= 0.002 * n_score
    return frac_div, first_div, n_cmp


def _chain_parity_opts(torch, R, oracle, target_obj, params_gpu, params_orc, N, M, T, seed, opts, x_tol=1e-4):
    """_chain_parity with renderer options set before the upload."""
    orig = R.Renderer

    class _R(orig):
        def __init__(self, *args, **kw):
            super().__init__(*args, **kw)
            for k, v in opts.items():
                self.set_option(k, v)

    R.Renderer = _R
    try:
        return _chain_parity(torch, R, oracle, target_obj, params_gpu, params_orc, N, M, T, seed, x_tol)
    finally:
        R.Renderer = orig


def test_chain_parity_mixture_target(torch, R, oracle):
    mix = S.gaussian_mixture(seed=4, d=4, K=3, sig_range=(0.08, 0.12), width=16, height=16)
    k0 = 1.0 / (64 * 1e-5)
    pg = R.make_params(L=1, drift="adjoint", rb=True, k0=k0, steps_per_splat=4)
    po = oracle.make_params(L=1, drift="exact", rb=True, k0=k0)
    frac, first, n = _chain_parity(torch, R, oracle, mix, pg, po, N=8192, M=2048, T=16, seed=21)
    print("mixture divergent fraction", frac, "compared", n)
    assert frac <= 0.002


def test_chain_parity_cornell_fd(torch, R, oracle):
    scene = S.cornell_box(1, 64, 64)
    k0 = 5000.0
    pg = R.make_params(L=4, drift="fd", rb=True, k0=k0, fd_h=1e-3, steps_per_splat=8)
    po = oracle.make_params(L=4, drift="fd", rb=True, k0=k0, fd_h=1e-3)
    frac, first, n = _chain_parity(torch, R, oracle, scene, pg, po, N=4096, M=512, T=16, seed=5)
    print("cornell fd divergent fraction", frac, "compared", n)
    assert frac <= 0.01


def test_chain_parity_glossy_adjoint(torch, R, oracle):
    scene = S.cornell_box(1, 256, 256, glossy=True)
    k0 = 1e6
    pg = R.make_params(L=8, drift="adjoint", rb=True, k0=k0, steps_per_splat=16)
    po = oracle.make_params(L=8, drift="exact", rb=True, k0=k0)
    frac, first, n = _chain_parity(torch, R, oracle, scene, pg, po, N=65536, M=512, T=16, seed=6)
    print("glossy adjoint divergent fraction", frac, "compared", n)
    assert frac <= 0.01


@pytest.mark.parametrize("which", ["mixture", "glossy"])
def test_chain_parity_mala_restore(torch, R, oracle, which):
    """MALA Restore (the comparison method of Sec. 6: Metropolis-adjusted
    Langevin local moves, holding rate 1, i.e. dt = 1) against the oracle's:
    proposals, Metropolis-Hastings decisions (FP64 on both sides), clock,
    splat values and the stored score over 16 steps.  A decision that FP32
    inputs move across its threshold makes a chain divergent (counted)."""
    if which == "mixture":
        target = S.gaussian_mixture(seed=4, d=4, K=3, sig_range=(0.08, 0.12), width=16, height=16)
        L, k0, stddev = 1, 1.0 / 64, 0.03
    else:
        target = S.cornell_box(1, 64, 64, glossy=True)
        L, k0, stddev = 6, 2000.0 / 64, 5e-3
    pg = R.make_params(L=L, drift="mala", rb=True, k0=k0, stddev=stddev, dt=1.0, steps_per_splat=8)
    po = oracle.make_params(L=L, drift="mala", rb=True, k0=k0, stddev=stddev, dt=1.0)
    frac, first, n = _chain_parity(torch, R, oracle, target, pg, po, N=4096, M=512, T=16, seed=31)
    print(f"MALA Restore ({which}) divergent fraction", frac, "compared", n)
    assert frac <= 0.01


def test_mala_restore_graph_frames_and_refusals(torch, R):
    """dr_frame replays MALA steps exactly as dr_step + dr_splat; MALA chains
    are not checkpointed and a batch does not run them (both refused)."""
    from paper_2605_08916_gb300 import _lib
    scene = S.cornell_box(1, 32, 32, glossy=True)
    prm = R.make_params(L=5, drift="mala", rb=True, k0=0.0, stddev=5e-3, dt=1.0, steps_per_splat=4)
    res = []
    for graph in (False, True):
        s = torch.cuda.Stream()
        r = R.Renderer(0, s)
        r.upload_scene(scene)
        r.init_chains(8192, 12, prm)
        for _ in range(3):
            if graph:
                r.frame(4)
            else:
                r.step(4)
                r.splat()
        s.synchronize()
        res.append((r.readback_state(fields=("x", "killed", "score")), r.readback_accum(), r.counters()))
        if graph:
            with pytest.raises(_lib.DRError):
                r.state_save()
        r.close()
    (a, acc_a, c_a), (b, acc_b, c_b) = res
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["killed"], b["killed"])
    assert np.array_equal(acc_a, acc_b) and c_a["tour_count"] == c_b["tour_count"] > 0
    rb = R.Renderer()
    rb.upload_scenes(batch_items())
    with pytest.raises(_lib.DRError):
        rb.init_chains(sum(n for _, _, n in batch_items()), 5, prm)
    rb.close()


@pytest.mark.parametrize("wavefront", [0, 1])
def test_chain_parity_without_drift(torch, R, oracle, wavefront):
    """Drift mode none (LocalDynamics with a zero score: the drift ablation
    of the equal-time comparison) in both execution modes: the score stays
    zero and the chains follow the oracle's."""
    scene = S.cornell_box(2, 64, 64, glossy=True)
    k0 = 1e6
    pg = R.make_params(L=6, drift="none", rb=True, k0=k0, steps_per_splat=8)
    po = oracle.make_params(L=6, drift="none", rb=True, k0=k0)
    frac, first, n = _chain_parity_opts(torch, R, oracle, scene, pg, po, N=1 << 17, M=512, T=12, seed=19,
                                        opts={"wavefront": wavefront})
    print("no-drift divergent fraction", frac, "compared", n)
    assert frac <= 0.01


@pytest.mark.parametrize("wavefront", [0, 1])
def test_chain_parity_conductor_adjoint(torch, R, oracle, wavefront):
    """Rough conductor boxes (complex-index Fresnel per channel) with the
    adjoint drift, in both execution modes."""
    scene = S.cornell_box(4, 128, 128, metal=True)
    k0 = 1e6
    pg = R.make_params(L=8, drift="adjoint", rb=True, k0=k0, steps_per_splat=16)
    po = oracle.make_params(L=8, drift="exact", rb=True, k0=k0)
    frac, first, n = _chain_parity_opts(torch, R, oracle, scene, pg, po, N=16384, M=512, T=16, seed=9,
                                        opts={"wavefront": wavefront})
    print("conductor adjoint divergent fraction", frac, "compared", n)
    assert frac <= 0.01


def test_chain_parity_race_clock(torch, R, oracle):
    scene = S.cornell_box(2, 32, 32)
    k0 = 2000.0
    pg = R.make_params(L=4, drift="adjoint", rb=False, k0=k0, steps_per_splat=4)
    po = oracle.make_params(L=4, drift="exact", rb=False, k0=k0)
    frac, first, n = _chain_parity(torch, R, oracle, scene, pg, po, N=1024, M=512, T=16, seed=8)
    print("race-clock divergent fraction", frac)
    assert frac <= 0.01


def test_image_relmse_distribution_matches_oracle(torch, R, oracle):
    """At equal chain-step counts, the relMSE of the GPU's Restore images over
    16 seeds is statistically indistinguishable from the oracle's on the same
    seeds (Welch t-test, p > 0.01), against an oracle path-traced reference."""
    stats = pytest.importorskip("scipy.stats")
    scene = S.cornell_box(1, 16, 16)
    L, N, T = 4, 1024, 128
    tgt = oracle.OracleScene(scene)
    xs = np.random.default_rng(11).random((4096, S.pss_dim(L)))
    p_hat = float(np.mean(np.exp(oracle.evaluate(tgt, xs, L)["logp"])))
    k0 = p_hat / (64 * 1e-5)
    ref, _ = oracle.pt_image(tgt, L, 1 << 14, seed=3)
    ref = ref.reshape(16, 16, 3)
    pg = R.make_params(L=L, drift="adjoint", rb=True, k0=k0, steps_per_splat=16)
    po = oracle.make_params(L=L, drift="exact", rb=True, k0=k0)
    r = R.Renderer()
    r.upload_scene(scene)
    e_gpu, e_orc = [], []
    for seed in range(100, 116):
        r.init_chains(N, seed, pg)
        r.step(T)
        img = r.resolve().cpu().numpy().astype(np.float64)
        e_gpu.append(oracle.rel_mse(img, ref))
        ro = oracle.restore_run(tgt, po, seed=seed, chain_ids=np.arange(N), n_steps=T, record=False)
        img_o = oracle.resolve(ro["accum"], k0, ro["tour_count"]).reshape(16, 16, 3)
        e_orc.append(oracle.rel_mse(img_o, ref))
    r.close()
    e_gpu, e_orc = np.array(e_gpu), np.array(e_orc)
    t = stats.ttest_ind(e_gpu, e_orc, equal_var=False)
    print(f"relMSE gpu {e_gpu.mean():.4g} +- {e_gpu.std(ddof=1):.2g}, oracle {e_orc.mean():.4g} +- "
          f"{e_orc.std(ddof=1):.2g}, Welch p = {t.pvalue:.3g}")
    assert t.pvalue > 0.01
    assert np.all(np.abs(e_gpu - e_orc) <= 0.05 * e_orc + 1e-3)


def test_pt_reference_image_matches_oracle(torch, R, oracle):
    """Stratified path tracing on the GPU and in the oracle draw the same
    Philox numbers, so their per-pixel means agree sample for sample."""
    scene = S.cornell_box(3, 16, 16, glossy=True)
    L, spp = 5, 256
    r = R.Renderer()
    r.upload_scene(scene)
    img = r.pt_render(L, spp, seed=99).cpu().numpy().reshape(-1, 3)
    mean, var = oracle.pt_image(oracle.OracleScene(scene), L, spp, seed=99)
    err = np.abs(img - mean)
    close = err <= 1e-3 * np.maximum(mean, 1e-3) + 3e-3 * np.sqrt(var)
    assert close.mean() > 0.98, close.mean()
    assert abs(img.mean() / mean.mean() - 1) < 1e-3
    r.close()


def _sampled_parity(st_x, st_logp, st_killed, ro, sample, x_tol=1e-4):
    """Fraction of sampled chains whose final state differs from the oracle's."""
    xo, lo_, ko = ro["x"][-1], ro["logp"][-1], ro["killed"][-1]
    ok = (st_killed[sample] == ko) & (torus_dist(st_x[sample], xo).max(1) <= x_tol)
    ok &= np.abs(st_logp[sample] - lo_) <= 1e-4 * np.maximum(1.0, np.abs(lo_))
    return 1.0 - ok.mean()


def test_full_size_bench_configuration_matches_oracle_on_sampled_chains(torch, R, oracle):
    """The bench's own workload and launch configuration (1M-triangle
    procedural scene, 2^20 chains, L = 12, bounce-by-bounce passes with the
    4-wide BVH, camera-ray sort and CUDA-graph frames), checked on 192
    sampled chains that the oracle follows one by one over two frames."""
    scene = S.procedural_scene(1, 1280, 720)
    N, L, F, seed = 1 << 20, 12, 4, 91
    k0 = 2.0e6
    stream = torch.cuda.Stream()
    r = R.Renderer(0, stream)
    r.upload_scene(scene)
    r.init_chains(N, seed, R.make_params(L=L, drift="adjoint", rb=True, k0=k0, steps_per_splat=F))
    r.frame(F)
    r.frame(F)
    stream.synchronize()
    st = r.readback_state(("x", "killed", "logp"))
    r.close()
    sample = np.sort(np.random.default_rng(5).choice(N, 192, replace=False))
    tgt = oracle.OracleScene(scene)
    ro = oracle.restore_run(tgt, oracle.make_params(L=L, drift="exact", rb=True, k0=k0), seed=seed,
                            chain_ids=sample, n_steps=2 * F)
    frac = _sampled_parity(st["x"], st["logp"], st["killed"], ro, np.arange(N)[sample])
    print(f"full-size sampled chains: divergent fraction {frac:.4f}")
    assert frac <= 0.02


def test_full_size_caustic_matches_oracle_on_sampled_chains(torch, R, oracle):
    """The caustic workload at full size in the bench's launch configuration
    (19,800-triangle glass sphere, 512 x 512, L = 10, 2^18 chains,
    bounce-by-bounce passes, one 16-step CUDA-graph frame, k0 estimated on
    the device): 512 sampled chains followed by the oracle with the
    device's k0 over the 16 steps; x, log p, kill flags and the stored
    score of survivors compared at the end (most caustic chains sit on dark
    paths and die within a few steps, so 512 are sampled)."""
    scene = S.caustic_scene(1, 512, 512)
    N, L, F, seed = 1 << 18, 10, 16, 97
    stream = torch.cuda.Stream()
    r = R.Renderer(0, stream)
    r.upload_scene(scene)
    r.init_chains(N, seed, R.make_params(L=L, drift="adjoint", rb=True, k0=0.0, steps_per_splat=F))
    r.frame(F)
    stream.synchronize()
    st = r.readback_state(("x", "killed", "logp", "score"))
    k0 = r.counters()["k0"]
    r.close()
    assert k0 > 0
    sample = np.sort(np.random.default_rng(7).choice(N, 512, replace=False))
    ro = oracle.restore_run(oracle.OracleScene(scene), oracle.make_params(L=L, drift="exact", rb=True, k0=k0),
                            seed=seed, chain_ids=sample, n_steps=F)
    frac = _sampled_parity(st["x"], st["logp"], st["killed"], ro, sample)
    xo_ok = torus_dist(st["x"][sample], ro["x"][-1]).max(1) <= 1e-4
    surv = (st["killed"][sample] == 0) & (ro["killed"][-1] == 0) & xo_ok
    so = ro["score"][-1][surv]
    sg = st["score"][sample][surv].astype(np.float64)
    srel = np.linalg.norm(sg - so, axis=1) / np.maximum(np.linalg.norm(so, axis=1), 1.0)
    print(f"caustic full size: divergent fraction {frac:.4f}; survivors compared {surv.sum()}, "
          f"score within 1e-4: {np.mean(srel <= 1e-4):.4f}")
    assert frac <= 0.03
    assert surv.sum() >= 100 and np.mean(srel <= 1e-4) >= 0.97 and np.mean(srel <= 1e-3) >= 0.99


def test_full_size_batch_matches_oracle_on_sampled_chains(torch, R, oracle):
    """The 64-scene batch workload (2^21 chains, L 4..16), in the bench's
    launch configuration: sampled chains of four scenes against the oracle
    run on each scene with the batch's key (seed_lo, seed_hi + scene)."""
    items = S.procedural_batch()
    N = sum(n for _, _, n in items)
    seed, F, k0 = 93, 2, 2.0e6
    stream = torch.cuda.Stream()
    r = R.Renderer(0, stream)
    r.upload_scenes(items)
    r.init_chains(N, seed, R.make_params(L=16, drift="adjoint", rb=True, k0=k0, steps_per_splat=F))
    r.frame(F)
    stream.synchronize()
    st = r.readback_state(("x", "killed", "logp"))
    r.close()
    starts = np.concatenate([[0], np.cumsum([n for _, _, n in items])])
    rng = np.random.default_rng(6)
    fracs = []
    for s_i in (0, 17, 40, 63):
        scene, L, n = items[s_i]
        local = np.sort(rng.choice(n, 48, replace=False))
        ro = oracle.restore_run(oracle.OracleScene(scene), oracle.make_params(L=L, drift="exact", rb=True, k0=k0),
                                seed=seed + (s_i << 32), chain_ids=local, n_steps=F)
        d = S.pss_dim(L)
        fracs.append(_sampled_parity(st["x"][:, :d], st["logp"], st["killed"], ro, starts[s_i] + local))
    print("batch sampled chains: divergent fractions", fracs)
    assert max(fracs) <= 0.05 and np.mean(fracs) <= 0.02


@pytest.mark.parametrize("which", ["glossy", "conductor", "procedural"])
def test_wavefront_matches_fused(torch, R, which):
    """The bounce-by-bounce execution performs the same operations per path
    as the fused kernel; the compiler may contract multiply-adds
    differently in the two, so values agree to the last bit or two (chains
    whose discrete choices flip on such a difference are counted)."""
    if which == "glossy":
        scene, L = S.cornell_box(1, 64, 64, glossy=True), 8
    elif which == "conductor":
        scene, L = S.cornell_box(1, 64, 64, metal=True), 8
    else:
        scene, L = S.procedural_scene(1, 64, 36, target_tris=60000, n_objects=40), 12
    out = []
    for wf in (0, 1):
        r = R.Renderer()
        r.set_option("wavefront", wf)
        r.upload_scene(scene)
        r.init_chains(16384, 33, R.make_params(L=L, drift="adjoint", k0=0.0, steps_per_splat=4))
        r.step(9)
        st = r.readback_state()
        acc = r.readback_accum()
        c = r.counters()
        r.close()
        out.append((st, acc, c))
    (a, acc_a, c_a), (b, acc_b, c_b) = out
    same = (a["killed"] == b["killed"]) & (a["pix"] == b["pix"])
    same &= torus_dist(a["x"], b["x"]).max(1) <= 1e-6
    same &= np.abs(a["logp"] - b["logp"]) <= 1e-5 * np.maximum(1.0, np.abs(a["logp"]))
    same &= np.linalg.norm(a["val"] - b["val"], axis=1) <= 1e-5 * np.linalg.norm(a["val"], axis=1) + 1e-30
    print(f"{which}: bit-identical x {np.mean(np.all(a['x'] == b['x'], 1)):.4f}, agreeing chains {same.mean():.5f}")
    assert same.mean() >= 0.999
    alive = (a["killed"] == 0) & same
    ga, gb = a["score"][alive], b["score"][alive]
    rel = np.linalg.norm(ga - gb, axis=1) / np.maximum(np.linalg.norm(ga, axis=1), 1e-6)
    assert np.mean(rel <= 1e-4) >= 0.999
    assert np.allclose(acc_a, acc_b, rtol=1e-3, atol=1e-9 * np.abs(acc_a).max())
    assert abs(c_a["tour_count"] - c_b["tour_count"]) <= 1e-3 * c_a["tour_count"] + 5


@pytest.mark.parametrize("tail", [0, 4])
def test_bvh_widths_give_the_same_chains(torch, R, tail):
    """Restore steps (wavefront, adjoint drift) through the binary, the
    4-wide and the 8-wide BVH (with and without the tail pass): all return
    the same hits, so the chains agree."""
    scene, L = S.procedural_scene(1, 64, 36, target_tris=60000, n_objects=40), 12
    out = []
    for width in (2, 4, 8):
        r = R.Renderer()
        r.set_option("wavefront", 1)
        r.set_option("bvh_width", width)
        r.set_option("tail_bounce", tail)
        r.upload_scene(scene)
        assert (r.bvh8_info() is not None) == (width == 8)
        r.init_chains(16384, 35, R.make_params(L=L, drift="adjoint", k0=0.0, steps_per_splat=4))
        r.step(9)
        out.append((r.readback_state(), r.readback_accum()))
        r.close()
    (a, acc_a) = out[0]
    for b, acc_b in out[1:]:
        same = (a["killed"] == b["killed"]) & (a["pix"] == b["pix"]) & np.all(a["x"] == b["x"], 1)
        same &= a["logp"] == b["logp"]
        print(f"bit-identical chains {same.mean():.5f}")
        assert same.mean() >= 0.999
        assert np.allclose(acc_a, acc_b, rtol=1e-3, atol=1e-9 * np.abs(acc_a).max())


def batch_items():
    return [(S.cornell_box(1, 32, 32), 4, 8192),
            (S.cornell_box(2, 48, 40, glossy=True), 6, 12000),
            (S.procedural_scene(3, 64, 36, target_tris=20000, n_objects=20), 8, 20000)]


@pytest.mark.parametrize("width", [4, 8])
def test_batch_matches_separate_contexts(torch, R, width):
    """A multi-scene batch advances each scene exactly as a context of its
    own with key (seed_lo, seed_hi + scene): same chain states, k0, tour
    counts and images, bit for bit (4-wide and 8-wide BVHs)."""
    items = batch_items()
    seed, T = 77, 6
    rb = R.Renderer()
    rb.set_option("bvh_width", width)
    rb.upload_scenes(items)
    N = sum(n for _, _, n in items)
    rb.init_chains(N, seed, R.make_params(L=16, drift="adjoint", k0=0.0, steps_per_splat=4))
    rb.step(T)
    stb = rb.readback_state(("x", "killed", "logp", "score"))
    imgs = [rb.resolve_scene(s).cpu().numpy() for s in range(len(items))]
    cnt = [rb.scene_counters(s) for s in range(len(items))]
    rb.close()
    c0 = 0
    for s, (scene, L, n) in enumerate(items):
        r = R.Renderer()
        r.set_option("wavefront", 1)
        r.set_option("bvh_width", width)
        r.upload_scene(scene)
        r.init_chains(n, seed + (s << 32), R.make_params(L=L, drift="adjoint", k0=0.0, steps_per_splat=4))
        r.step(T)
        st = r.readback_state(("x", "killed", "logp", "score"))
        img = r.resolve().cpu().numpy()
        c = r.counters()
        r.close()
        d = S.pss_dim(L)
        assert np.array_equal(stb["x"][c0:c0 + n, :d], st["x"])
        assert np.array_equal(stb["killed"][c0:c0 + n], st["killed"])
        assert np.array_equal(stb["logp"][c0:c0 + n], st["logp"])
        alive = st["killed"] == 0
        assert np.array_equal(stb["score"][c0:c0 + n, :d][alive], st["score"][alive])
        assert cnt[s]["k0"] == c["k0"] and cnt[s]["tour_count"] == c["tour_count"]
        assert np.array_equal(imgs[s], img)
        c0 += n


def test_batch_with_conductors_matches_separate_contexts(torch, R):
    """A batch holding a conductor scene runs the batch kernels compiled
    with the conductor branches (and, with paths of 16 segments, the tail
    pass): still bit-identical to one context per scene."""
    items = [(S.cornell_box(3, 32, 32, metal=True), 16, 8192),
             (S.procedural_scene(3, 64, 36, target_tris=20000, n_objects=20), 8, 8192)]
    seed, T = 91, 5
    rb = R.Renderer()
    rb.upload_scenes(items)
    rb.init_chains(sum(n for _, _, n in items), seed, R.make_params(L=16, drift="adjoint", k0=0.0, steps_per_splat=4))
    rb.step(T)
    stb = rb.readback_state(("x", "killed", "logp"))
    rb.close()
    c0 = 0
    for s_i, (scene, L, n) in enumerate(items):
        r = R.Renderer()
        r.set_option("wavefront", 1)
        r.set_option("tail_bounce", 4)
        r.upload_scene(scene)
        r.init_chains(n, seed + (s_i << 32), R.make_params(L=L, drift="adjoint", k0=0.0, steps_per_splat=4))
        r.step(T)
        st = r.readback_state(("x", "killed", "logp"))
        r.close()
        d = S.pss_dim(L)
        assert np.array_equal(stb["x"][c0:c0 + n, :d], st["x"])
        assert np.array_equal(stb["killed"][c0:c0 + n], st["killed"])
        assert np.array_equal(stb["logp"][c0:c0 + n], st["logp"])
        c0 += n


def test_batch_graph_frames_and_errors(torch, R):
    from paper_2605_08916_gb300 import _lib
    items = batch_items()
    N = sum(n for _, _, n in items)
    stream = torch.cuda.Stream()
    r = R.Renderer(0, stream)
    r.upload_scenes(items)
    with pytest.raises(_lib.DRError):
        r.init_chains(N + 1, 5, R.make_params(L=8, drift="adjoint", k0=0.0))
    with pytest.raises(_lib.DRError):
        r.init_chains(N, 5, R.make_params(L=8, drift="fd", k0=0.0))
    with pytest.raises(_lib.DRError):
        r.resolve()
    prm = R.make_params(L=8, drift="adjoint", k0=0.0, steps_per_splat=4)
    r.init_chains(N, 5, prm)
    r.step(8)
    a = [r.resolve_scene(s).cpu().numpy() for s in range(3)]
    r.init_chains(N, 5, prm)
    r.frame(4)
    r.frame(4)
    b = [r.resolve_scene(s).cpu().numpy() for s in range(3)]
    stream.synchronize()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
        assert np.isfinite(x).all() and x.max() > 0
    one = S.cornell_box(1, 8, 8)
    keep = np.zeros(one.n_tris, bool)
    keep[0] = True
    tiny = S.Scene(verts=one.verts, tris=np.ascontiguousarray(one.tris[keep]),
                   tri_mat=np.ascontiguousarray(one.tri_mat[keep]), materials=one.materials, camera=one.camera,
                   width=8, height=8, normals=one.normals).check()
    with pytest.raises(_lib.DRError):
        r.upload_scenes([(tiny, 4, 128)])
    r.close()


@pytest.mark.parametrize("tail", [2, 5])
def test_tail_pass_gives_the_same_chains(torch, R, tail):
    """Running the late bounces as one persistent pass performs each path's
    work in the same order as the bounce-by-bounce passes: identical chain
    states, counters and images."""
    scene, L = S.procedural_scene(1, 64, 36, target_tris=60000, n_objects=40), 12
    out = []
    for tb in (0, tail):
        r = R.Renderer()
        r.set_option("wavefront", 1)
        r.set_option("tail_bounce", tb)
        r.upload_scene(scene)
        r.init_chains(16384, 37, R.make_params(L=L, drift="adjoint", k0=0.0, steps_per_splat=4))
        r.step(7)
        out.append((r.readback_state(("x", "killed", "logp", "score")), r.readback_accum(), r.counters()))
        r.close()
    (a, acc_a, c_a), (b, acc_b, c_b) = out
    for key in ("x", "killed", "logp", "score"):
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(acc_a, acc_b)
    assert c_a["tour_count"] == c_b["tour_count"] and c_a["rays"] == c_b["rays"]


def test_bounce_rays_count_the_traced_rays(torch, R):
    """The profile's rays per bounce: every chain's camera ray at bounce 1,
    and closest-hit plus shadow rays over all bounces equal the rays the
    traversal passes counted."""
    scene, L, N = S.procedural_scene(2, 64, 36, target_tris=20000, n_objects=20), 8, 8192
    r = R.Renderer()
    r.set_option("wavefront", 1)
    r.upload_scene(scene)
    r.init_chains(N, 3, R.make_params(L=L, drift="adjoint", k0=0.0, steps_per_splat=4))
    r.set_option("profile", 1)
    r.profile()
    c0 = r.counters()["rays"]
    r.step(2)
    c1 = r.counters()["rays"]
    bp = r.bounce_profile(L)
    r.profile()
    r.close()
    assert bp["rays"][0] == 2 * N
    assert all(x >= y for x, y in zip(bp["rays"], bp["rays"][1:]))
    assert sum(bp["rays"]) + sum(bp["shadow_rays"]) == c1 - c0


@pytest.mark.parametrize("chains", [8192, 1 << 17])
def test_graph_frames_match_plain_steps(torch, R, chains):
    """dr_frame (captured once, replayed with the step index in device
    memory) draws the same Philox numbers and runs the same kernels as
    dr_step + dr_splat: identical chains and image."""
    scene = S.cornell_box(1, 64, 64, glossy=True)
    F = 5
    res = []
    for graph in (False, True):
        s = torch.cuda.Stream()
        r = R.Renderer(0, s)
        r.upload_scene(scene)
        r.init_chains(chains, 44, R.make_params(L=6, drift="adjoint", k0=0.0, steps_per_splat=F))
        for _ in range(3):
            if graph:
                r.frame(F)
            else:
                r.step(F)
                r.splat()
        s.synchronize()
        st = r.readback_state(fields=("x", "killed", "score"))
        acc = r.readback_accum()
        c = r.counters()
        res.append((st, acc, c))
        r.close()
    (a, acc_a, c_a), (b, acc_b, c_b) = res
    assert c_a["steps"] == c_b["steps"] == 3 * F
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["killed"], b["killed"])
    assert np.array_equal(acc_a, acc_b)
    assert c_a["tour_count"] == c_b["tour_count"]


def test_profile_reports_phases(torch, R):
    r = R.Renderer()
    r.upload_scene(S.cornell_box(1, 32, 32, glossy=True))
    r.init_chains(1 << 17, 5, R.make_params(L=6, drift="adjoint", k0=0.0, steps_per_splat=2))
    r.set_option("profile", 1)
    r.profile()
    r.step(3)
    r.splat()
    b = r.bounce_profile(6)
    p = r.profile()
    assert p["trace"][1] == 3 * 6 and p["trace"][0] > 0
    assert p["adjoint"][1] == 3 and p["splat"][1] >= 1
    # 4-wide BVH: the trace row holds the combined passes (closest-hit rays
    # of bounce k and shadow rays of bounce k - 1), the shadow row the last
    # bounce's shadow rays
    assert min(b["trace"]) > 0 and min(b["shade"]) > 0 and b["shadow"][-1] > 0
    for name in ("trace", "shade", "shadow"):
        assert len(b[name]) == 6
        assert abs(sum(b[name]) - p[name][0]) <= 1e-6 * p[name][0] + 1e-9
    assert sum(r.bounce_profile(6)["trace"]) == 0.0  # cleared by profile()
    r.close()


def test_k0_estimate_matches_oracle(torch, R, oracle):
    scene = S.cornell_box(1, 64, 64)
    N = 4096
    r = R.Renderer()
    r.upload_scene(scene)
    r.init_chains(N, 17, R.make_params(L=4, drift="adjoint", k0=0.0))
    c = r.counters()
    ro = oracle.restore_run(oracle.OracleScene(scene), oracle.make_params(L=4, drift="none", k0=1.0), seed=17,
                            chain_ids=np.arange(N), n_steps=0, record=False)
    p_lambda = ro["p_init_sum"] / N
    assert abs(c["p_lambda"] / p_lambda - 1.0) < 1e-4
    assert abs(c["k0"] - p_lambda / (64 * 1e-5)) < 1e-4 * c["k0"]
    r.close()


def test_splat_is_bit_exact_sequential_sum(torch, R):
    r = R.Renderer()
    W, H = 64, 48
    r.set_mixture(S.constant_target(d=2, value=1.0, width=W, height=H))
    r.init_chains(16, 1, R.make_params(L=1, drift="none", k0=1.0))
    r.clear_image()
    rng = np.random.default_rng(7)
    M = 300000
    pix = (rng.zipf(1.3, M) % (W * H)).astype(np.uint32)   # heavy duplicates
    val = rng.normal(size=(M, 3)).astype(np.float32) * np.float32(1e-3)
    rec = np.zeros((M, 4), np.int32)
    rec[:, 0] = pix.view(np.int32)
    rec[:, 1:] = val.view(np.int32)
    r.splat_records(torch.from_numpy(rec).cuda())
    acc = r.readback_accum()
    ref = np.zeros((W * H, 3))
    for c in range(3):
        ref[:, c] = np.bincount(pix, weights=val[:, c].astype(np.float64), minlength=W * H)
    assert np.array_equal(acc, ref)
    # a pixel index >= W * H fails this call only (the kernel skips the
    # record); the context goes on stepping and splatting
    from paper_2605_08916_gb300 import _lib
    bad = rec[:1000].copy()
    bad[17, 0] = W * H
    with pytest.raises(_lib.DRError) as e:
        r.splat_records(torch.from_numpy(bad).cuda())
    assert e.value.code == _lib.DR_ERR_DEVICE_CHECK
    r.clear_image()
    r.splat_records(torch.from_numpy(rec).cuda())
    assert np.array_equal(r.readback_accum(), ref)
    r.step(2)
    r.close()


def test_resolve_is_k0_over_tourcount_times_accum(torch, R):
    r = R.Renderer()
    scene = S.cornell_box(1, 32, 32)
    r.upload_scene(scene)
    r.init_chains(2048, 3, R.make_params(L=4, drift="adjoint", k0=0.0, steps_per_splat=4))
    r.step(10)
    img = r.resolve().cpu().numpy().reshape(-1, 3)
    acc = r.readback_accum()
    c = r.counters()
    assert c["tour_count"] > 0 and c["steps"] == 10
    ref = (acc * (c["k0"] / c["tour_count"])).astype(np.float32)
    assert np.allclose(img, ref, rtol=1e-6, atol=0)
    r.close()


def test_replica_calls_resolve_and_pool_like_the_context(torch, R):
    """The context-free calls the replicas use: dr_resolve_accum on a copy of
    the accumulator equals dr_resolve bit for bit (zero image and STATE at
    tourCount 0), and the initial-sample sums give back the context's own
    p_lambda and k0 through dr_k0_from_p_sum."""
    from paper_2605_08916_gb300 import _lib
    r = R.Renderer()
    r.upload_scene(S.cornell_box(1, 32, 32))
    prm = R.make_params(L=4, drift="adjoint", k0=0.0, steps_per_splat=4)
    r.init_chains(4096, 3, prm)
    c = r.counters()
    p_sum, n = r.p_sum()
    assert n == 4096 and p_sum / n == c["p_lambda"]
    assert R.k0_from_p_sum(p_sum, n, prm) == c["k0"]
    r.step(10)
    img = r.resolve()
    acc = torch.from_numpy(r.readback_accum()).cuda()
    c = r.counters()
    out = R.resolve_accum(acc, c["tour_count"], c["k0"])
    torch.cuda.synchronize()
    assert torch.equal(out.reshape(-1), img.reshape(-1))
    zero = R.resolve_accum(acc, 0, c["k0"])
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(zero)) == 0
    L = _lib.load()
    assert L.dr_resolve_accum(None, -1, 1, 1.0, None, None) == _lib.DR_ERR_INVALID_ARG
    import ctypes
    k0 = ctypes.c_double()
    assert L.dr_k0_from_p_sum(1.0, 0, ctypes.byref(prm), ctypes.byref(k0)) == _lib.DR_ERR_INVALID_ARG
    # with k0 given there is no estimate to pool
    r.init_chains(4096, 3, R.make_params(L=4, drift="adjoint", k0=5.0, steps_per_splat=4))
    with pytest.raises(_lib.DRError):
        r.p_sum()
    r.close()


def test_constant_target_kill_fraction_and_image(torch, R):
    c = 2.0
    m, dt = 64.0, 1e-5
    k0 = c / (m * dt)
    r = R.Renderer()
    r.set_mixture(S.constant_target(d=4, value=c, width=4, height=4))
    N, T = 65536, 64
    r.init_chains(N, 9, R.make_params(L=1, drift="adjoint", rb=True, k0=k0, m=m, dt=dt, steps_per_splat=16))
    r.step(T)
    cnt = r.counters()
    n = N * (T + 1)
    p = 1.0 / (m + 1.0)
    assert abs(cnt["tour_count"] / n - p) < 4 * math.sqrt(p * (1 - p) / n)
    img = r.resolve().cpu().numpy().reshape(-1, 3)
    assert np.allclose(img.sum(0), c, rtol=4 / math.sqrt(cnt["tour_count"]))
    r.close()


def test_checkpoint_resume_is_bit_identical(torch, R):
    scene = S.cornell_box(1, 32, 32, glossy=True)
    prm = R.make_params(L=5, drift="adjoint", k0=0.0, steps_per_splat=3)
    a = R.Renderer()
    a.upload_scene(scene)
    a.init_chains(4096, 12, prm)
    a.step(7)
    blob = a.state_save()
    a.step(9)
    img_a = a.readback_accum()
    st_a = a.readback_state(fields=("x", "killed"))
    b = R.Renderer()
    b.upload_scene(scene)
    # damaged checkpoints are rejected on the host, before any device work,
    # and leave the context usable (the header's magic, version and chain
    # count are its first three 64-bit words)
    from paper_2605_08916_gb300 import _lib
    bad = [blob[:-1], blob[:16]]
    for word, value in [(0, 0x1234), (1, 2), (2, 0), (2, (1 << 31) + 1)]:
        c = blob.copy()
        c[8 * word:8 * word + 8] = np.frombuffer(np.uint64(value).tobytes(), np.uint8)
        bad.append(c)
    for c in bad:
        with pytest.raises(_lib.DRError) as e:
            b.state_load(c)
        assert e.value.code == _lib.DR_ERR_INVALID_ARG
    b.state_load(blob)
    b.step(9)
    img_b = b.readback_accum()
    st_b = b.readback_state(fields=("x", "killed"))
    assert np.array_equal(st_a["x"], st_b["x"]) and np.array_equal(st_a["killed"], st_b["killed"])
    assert np.array_equal(img_a, img_b)
    a.close()
    b.close()


def test_errors_are_reported_not_raised_on_device(torch, R):
    from paper_2605_08916_gb300 import _lib
    r = R.Renderer()
    L = _lib.load()
    assert L.dr_step(r.h, 1) == _lib.DR_ERR_STATE
    bad = R.make_params(L=0)
    import ctypes
    assert L.dr_chains_init(r.h, 16, 1, 0, ctypes.byref(bad)) in (_lib.DR_ERR_INVALID_ARG, _lib.DR_ERR_STATE)
    scene = S.cornell_box(1, 8, 8)
    tris = scene.tris.copy()
    tris[0, 0] = 10 ** 6
    with pytest.raises(_lib.DRError) as e:
        r.upload_scene(S.Scene(scene.verts, tris, scene.tri_mat, scene.materials, scene.camera, 8, 8))
    assert e.value.code == _lib.DR_ERR_INVALID_ARG
    metal = S.cornell_box(1, 8, 8, metal=True)
    for slot in (2, 10):  # eta and k of a conductor must be > 0
        mats = metal.materials.copy()
        mats[mats[:, 0] == S.MAT_CONDUCTOR, slot] = 0.0
        with pytest.raises(_lib.DRError) as e:
            r.upload_scene(S.Scene(metal.verts, metal.tris, metal.tri_mat, mats, metal.camera, 8, 8))
        assert e.value.code == _lib.DR_ERR_INVALID_ARG
    # a non-finite vertex, a material index past the table, an unknown
    # material type: all rejected on the host
    for bad in ("vertex", "material index", "material type"):
        v, tm, mats = scene.verts.copy(), scene.tri_mat.copy(), scene.materials.copy()
        if bad == "vertex":
            v[3, 1] = np.nan
        elif bad == "material index":
            tm[5] = mats.shape[0]
        else:
            mats[0, 0] = 7.0
        with pytest.raises(_lib.DRError) as e:
            r.upload_scene(S.Scene(v, scene.tris, tm, mats, scene.camera, 8, 8))
        assert e.value.code == _lib.DR_ERR_INVALID_ARG, bad
    r.upload_scene(scene)
    r.init_chains(64, 1, R.make_params(L=3, drift="adjoint", k0=100.0))
    r.step(2)
    assert r.counters()["steps"] == 2
    r.close()


@pytest.mark.parametrize("wavefront", [0, 1])
def test_chain_parity_longest_paths(torch, R, oracle, wavefront):
    """The largest PSS the library takes: L = 16 (d = 62) on the glossy Cornell
    box, in both execution modes."""
    scene = S.cornell_box(1, 64, 64, glossy=True)
    k0 = 1e6
    pg = R.make_params(L=16, drift="adjoint", rb=True, k0=k0, steps_per_splat=4)
    po = oracle.make_params(L=16, drift="exact", rb=True, k0=k0)
    r_opts = {"wavefront": wavefront}
    frac, first, n = _chain_parity_opts(torch, R, oracle, scene, pg, po, N=2048, M=128, T=6, seed=61, opts=r_opts)
    print("L = 16 divergent fraction", frac)
    assert frac <= 0.02


def test_chain_parity_camera_only_paths(torch, R, oracle):
    """L = 1 (d = 2): only the emission seen directly through each pixel."""
    scene = S.cornell_box(1, 32, 32)
    k0 = 500.0
    pg = R.make_params(L=1, drift="adjoint", rb=True, k0=k0, steps_per_splat=4)
    po = oracle.make_params(L=1, drift="exact", rb=True, k0=k0)
    frac, first, n = _chain_parity(torch, R, oracle, scene, pg, po, N=4096, M=512, T=8, seed=62)
    assert frac <= 0.01


@pytest.mark.parametrize("chains", [1, 33, 1000])
def test_ragged_chain_counts(torch, R, oracle, chains):
    """Chain counts that fill no warp or block exactly, down to a single
    chain, through the bounce-by-bounce passes with every option on."""
    scene = S.procedural_scene(2, 48, 32, target_tris=30000, n_objects=20)
    k0 = 2.0e6
    pg = R.make_params(L=6, drift="adjoint", rb=True, k0=k0, steps_per_splat=4)
    po = oracle.make_params(L=6, drift="exact", rb=True, k0=k0)
    opts = {"wavefront": 1, "ray_order": 1, "tail_bounce": 3}
    frac, first, n = _chain_parity_opts(torch, R, oracle, scene, pg, po, N=chains, M=chains, T=6, seed=63,
                                        opts=opts)
    assert frac <= (0.0 if chains < 100 else 0.01)


def test_zero_steps_and_size_limits(torch, R):
    from paper_2605_08916_gb300 import _lib
    import ctypes
    stream = torch.cuda.Stream()
    r = R.Renderer(0, stream)
    r.upload_scene(S.cornell_box(1, 8, 8))
    prm = R.make_params(L=3, drift="adjoint", k0=100.0)
    L = _lib.load()
    assert L.dr_chains_init(r.h, (1 << 31) + 1, 1, 0, ctypes.byref(prm)) == _lib.DR_ERR_INVALID_ARG
    assert L.dr_chains_init(r.h, 0, 1, 0, ctypes.byref(prm)) == _lib.DR_ERR_INVALID_ARG
    r.init_chains(256, 1, prm)
    before = r.readback_state(("x",))["x"]
    r.step(0)
    r.frame(0)
    stream.synchronize()
    assert np.array_equal(before, r.readback_state(("x",))["x"])
    assert r.counters()["steps"] == 0
    r.close()


def small_instanced():
    return S.procedural_scene_instanced(1, 64, 36, target_tris=60000, n_objects=40)


def test_instanced_upload_is_its_flattening(torch, R):
    """The library's flattening of an instanced scene equals the one the
    oracle takes (same FP64 formulas, no contraction): with the two-level
    walk off, chains on the instanced upload and on the flat upload of the
    Python flattening are bit-identical."""
    isc = small_instanced()
    out = []
    for inst in (True, False):
        r = R.Renderer()
        r.set_option("wavefront", 1)
        if inst:
            r.set_option("two_level", 1)
            r.upload_instanced(isc)
            assert r.two_level_info() is not None
            r.set_option("two_level", 0)  # built, not walked
        else:
            r.upload_scene(isc.flatten())
        r.init_chains(16384, 41, R.make_params(L=12, drift="adjoint", k0=0.0, steps_per_splat=4))
        r.step(6)
        out.append(r.readback_state())
        r.close()
    a, b = out
    for k in ("x", "killed", "logp", "score", "pix"):
        assert np.array_equal(a[k], b[k]), k


def test_two_level_hits_match_flat_and_oracle(torch, R, oracle):
    """Rays through the two-level BVH (object-space triangle tests) hit the
    same triangles as the flattened scene's BVH and the oracle, up to hits
    on shared edges; distances agree to the FP32 rounding of the mapped
    rays."""
    isc = small_instanced()
    flat = isc.flatten()
    o, d = random_rays(flat, 20000, 5)
    rays = torch.from_numpy(np.concatenate([o, d], 1)).cuda()
    r = R.Renderer()
    r.set_option("two_level", 1)
    r.upload_instanced(isc)
    info = r.two_level_info()
    assert info is not None and info["n_instances"] == len(isc.instances)
    tri_t, t_t = r.trace_closest(rays)
    r.close()
    r = R.Renderer()
    r.upload_scene(flat)
    tri_f, t_f = r.trace_closest(rays)
    r.close()
    torch.cuda.synchronize()
    tri_t, t_t, tri_f, t_f = tri_t.cpu().numpy(), t_t.cpu().numpy(), tri_f.cpu().numpy(), t_f.cpu().numpy()
    same = tri_t == tri_f
    assert same.mean() >= 0.999, same.mean()
    hit = same & (tri_f >= 0)
    # object-space distances carry the rounding of the mapped ray origin
    assert np.allclose(t_t[hit], t_f[hit], rtol=1e-4, atol=1e-5)
    tri_o, t_o = oracle.OracleScene(flat).trace(o.astype(np.float64), d.astype(np.float64))
    assert (tri_t == tri_o).mean() >= 0.999


@pytest.mark.parametrize("tail", [0, 4])
def test_two_level_chains_match_the_flat_walk(torch, R, tail):
    """Restore steps walking the two-level BVH vs the flattened BVH of the
    same instanced upload: the hit point and shading always come from the
    flattened triangle, so chains whose hits agree are bit-identical."""
    isc = small_instanced()
    out = []
    for tl in (1, 0):
        r = R.Renderer()
        r.set_option("wavefront", 1)
        r.set_option("two_level", 1)
        r.set_option("tail_bounce", tail)
        r.upload_instanced(isc)
        r.set_option("two_level", tl)  # the same upload, either walk
        r.init_chains(16384, 43, R.make_params(L=12, drift="adjoint", k0=0.0, steps_per_splat=4))
        r.step(9)
        out.append((r.readback_state(), r.readback_accum()))
        r.close()
    (a, acc_a), (b, acc_b) = out
    same = (a["killed"] == b["killed"]) & (a["pix"] == b["pix"]) & np.all(a["x"] == b["x"], 1)
    same &= a["logp"] == b["logp"]
    print(f"bit-identical chains {same.mean():.5f}")
    assert same.mean() >= 0.999
    assert np.allclose(acc_a, acc_b, rtol=1e-3, atol=1e-9 * np.abs(acc_a).max())


def test_chain_parity_instanced_two_level(torch, R, oracle):
    """An instanced scene on the two-level walk against the oracle on its
    flattening, 16-step horizons."""
    isc = small_instanced()
    flat = isc.flatten()
    k0 = 1e6
    pg = R.make_params(L=8, drift="adjoint", rb=True, k0=k0, steps_per_splat=16)
    po = oracle.make_params(L=8, drift="exact", rb=True, k0=k0)
    orig = R.Renderer

    class _R(orig):
        def upload_scene(self, scene):
            self.set_option("wavefront", 1)
            self.set_option("two_level", 1)
            self.upload_instanced(isc)

    R.Renderer = _R
    try:
        frac, first, n = _chain_parity(torch, R, oracle, flat, pg, po, N=16384, M=512, T=16, seed=12)
    finally:
        R.Renderer = orig
    print("instanced two-level divergent fraction", frac, "compared", n)
    assert frac <= 0.01


def test_instanced_upload_errors(torch, R):
    from paper_2605_08916_gb300 import _lib
    isc = small_instanced()
    bad = S.InstancedScene(isc.meshes, [(0, -1, [0.0] * 12)] + isc.instances[1:], isc.materials, isc.camera,
                           isc.width, isc.height)
    r = R.Renderer()
    with pytest.raises(_lib.DRError) as e:
        r.upload_instanced(bad)  # singular map
    assert e.value.code == _lib.DR_ERR_INVALID_ARG
    bad = S.InstancedScene(isc.meshes, [(len(isc.meshes), -1, isc.instances[0][2])], isc.materials, isc.camera,
                           isc.width, isc.height)
    with pytest.raises(_lib.DRError) as e:
        r.upload_instanced(bad)  # mesh index out of range
    assert e.value.code == _lib.DR_ERR_INVALID_ARG
    r.upload_instanced(isc)
    assert r.two_level_info() is None  # not asked for
    r.init_chains(64, 1, R.make_params(L=3, drift="adjoint", k0=100.0))
    r.step(2)
    r.close()


# ---------------------------------------------------------------------------
# Independent count of the traversal's work (the roofline's algorithmic
# bytes are 112 B per node step and 48 B per triangle test, summed by the
# library's statistics instantiation).  A host walker written from the
# documented BVH layout and walk rules visits the downloaded 4-wide BVH:
# hit children nearest first (ties by slot), the others pushed far-to-near,
# leaves tested on the spot, boxes culled against the closest hit so far.

_F = np.float32


def _fma32(a, b, c):
    # a * b is exact in float64 for float32 inputs; one rounding to float32
    return _F(np.float64(a) * np.float64(b) + np.float64(c))


def _cross32(a, b):
    return [_F(a[1] * b[2] - a[2] * b[1]), _F(a[2] * b[0] - a[0] * b[2]), _F(a[0] * b[1] - a[1] * b[0])]


def _dot32(a, b):
    return _F(_F(a[0] * b[0]) + _F(a[1] * b[1]) + _F(a[2] * b[2]))


def _tri_test32(v0, e1, e2, o, d, tmin, tmax):
    p = _cross32(d, e2)
    det = _dot32(e1, p)
    if det == 0:
        return None
    sg = _F(-1.0) if det < 0 else _F(1.0)
    adet = abs(det)
    tv = [_F(o[i] - v0[i]) for i in range(3)]
    du = _dot32(tv, p)
    if du * sg < 0 or du * sg > adet:
        return None
    q = _cross32(tv, e1)
    dv = _dot32(d, q)
    if dv * sg < 0 or _F(du + dv) * sg > adet:
        return None
    inv = _F(1.0) / det
    u = _F(du * inv)
    if u < 0 or u > 1:
        return None
    v = _F(dv * inv)
    if v < 0 or _F(u + v) > 1:
        return None
    t = _F(_dot32(e2, q) * inv)
    return t if (t > tmin and t < tmax) else None


def _walk4_counts(nodes, tris, links, tri_ids, o, d, tmin):
    """Closest hit, node steps and triangle tests of one ray."""
    o = [_F(x) for x in o]
    d = [_F(x) for x in d]
    inv = []
    for v in d:
        vv = v if abs(v) > _F(1e-20) else _F(np.copysign(_F(1e-20), v))
        inv.append(_F(_F(1.0) / vv))
    oinv = [_F(o[a] * inv[a]) for a in range(3)]
    kM = _F(2.384185791015625e-07)
    on = [_fma32(abs(oinv[a]), kM, oinv[a]) for a in range(3)]
    of = [_fma32(-abs(oinv[a]), kM, oinv[a]) for a in range(3)]
    sx = [1 if inv[a] < 0 else 0 for a in range(3)]
    tbest, best = _F(np.inf), -1
    stack, node, n_steps, n_tests = [], 0, 0, 0
    while True:
        if node < 0:
            first, cnt = (node & 0x7fffffff) >> 3, (node & 7) + 1
            tmax = _F(tbest * _F(1.0000001) + _F(1e-30))
            for i in range(first, first + cnt):
                n_tests += 1
                rec = tris[i]
                th = _tri_test32(rec[0:3], rec[4:7], rec[8:11], o, d, tmin, tmax)
                tid = int(tri_ids[i])
                if th is not None and (th < tbest or (th == tbest and tid < best)):
                    tbest, best = th, tid
            if not stack:
                break
            node = stack.pop()
            continue
        n_steps += 1
        nb = nodes[node]
        keys = []
        for k in range(4):
            tn = _F(0.0)
            tf = tbest
            for a in range(3):
                near = nb[(2 * a + sx[a]) * 4 + k]
                far = nb[(2 * a + 1 - sx[a]) * 4 + k]
                tn = max(tn, _fma32(near, inv[a], -on[a]))
                tf = min(tf, _fma32(far, inv[a], -of[a]))
            e = tn if tn <= _F(tf * _F(1.0000002)) else _F(-1.0)
            c = int(links[node, k])
            if c != 0x7fffffff and e >= 0 and e <= tbest:
                keys.append(((int(np.array(e, np.float32).view(np.uint32)) & ~3) | k, c))
        if not keys:
            if not stack:
                break
            node = stack.pop()
            continue
        keys.sort()
        node = keys[0][1]
        for _, c in reversed(keys[1:]):
            stack.append(c)
    return best, n_steps, n_tests


def test_node_steps_match_an_independent_walk(torch, R):
    scene = S.procedural_scene(3, 64, 36, target_tris=30000, n_objects=24)
    r = R.Renderer()
    r.upload_scene(scene)
    nodes, tris = r.bvh4_download()
    links = nodes[:, 24:28].view(np.int32)
    tri_ids = tris[:, 3].view(np.int32)
    lo, hi = scene.verts.min(0).astype(np.float64), scene.verts.max(0).astype(np.float64)
    tmin = _F(1e-5 * float((hi - lo).max()))
    rng = np.random.default_rng(4)
    n = 1500
    # rays leaving points on triangles (secondary-ray-like) and rays from
    # inside the scene box, in uniformly random directions
    k = rng.integers(0, scene.n_tris, n)
    bu, bv = rng.random(n), rng.random(n)
    flip = bu + bv > 1
    bu[flip], bv[flip] = 1 - bu[flip], 1 - bv[flip]
    v0, v1, v2 = (scene.verts[scene.tris[k, i]].astype(np.float64) for i in range(3))
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True) + 1e-30
    o = v0 + bu[:, None] * (v1 - v0) + bv[:, None] * (v2 - v0) + nrm * (2e-3 * float((hi - lo).max()))
    o[n // 2:] = lo + rng.random((n - n // 2, 3)) * (hi - lo)
    dr = rng.normal(size=(n, 3))
    dr /= np.linalg.norm(dr, axis=1, keepdims=True)
    rays = np.concatenate([o, dr], 1).astype(np.float32)
    hit, _, steps, tests = r.trace_closest_counted(torch.from_numpy(rays).cuda())
    hit, steps, tests = hit.cpu().numpy(), steps.cpu().numpy(), tests.cpu().numpy()
    r.close()
    ref = np.array([_walk4_counts(nodes, tris, links, tri_ids, rays[i, :3], rays[i, 3:], tmin) for i in range(n)])
    same_hit = hit == ref[:, 0]
    same_steps = (steps == ref[:, 1]) & (tests == ref[:, 2])
    print(f"independent walk: hits {same_hit.mean():.4f}, per-ray counts {same_steps.mean():.4f}, "
          f"node steps {steps.sum()} vs {ref[:, 1].sum()}, tests {tests.sum()} vs {ref[:, 2].sum()}")
    assert (ref[:, 0] >= 0).mean() > 0.3 and steps.mean() > 5
    assert same_hit.mean() >= 0.998
    assert same_steps.mean() >= 0.99
    assert abs(steps.sum() / ref[:, 1].sum() - 1) <= 0.005
    assert abs(tests.sum() / ref[:, 2].sum() - 1) <= 0.005
