"""Pins of the oracle's path contribution f(x), its gradient, the BSDFs and
Philox against things fixed by mathematics or by independent code.

P4  grad log p by forward-mode duals == central finite differences (FP64)
    on points whose discrete choices do not change within +-h.
P5  (i) BVH closest hit == brute force (identical triangle ids and t);
    (ii) white furnace: closed room reflecting with albedo a and emitting Le
    everywhere has radiance sum_{k<L} a^k Le after L segments;
    (iii) one bounce under a parallel coaxial square emitter: radiance
    albedo * Le * F with F the point-to-parallel-square form factor;
    (iv) BSDF sampler vs its pdf: E[g / pdf] = integral of g over the
    hemisphere for g = 1 and g = cos; sampler weight == fs cos / pdf;
    reciprocity; energy <= 1;
    (v) conductor Fresnel (complex index) vs the normal-incidence closed
    form, the dielectric equations at k = 0, the grazing limit and the
    real-variable (a, b) form of the same equations.
P7  Philox4x32-10 (cited in Sec. 4.3) vs Triton's independent implementation
    run by its CPU interpreter.
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2605_08916_gb300 import scenes as S


def _info_equal(a, b):
    return np.array_equal(a, b)


def test_gradient_matches_central_differences(oracle):
    O = oracle
    for scene, L in [(S.cornell_box(1, 16, 16), 4), (S.cornell_box(2, 16, 16, glossy=True), 5),
                     (S.cornell_box(3, 16, 16, metal=True), 5),
                     (S.caustic_scene(1, 16, 16, n_theta=12, n_phi=12), 6)]:
        tgt = O.target(scene)
        d = S.pss_dim(L)
        rng = np.random.default_rng(11)
        x = rng.random((300, d))
        r = O.evaluate(tgt, x, L, grad=True, info=True)
        h = 1e-6
        checked = 0
        for m in range(x.shape[0]):
            if not np.isfinite(r["logp"][m]) or r["f"][m].sum() <= 0:
                continue
            for i in range(d):
                xp = x[m].copy()
                xm = x[m].copy()
                xp[i] += h
                xm[i] -= h
                rp = O.evaluate(tgt, xp[None], L, info=True)
                rm = O.evaluate(tgt, xm[None], L, info=True)
                if not (_info_equal(rp["info"][0], r["info"][m]) and _info_equal(rm["info"][0], r["info"][m])):
                    continue
                if rp["pix"][0] != r["pix"][m] or rm["pix"][0] != r["pix"][m]:
                    continue
                fd = (rp["logp"][0] - rm["logp"][0]) / (2 * h)
                g = r["grad"][m, i]
                assert abs(fd - g) <= 1e-5 * max(1.0, abs(g)) + 2e-4 * abs(g), (scene.name, m, i, fd, g)
                checked += 1
        assert checked > 200, (scene.name, checked)


def test_bvh_matches_brute_force(oracle):
    O = oracle
    scene = S.caustic_scene(1, 8, 8, n_theta=20, n_phi=20)
    bvh = O.OracleScene(scene, use_bvh=True)
    brute = O.OracleScene(scene, use_bvh=False)
    rng = np.random.default_rng(3)
    o = rng.uniform(-2.5, 2.5, (20000, 3)) + np.array([0.0, 1.5, 0.5])
    d = rng.normal(size=(20000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t1, h1 = bvh.trace(o, d)
    t2, h2 = brute.trace(o, d)
    assert np.array_equal(t1, t2)
    hit = t1 >= 0
    assert hit.mean() > 0.8   # origins below the floor see nothing
    assert np.array_equal(h1[hit], h2[hit])


@pytest.mark.parametrize("L", [1, 2, 4])
def test_white_furnace(oracle, L):
    O = oracle
    a, Le = 0.5, 1.0
    scene = S.furnace_box(albedo=a, emission=Le, width=4, height=4)
    tgt = O.target(scene)
    d = S.pss_dim(L)
    rng = np.random.default_rng(1)
    x = rng.random((40000, d))
    f = O.evaluate(tgt, x, L)["f"][:, 0] / (scene.width * scene.height)
    expect = sum(a ** k for k in range(L)) * Le
    se = f.std() / math.sqrt(f.size)
    assert abs(f.mean() - expect) < 4 * se + 1e-12, (f.mean(), expect, se)
    if L == 1:
        assert np.allclose(f, Le)


def _form_factor_point_to_square(half, height):
    """Differential area to a parallel square of half side `half` centred
    above it at distance `height`: four corner rectangles (Howell's catalog
    configuration: differential element below one corner of a rectangle)."""
    A = B = half / height

    def corner(A, B):
        return (A / math.sqrt(1 + A * A) * math.atan(B / math.sqrt(1 + A * A)) +
                B / math.sqrt(1 + B * B) * math.atan(A / math.sqrt(1 + B * B))) / (2 * math.pi)

    return 4 * corner(A, B)


def test_single_bounce_form_factor(oracle):
    O = oracle
    half, hgt, alb, Le = 0.5, 1.0, 0.5, 1.0
    scene = S.parallel_squares(half_light=half, height=hgt, albedo=alb, radiance=Le)
    tgt = O.target(scene)
    L = 2
    d = S.pss_dim(L)
    rng = np.random.default_rng(2)
    x = rng.random((200000, d))
    x[:, 0] = 0.5
    x[:, 1] = 0.5
    f = O.evaluate(tgt, x, L)["f"][:, 0]
    F = _form_factor_point_to_square(half, hgt)
    expect = alb * Le * F
    se = f.std() / math.sqrt(f.size)
    assert abs(f.mean() - expect) < 4 * se, (f.mean(), expect, se)
    assert se < 0.01 * expect


GLOSSY = S.material(S.MAT_GLOSSY, (0.7, 0.5, 0.3), roughness=0.15, f0=0.04)
DIFFUSE = S.material(S.MAT_DIFFUSE, (0.7, 0.5, 0.3))
METAL = S.conductor((0.2, 1.1, 1.5), (3.0, 2.5, 2.0), roughness=0.5)


@pytest.mark.parametrize("mat", [GLOSSY, DIFFUSE, METAL], ids=["glossy", "diffuse", "conductor"])
def test_bsdf_sampler_matches_pdf(oracle, mat):
    O = oracle
    n = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(4)
    for theta in [0.2, 0.8, 1.3]:
        wo = np.array([math.sin(theta), 0.0, math.cos(theta)])
        s1 = s_cos = 0.0
        cnt = 40000
        vals1, valsc = [], []
        for _ in range(cnt):
            u1, u2 = rng.random(2)
            ok, wi, w, pdf, lobe = O.bsdf_sample(mat, n, wo, u1, u2)
            if not ok:
                vals1.append(0.0)
                valsc.append(0.0)
                continue
            fs, pdf2 = O.bsdf_eval(mat, n, wo, wi)
            assert abs(pdf - pdf2) <= 1e-12 * pdf2
            assert np.allclose(w, fs * wi[2] / pdf2, rtol=1e-12)
            fs_rev, _ = O.bsdf_eval(mat, n, wi, wo)
            assert np.allclose(fs, fs_rev, rtol=1e-12)
            vals1.append(1.0 / pdf)
            valsc.append(wi[2] / pdf)
        v1, vc = np.array(vals1), np.array(valsc)
        # pdf > 0 on the whole upper hemisphere (the cosine lobe of the
        # mixtures; for the conductor, D(h) > 0 for every half-vector above
        # the surface): E[1/pdf] = 2 pi and E[cos/pdf] = pi exactly
        assert abs(v1.mean() - 2 * math.pi) < 4 * v1.std() / math.sqrt(cnt)
        assert abs(vc.mean() - math.pi) < 4 * vc.std() / math.sqrt(cnt)


def test_ggx_lobe_white_furnace(oracle):
    """Specular lobe alone (albedo 0, F0 = 1): the single-scattering GGX
    furnace integral of D G2 / (4 cos_o cos_i) * cos_i never exceeds 1 and
    is close to 1 for a smooth surface at near-normal incidence (only
    multiple-scattering energy is lost)."""
    O = oracle
    n = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(5)
    prev = 2.0
    for rough, theta, lo in [(0.05, 0.2, 0.98), (0.3, 0.2, 0.5), (0.5, 0.2, 0.4)]:
        mirror = S.material(S.MAT_GLOSSY, (0.0, 0.0, 0.0), roughness=rough, f0=1.0)
        wo = np.array([math.sin(theta), 0.0, math.cos(theta)])
        acc = []
        for _ in range(20000):
            ok, wi, w, pdf, lobe = O.bsdf_sample(mirror, n, wo, *rng.random(2))
            acc.append(w[0] if ok else 0.0)
        acc = np.array(acc)
        se = acc.std() / math.sqrt(acc.size)
        assert lo <= acc.mean() <= 1.0 + 4 * se, (rough, theta, acc.mean())
        # single-scattering energy loss grows with roughness
        assert acc.mean() < prev
        prev = acc.mean()


def test_conductor_lobe_matches_ggx_coat_lobe(oracle):
    """A conductor with a huge extinction k reflects everything (F -> 1),
    so its single-scattering albedo equals that of the glossy material's
    specular lobe with F0 = 1 and no base (the same D G2 / (4 cos cos)
    integral), although the two are sampled differently (one lobe vs a
    half/half mixture with the cosine lobe)."""
    O = oracle
    n = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(6)
    for rough, theta in [(0.1, 0.3), (0.4, 1.0)]:
        metal = S.conductor((1.0, 1.0, 1.0), (1e6, 1e6, 1e6), roughness=rough)
        coat = S.material(S.MAT_GLOSSY, (0.0, 0.0, 0.0), roughness=rough, f0=1.0)
        wo = np.array([math.sin(theta), 0.0, math.cos(theta)])
        est = []
        for mat in (metal, coat):
            acc = np.array([(lambda r: r[2][1] if r[0] else 0.0)(O.bsdf_sample(mat, n, wo, *rng.random(2)))
                            for _ in range(30000)])
            est.append((acc.mean(), acc.std() / math.sqrt(acc.size)))
        (m1, s1), (m2, s2) = est
        assert m1 <= 1.0 + 4 * s1
        assert abs(m1 - m2) < 4 * math.hypot(s1, s2), (rough, theta, est)


def test_fresnel_conductor_closed_forms(oracle):
    L = oracle.lib()
    for eta, k in [(0.2, 3.0), (1.1, 2.5), (0.05, 5.0), (2.0, 0.5)]:
        # normal incidence: ((eta - 1)^2 + k^2) / ((eta + 1)^2 + k^2)
        ref = ((eta - 1) ** 2 + k * k) / ((eta + 1) ** 2 + k * k)
        assert abs(L.orc_fresnel_conductor(1.0, eta, k) - ref) < 1e-14
        # grazing incidence reflects everything
        assert L.orc_fresnel_conductor(1e-9, eta, k) > 1 - 1e-7
        # the same equations in real variables (a^2 + b^2 from the complex
        # index, then R_s and R_p as real ratios), a separate formulation
        for ci in (0.95, 0.6, 0.25, 0.02):
            s2 = 1 - ci * ci
            t0 = eta * eta - k * k - s2
            ab = math.sqrt(t0 * t0 + 4 * eta * eta * k * k)
            a = math.sqrt(0.5 * (ab + t0))
            rs = (ab + ci * ci - 2 * a * ci) / (ab + ci * ci + 2 * a * ci)
            q = (ci * ci * ab + s2 * s2 - 2 * a * ci * s2) / (ci * ci * ab + s2 * s2 + 2 * a * ci * s2)
            ref = 0.5 * (rs + rs * q)
            assert abs(L.orc_fresnel_conductor(ci, eta, k) - ref) < 1e-13, (eta, k, ci)
    # k = 0 is a dielectric interface: the real Fresnel equations
    eta = 1.5
    for ci in (0.9, 0.5, 0.1):
        ct = math.sqrt(1 - (1 - ci * ci) / eta ** 2)
        assert abs(L.orc_fresnel_conductor(ci, eta, 0.0) - L.orc_fresnel_dielectric(ci, ct, eta)) < 1e-15


def test_fresnel_dielectric_closed_forms(oracle):
    O = oracle
    eta = 1.5
    # normal incidence: ((eta - 1) / (eta + 1))^2
    assert abs(O.lib().orc_fresnel_dielectric(1.0, 1.0, eta) - ((eta - 1) / (eta + 1)) ** 2) < 1e-15
    # Brewster angle: rp = 0, so F = rs^2 / 2
    tb = math.atan(eta)
    ci = math.cos(tb)
    ct = math.sqrt(1 - (1 - ci * ci) / eta ** 2)
    rs = (ci - eta * ct) / (ci + eta * ct)
    assert abs(O.lib().orc_fresnel_dielectric(ci, ct, eta) - 0.5 * rs * rs) < 1e-15


def test_philox_matches_independent_implementation(oracle):
    """Triton's Philox (a separate implementation of the same published
    generator) run by its CPU interpreter in a subprocess."""
    pytest.importorskip("triton")
    code = textwrap.dedent("""
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import numpy as np, torch, triton, triton.language as tl
        @triton.jit
        def k(c_ptr, out_ptr, seed, n: tl.constexpr):
            i = tl.arange(0, n)
            c0 = tl.load(c_ptr + 4 * i + 0)
            c1 = tl.load(c_ptr + 4 * i + 1)
            c2 = tl.load(c_ptr + 4 * i + 2)
            c3 = tl.load(c_ptr + 4 * i + 3)
            a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
            tl.store(out_ptr + 4 * i + 0, a)
            tl.store(out_ptr + 4 * i + 1, b)
            tl.store(out_ptr + 4 * i + 2, c)
            tl.store(out_ptr + 4 * i + 3, d)
        seeds = json.loads(sys.argv[1])
        ctr = np.array(json.loads(sys.argv[2]), np.uint32).reshape(-1, 4)
        res = []
        for s in seeds:
            out = torch.zeros(ctr.size, dtype=torch.int32)
            k[(1,)](torch.from_numpy(ctr.view(np.int32).ravel().copy()), out, s, ctr.shape[0])
            res.append((out.numpy().view(np.uint32)).tolist())
        print(json.dumps(res))
    """)
    rng = np.random.default_rng(9)
    ctr = rng.integers(0, 2 ** 32, (16, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    seeds = [0, 1, 0x5EED, 0x123456789ABCDEF, 2 ** 64 - 1]
    import json
    env = dict(os.environ)
    env["TRITON_INTERPRET"] = "1"
    out = subprocess.run([sys.executable, "-c", code, json.dumps(seeds), json.dumps(ctr.ravel().tolist())],
                         capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr[-300:])
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for s, r in zip(seeds, ref):
        key = np.tile(np.array([s & 0xFFFFFFFF, (s >> 32) & 0xFFFFFFFF], np.uint32), (ctr.shape[0], 1))
        mine = oracle.philox4x32_10(ctr, key)
        assert np.array_equal(mine.ravel(), np.array(r, np.uint32)), s


def _mixture_grad_logp(mix, x, eps):
    """Closed-form grad log(g + eps) of an isotropic Gaussian mixture on the
    torus (nearest-image differences): grad g = -sum_k c_k delta_k / s_k^2."""
    g = np.zeros(x.shape[0])
    gg = np.zeros_like(x)
    for k in range(mix.K):
        dd = x - mix.mu[k]
        dd -= np.round(dd)
        s2 = mix.sig[k] ** 2
        c = mix.w[k] * np.exp(-0.5 * (dd * dd).sum(1) / s2) / (2 * math.pi * s2) ** (0.5 * mix.d)
        g += c
        gg -= c[:, None] * dd / s2
    return gg / (g + eps)[:, None]


def test_fd_score_matches_mixture_gradient(oracle):
    """The finite-difference drift (Alg. 4's score by central differences,
    the plain form of the numerical study) against the mixture's closed-form
    gradient.  Central differences with step h err by at most
    h^2 / 6 max|d^3 log p|; with components of s >= 0.05 and points within
    three s of a mean, |d^3 log p| < (3 / s)^3 = 2.2e5, so at h = 1e-5 the
    truncation is below 4e-6 and FP64 rounding (1e-16 / h) below 1e-10.
    A dropped factor 2, a sign or an index error fails by orders of
    magnitude.  Points next to the torus seam (a coordinate within h of 0)
    check that x +- h wraps: the nearest-image density is smooth across it."""
    mix = S.gaussian_mixture(seed=7, d=4, K=3, sig_range=(0.05, 0.09))
    tgt = oracle.target(mix)
    rng = np.random.default_rng(12)
    comp = rng.integers(0, mix.K, 400)
    x = mix.mu[comp] + rng.normal(size=(400, mix.d)) * mix.sig[comp][:, None] * rng.uniform(0, 1, (400, 1))
    x -= np.floor(x)
    # points on the seam of a component moved next to it
    seam = S.single_gaussian([0.0, 0.3, 0.6, 0.99], 0.06)
    xs = np.array([[1e-6, 0.31, 0.58, 0.985], [0.999999, 0.29, 0.61, 0.995], [0.02, 0.3, 0.6, 1e-7]])
    h, eps = 1e-5, 1e-8
    for m, pts, big in ((mix, x, 10.0), (seam, xs, 2.0)):
        t = oracle.target(m)
        s = oracle.fd_score(t, pts, L=1, eps=eps, h=h)
        ref = _mixture_grad_logp(m, pts, eps)
        err = np.abs(s - ref)
        assert np.all(err <= 4e-6 + 1e-9 * np.abs(ref)), err.max()
        assert np.abs(ref).max() > big
    # on a scene, a coordinate within h of the seam must be differenced
    # across it: the neighbour of 1 - h/2 at +h is h/2 (x lives on T^d)
    scene, L = S.cornell_box(1, 16, 16), 4
    st = oracle.target(scene)
    d = S.pss_dim(L)
    xq = np.random.default_rng(14).random((64, d))
    for i, at, hi, lo in ((4, 1.0 - h / 2, h / 2, 1.0 - 1.5 * h), (5, h / 2, 1.5 * h, 1.0 - h / 2)):
        xs_ = xq.copy()
        xs_[:, i] = at
        s = oracle.fd_score(st, xs_, L=L, eps=eps, h=h)[:, i]
        up, dn = xs_.copy(), xs_.copy()
        up[:, i] = hi
        dn[:, i] = lo
        ref = (oracle.evaluate(st, up, L)["logp"] - oracle.evaluate(st, dn, L)["logp"]) / (2 * h)
        assert np.allclose(s, ref, rtol=1e-6, atol=1e-6) and np.abs(ref).max() > 100.0, i
    # the dual gradient of the exact drift agrees too
    r = oracle.evaluate(tgt, x, L=1, grad=True)
    assert np.allclose(r["grad"], _mixture_grad_logp(mix, x, eps), rtol=1e-12, atol=1e-12)


def test_fd_score_matches_dual_gradient_on_scenes(oracle):
    """fd_score (FP64 central differences at h = 1e-6) against the
    forward-mode dual gradient of the same f on scene points whose discrete
    choices (triangles, lobes, light visibility, pixel) are the same at
    every x +- h e_i; the bound is that of P4."""
    h = 1e-6
    for scene, L in [(S.cornell_box(1, 16, 16), 4), (S.cornell_box(2, 16, 16, glossy=True), 5),
                     (S.caustic_scene(1, 16, 16, n_theta=12, n_phi=12), 6)]:
        tgt = oracle.target(scene)
        d = S.pss_dim(L)
        x = np.random.default_rng(13).random((800, d))
        r = oracle.evaluate(tgt, x, L, grad=True, info=True)
        lit = r["f"].sum(1) > 0
        x, g, info, pix = x[lit], r["grad"][lit], r["info"][lit], r["pix"][lit]
        M = x.shape[0]
        xp = np.repeat(x, d, 0)
        xm = xp.copy()
        idx = np.tile(np.arange(d), M)
        xp[np.arange(M * d), idx] += h
        xm[np.arange(M * d), idx] -= h
        same = np.ones(M, bool)
        for xx in (xp, xm):
            rr = oracle.evaluate(tgt, xx, L, info=True)
            ok = np.all(rr["info"] == np.repeat(info, d, 0), 1) & (rr["pix"] == np.repeat(pix, d, 0))
            same &= ok.reshape(M, d).all(1)
        s = oracle.fd_score(tgt, x[same], L=L, eps=1e-8, h=h)
        gs = g[same]
        assert same.sum() > 50, (scene.name, same.sum())
        assert np.all(np.abs(s - gs) <= 1e-5 * np.maximum(1.0, np.abs(gs)) + 2e-4 * np.abs(gs)), scene.name
