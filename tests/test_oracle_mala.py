"""Pins of the oracle's MALA Restore (the comparison method of Sec. 6: Jump
Restore with Metropolis-adjusted Langevin local moves and holding rate 1).

The Metropolis-Hastings test makes the local kernel pi-invariant, so the
killing rate k0 / p is the invariant one (Eq. invariant-killing-rate with
L* p = 0): the Restore estimate is exact for any step size, jumps included.
The pins check what that fixes:

M1  a density with a jump (c1 = 1 | c2 = 4): the mass of the low half is
    0.2 within the standard error at the paper's stddev = 5e-3, where the
    unadjusted Diffusion Restore move is biased (tests/test_oracle_bias.py);
M2  Gaussian-mixture moments at a step (stddev = 0.05) far too large for an
    unadjusted move: MALA Restore within 3.5 standard errors, the same move
    without the adjustment rejected;
M3  the Restore image of the 16 x 16 Cornell box at the paper's stddev
    matches path tracing of the same f within 3 sigma per pixel (the
    check P6 makes for Diffusion Restore only in the no-motion limit).
"""
import math

import numpy as np

from paper_2605_08916_gb300 import scenes as S

M_TOUR = 64


def _half_mass_estimate(oracle, tgt, prm, n_tours, seeds):
    ests, acc_rates = [], []
    for b in range(seeds):
        r = oracle.restore_tours(tgt, prm, seed=2000 + b, chain_ids=np.arange(n_tours // seeds), image=True)
        assert r["truncated"].sum() == 0
        a = r["accum"][:, 0]
        ests.append(a[0] / a.sum())
    return float(np.mean(ests)), float(np.std(ests, ddof=1) / math.sqrt(seeds))


def test_mala_restore_is_exact_across_a_jump(oracle):
    tgt = oracle.target(S.StepDensity(w=0.0))
    p_lambda = 2.5
    mala = oracle.make_params(L=1, drift="mala", rb=True, stddev=5e-3, dt=1.0, k0=p_lambda / M_TOUR)
    est, se = _half_mass_estimate(oracle, tgt, mala, 400000, 8)
    print(f"MALA Restore half mass {est:.4f} +- {se:.4f} (exact 0.2)")
    assert abs(est - 0.2) < 4 * se
    assert se < 0.002
    # the unadjusted move with the same proposal and clock is biased
    ula = oracle.make_params(L=1, drift="exact", rb=True, stddev=5e-3, dt=1.0, gamma_tilde=0.0,
                             k0=p_lambda / M_TOUR)
    est_u, se_u = _half_mass_estimate(oracle, tgt, ula, 400000, 8)
    print(f"unadjusted half mass {est_u:.4f} +- {se_u:.4f}")
    assert est_u - 0.2 > 10 * se_u


def _wrapped_moments_1d(mu, s, n=20001):
    x = (np.arange(n) + 0.5) / n
    dd = x - mu
    dd -= np.round(dd)
    w = np.exp(-0.5 * dd * dd / (s * s))
    w /= w.sum()
    return float((w * x).sum()), float((w * x * x).sum())


def test_mala_restore_mixture_moments_at_a_large_step(oracle):
    d, K = 2, 2
    w = np.array([0.4, 0.6])
    mu = np.array([[0.35, 0.4], [0.65, 0.62]])
    sig = np.array([0.08, 0.1])
    mix = S.Mixture(d, w, mu, sig, 4, 4)
    tgt = oracle.target(mix)
    m1 = np.zeros(d)
    m2d = np.zeros(d)
    for k in range(K):
        for i in range(d):
            e1, e2 = _wrapped_moments_1d(mu[k, i], sig[k])
            m1[i] += w[k] * e1
            m2d[i] += w[k] * e2
    M = 200000
    out = {}
    for drift in ("mala", "exact"):
        prm = oracle.make_params(L=1, drift=drift, rb=True, stddev=0.05, dt=1.0, gamma_tilde=0.0, k0=1.0 / M_TOUR)
        r = oracle.restore_tours(tgt, prm, seed=7, chain_ids=np.arange(M))
        assert r["truncated"].sum() == 0
        A1, Ax, Axx = r["I1"], r["Ix"], r["Ixx"]
        e1 = Ax.sum(0) / A1.sum()
        e2 = np.array([Axx[:, i, i].sum() for i in range(d)]) / A1.sum()
        mA = A1.mean()
        se1 = np.sqrt(np.var(Ax - e1[None] * A1[:, None], axis=0) / M) / mA
        se2 = np.sqrt(np.var(np.stack([Axx[:, i, i] for i in range(d)], 1) - e2[None] * A1[:, None], axis=0) / M) / mA
        out[drift] = (np.abs(e1 - m1) / se1, np.abs(e2 - m2d) / se2)
        print(drift, "z first moments", out[drift][0], "z second moments", out[drift][1])
    z1, z2 = out["mala"]
    assert z1.max() < 3.5 and z2.max() < 3.5
    zu1, zu2 = out["exact"]
    assert max(zu1.max(), zu2.max()) > 8.0     # the unadjusted move at this step is biased
    # a narrow Gaussian (s = 0.03) at a step as wide as the mode: the
    # Langevin shift of the reverse proposal, at the proposed point, is a
    # large part of the step, so the Hastings ratio must use the score there
    s_, c_ = 0.03, 0.5
    tgt1 = oracle.target(S.single_gaussian([c_, c_], s_))
    prm = oracle.make_params(L=1, drift="mala", rb=True, stddev=0.03, dt=1.0, gamma_tilde=0.0, k0=1.0 / M_TOUR)
    r = oracle.restore_tours(tgt1, prm, seed=9, chain_ids=np.arange(M))
    A1, Ax, Axx = r["I1"], r["Ix"][:, 0], r["Ixx"][:, 0, 0]
    m1_, m2_ = Ax.sum() / A1.sum(), Axx.sum() / A1.sum()
    var_est = m2_ - m1_ * m1_
    infl = (Axx - m2_ * A1) - 2 * m1_ * (Ax - m1_ * A1)
    se_v = np.sqrt(np.var(infl) / M) / A1.mean()
    e1, e2 = _wrapped_moments_1d(c_, s_)
    print(f"narrow Gaussian variance {var_est:.6e} vs {e2 - e1 * e1:.6e} (+- {se_v:.1e})")
    assert abs(var_est - (e2 - e1 * e1)) < 3.5 * se_v


def test_mala_restore_cornell_image_matches_path_tracing(oracle):
    scene = S.cornell_box(1, 16, 16)
    L = 4
    tgt = oracle.OracleScene(scene)
    xs = np.random.default_rng(11).random((20000, S.pss_dim(L)))
    p_hat = float(np.mean(np.exp(oracle.evaluate(tgt, xs, L)["logp"])))
    k0 = p_hat / M_TOUR
    prm = oracle.make_params(L=L, drift="mala", rb=True, k0=k0, stddev=5e-3, dt=1.0)
    M, n_seeds = 4096, 12
    imgs, steps = [], []
    for s in range(n_seeds):
        r = oracle.restore_tours(tgt, prm, seed=700 + s, chain_ids=np.arange(M), image=True)
        assert r["truncated"].sum() == 0
        imgs.append(oracle.resolve(r["accum"], k0, M))
        steps.append(r["steps"].mean())
    imgs = np.array(imgs)
    mean = imgs.mean(0)
    var = imgs.var(0, ddof=1) / n_seeds
    ref, ref_var = oracle.pt_image(tgt, L, 1 << 12, seed=3)
    z = (mean - ref) / np.sqrt(var + ref_var + 1e-300)
    print(f"MALA Restore at stddev 5e-3: image sum ratio {mean.sum() / ref.sum():.4f}, |z|<3: "
          f"{np.mean(np.abs(z) < 3):.3f}, mean z^2 {np.mean(z ** 2):.2f}, mean tour {np.mean(steps):.1f} steps")
    assert abs(mean.sum() / ref.sum() - 1.0) < 0.03
    assert np.mean(np.abs(z) < 3) >= 0.97
    assert np.mean(z ** 2) < 1.6
