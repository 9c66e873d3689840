"""The bias of the modified killing rate (Sec. 5.2, Eq. bias and
Eq. adjoint-bias; App. C) on targets the mathematics fixes.

The Restore estimate with the modified killing rate k = k0 / p is biased by
-(L* p / p), where L f = h (K f - f) is the generator of the local dynamics
(K the Euler-Maruyama kernel of Alg. 4, h = 1 / dt).  Sec. 5.2 derives
L* p / p = O(dt) for a regular p.  These tests pin the oracle's App. C
diagnostic (L* p / p by quadrature) and read the claim on a density with a
jump, the situation of primary-sample-space path contributions (visibility
and light edges):

B1  For a Gaussian far from the torus edges the kernel is linear, so K* p
    is a Gaussian in closed form: the quadrature must reproduce
    h (K* p / p - 1) to its accuracy.
B2  Mass conservation: the integral of L* p over T^2 is 0 (K is a Markov
    kernel), for a smooth target with a steep transition.
B3  Sec. 5.2's O(dt): for a smooth density L* p / p halves when dt halves
    (sigma = stddev / sqrt(dt) held fixed).  For a jump of p (score 0 on both
    sides) K* p is the Gaussian-smoothed step in closed form, and near the
    jump L* p / p grows like 1 / dt instead: the premise of Eq. adjoint-bias
    fails.
B4  The Restore estimate itself (complete tours, renewal-reward ratio) of
    the mass of one half of a jump density c1 = 1 | c2 = 4 at the paper's
    stddev = 5e-3, dt = 1e-5, m = 64: biased (towards 1/2, the uniform
    occupation of unadjusted moves) with mean tours shorter than m + 1
    steps; the bias halves when dt drops by 4 at fixed sigma (O(sqrt(dt)),
    the boundary layer of width stddev sqrt(m)); and it vanishes once the
    jump is smoothed over about one step length stddev, where the drift
    sees the transition.
"""
import math

import numpy as np
import pytest

from paper_2605_08916_gb300 import scenes as S

STDDEV, DT, M_TOUR = 5e-3, 1e-5, 64


def _phi_cdf(z):
    return 0.5 * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))


def test_lstar_over_p_matches_the_gaussian_closed_form(oracle):
    """p = N(c, s^2 I) on T^2 (s = 0.08, c = (0.5, 0.5)): one Euler-Maruyama
    step maps X ~ N(c, s^2 I) to A X + b + stddev xi with
    A = (1 - a / s^2) I - (gt / s^2) J, b = (a I + gt J) c / s^2, a = stddev^2 / 2,
    so K* p = N(A c + b, s^2 A A^T + stddev^2 I) and
    L* p / p = h (K* p / p - 1).  The target's floor eps is set to 1e-30
    here, so that p and its score are the Gaussian's (with the default
    1e-8, K* p gains eps / |det A| and the score a relative eps / g)."""
    s, c = 0.08, np.array([0.5, 0.5])
    tgt = oracle.target(S.single_gaussian(c, s))
    a, gt = 0.5 * STDDEV ** 2, 0.5 * STDDEV ** 2
    J = np.array([[0.0, 1.0], [-1.0, 0.0]])
    A = (1 - a / s ** 2) * np.eye(2) - (gt / s ** 2) * J
    b = (a * np.eye(2) + gt * J) @ c / s ** 2
    mu2, cov2 = A @ c + b, s ** 2 * A @ A.T + STDDEV ** 2 * np.eye(2)
    rng = np.random.default_rng(3)
    y = c + rng.normal(size=(40, 2)) * s
    ic = np.linalg.inv(cov2)
    e = y - mu2
    kp = np.exp(-0.5 * np.einsum("ij,jk,ik->i", e, ic, e)) / (2 * math.pi * math.sqrt(np.linalg.det(cov2)))
    p = np.exp(-0.5 * ((y - c) ** 2).sum(1) / s ** 2) / (2 * math.pi * s * s)
    ref = (kp / p - 1.0) / DT
    got = oracle.lstar_over_p(tgt, y, stddev=STDDEV, dt=DT, eps=1e-30)
    assert np.abs(ref).max() > 0.05          # not trivially zero
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-6), np.abs(got - ref).max()


def _smooth_step(w):
    return S.StepDensity(w=w)


def test_lstar_p_integrates_to_zero(oracle):
    """K is a Markov kernel, so the integral of K* p equals that of p and the
    integral of L* p over T^2 vanishes (p depends on x0 only here)."""
    tgt = oracle.target(_smooth_step(0.02))
    n = 4000
    y0 = (np.arange(n) + 0.5) / n
    y = np.stack([y0, np.full(n, 0.3)], 1)
    lp = oracle.lstar_over_p(tgt, y, stddev=STDDEV, dt=DT)
    p = oracle.evaluate(tgt, y, L=1)["f"][:, 0] + 1e-8
    lstar = lp * p
    assert np.abs(lstar).mean() > 1.0
    assert abs(lstar.mean()) <= 1e-6 * np.abs(lstar).mean() + 1e-9


def _sup_lstar_over_p(oracle, tgt, dt):
    sigma = STDDEV / math.sqrt(DT)
    y0 = (np.arange(2000) + 0.5) / 2000
    y = np.stack([y0, np.full(y0.size, 0.7)], 1)
    return np.abs(oracle.lstar_over_p(tgt, y, stddev=sigma * math.sqrt(dt), dt=dt)).max()


def _sharp_lstar_over_p(y0, c1, c2, stddev, dt):
    """Closed form for the sharp step (score 0 on both sides): K* p is the
    step convolved with N(0, stddev^2) in x0 (images over the torus)."""
    kp = np.zeros_like(y0)
    for k in range(-2, 3):
        # mass of [k, k + 1/2) (value c1) and [k + 1/2, k + 1) (value c2) seen from y0
        za, zb, zc = (k - y0) / stddev, (k + 0.5 - y0) / stddev, (k + 1.0 - y0) / stddev
        kp += c1 * (_phi_cdf(zb) - _phi_cdf(za)) + c2 * (_phi_cdf(zc) - _phi_cdf(zb))
    p = np.where(y0 < 0.5, c1, c2)
    return (kp / p - 1.0) / dt


def test_lstar_over_p_is_order_dt_for_smooth_p_but_not_across_a_jump(oracle):
    tgt = oracle.target(_smooth_step(0.05))
    sups = [_sup_lstar_over_p(oracle, tgt, dt) for dt in (4e-5, 2e-5, 1e-5)]
    print("smooth step, sup |L*p/p| at dt = 4e-5, 2e-5, 1e-5:", np.round(sups, 4))
    for a, b in zip(sups, sups[1:]):
        assert 1.8 < a / b < 2.2
    sigma = STDDEV / math.sqrt(DT)
    u = np.linspace(0.05, 3.0, 60)      # distance below the jump at 1/2, in step lengths
    sharp = []
    for dt in (4e-5, 2e-5, 1e-5):
        sd = sigma * math.sqrt(dt)
        sharp.append(np.abs(_sharp_lstar_over_p(0.5 - u * sd, 1.0, 4.0, sd, dt)).max())
    print("sharp step, sup |L*p/p| near the jump at dt = 4e-5, 2e-5, 1e-5:", np.round(sharp, 1))
    for a, b in zip(sharp, sharp[1:]):
        assert 1.8 < b / a < 2.2
    # at the paper's dt the jump's term dwarfs the killing rate k0 / p itself
    k0 = 2.5 / (M_TOUR * DT)
    assert sharp[-1] > k0


def _half_mass(w, c1=1.0, c2=4.0, n=400000):
    x = (np.arange(n) + 0.5) / n
    if w == 0.0:
        g = np.where(x < 0.5, c1, c2)
    else:
        g = c2 + (c1 - c2) * 0.5 * (1.0 + np.tanh(np.sin(2 * np.pi * x) / (2 * np.pi) / w))
    return g[x < 0.5].sum() / g.sum(), g.mean()


def _restore_half_mass(oracle, w, stddev, dt, n_tours=400000, seeds=8):
    """Complete-tour Restore estimate of the mass of x0 in (0, 1/2) (the
    time in pixel 0 of the 2 x 1 grid over the total time), with its
    standard error over seeds, and the mean tour length in steps."""
    tgt = oracle.target(S.StepDensity(w=w))
    exact, p_lambda = _half_mass(w)
    prm = oracle.make_params(L=1, drift="exact", rb=True, stddev=stddev, dt=dt, k0=p_lambda / (M_TOUR * dt))
    ests, steps = [], []
    for b in range(seeds):
        r = oracle.restore_tours(tgt, prm, seed=1000 + b, chain_ids=np.arange(n_tours // seeds), image=True)
        acc = r["accum"][:, 0]
        ests.append(acc[0] / acc.sum())
        steps.append(r["steps"].mean())
        assert r["truncated"].sum() == 0
    return exact, float(np.mean(ests)), float(np.std(ests, ddof=1) / math.sqrt(seeds)), float(np.mean(steps))


def test_restore_bias_across_a_jump(oracle):
    sigma = STDDEV / math.sqrt(DT)
    rows = {}
    for w in (0.0, 0.0005, STDDEV, 0.05):
        rows[w] = _restore_half_mass(oracle, w, STDDEV, DT)
    for dt in (DT / 4, DT / 16):
        rows[("sharp", dt)] = _restore_half_mass(oracle, 0.0, sigma * math.sqrt(dt), dt)
    for k, (exact, est, se, steps) in rows.items():
        print(f"{k}: exact {exact:.4f}, Restore {est:.4f} +- {se:.4f} (bias {est - exact:+.4f}), "
              f"mean tour {steps:.2f} steps")
    exact, est, se, steps = rows[0.0]
    bias0 = est - exact
    # a jump: biased towards the uniform occupation 1/2, shorter tours
    assert bias0 > 10 * se and est < 0.5
    assert steps < 0.97 * (M_TOUR + 1)
    # O(sqrt(dt)) at fixed sigma: a quarter of dt halves the bias
    b4 = rows[("sharp", DT / 4)][1] - rows[("sharp", DT / 4)][0]
    b16 = rows[("sharp", DT / 16)][1] - rows[("sharp", DT / 16)][0]
    assert 0.35 < b4 / bias0 < 0.65 and 0.35 < b16 / b4 < 0.65
    # smoothing over less than a step leaves part of it; over a step length
    # and more it is gone (within 4 standard errors), and tours are m + 1
    # steps long again
    e, est_w, se_w, _ = rows[0.0005]
    assert 3 * se_w < est_w - e < bias0
    for w in (STDDEV, 0.05):
        e, est_w, se_w, steps_w = rows[w]
        assert abs(est_w - e) < 4 * se_w + 2e-4, (w, est_w, e)
        assert abs(steps_w - (M_TOUR + 1)) < 0.02 * (M_TOUR + 1)
