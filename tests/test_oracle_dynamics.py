"""Pins of the oracle's Restore / Langevin logic against closed forms.

P1  LocalDynamics (Alg. 4) on a Gaussian far from the torus edges is the
    linear map x' = A (x - c) + c + stddev xi with
    A = (1 - a / s^2) I - (gamma_tilde / s^2) J, a = stddev^2 / 2 and
    J (v1, v2) = (v2, -v1): one-step mean and covariance, and the stationary
    covariance of the discrete chain from the Lyapunov equation
    Sigma = A Sigma A^T + stddev^2 I (Sec. 5.1 Euler-Maruyama, Sec. 5.3).
P2  Constant target: the kill probability per step is
    k / (h + k) = p_lambda / (m p + p_lambda) = 1 / (m + 1) and Resolve
    (Alg. 3) returns the constant (Eq. killing-rate-constant).
P3  pi-invariance: on a 4-D Gaussian mixture the time average of g over the
    Restore process matches the target's moments (Sec. 4, Def. 1 with the
    modified killing rate; ergodic average of Sec. 3).
P3b The discretisation bias vanishes at rate O(dt) (Sec. 5.2: the
    continuous-time embedding of the Euler-Maruyama kernel with holding rate
    h = 1/dt is invariant up to O(dt)).  With the diffusion coefficient
    sigma = stddev / sqrt(dt) held at the paper's value, the relative error
    of the Restore estimate of a Gaussian's variance at least halves with
    each halving of dt (within 3 standard errors), so it is O(dt) and
    vanishes as dt -> 0; at the largest dt it is far above its error bar.
P6  Whole image: with the local moves switched off (stddev -> 0) every tour
    stays at its uniform start and the complete-tour Restore image (Alg. 3)
    is an unbiased estimate of lambda(f 1_pixel); on the 16 x 16 Cornell box
    it matches path tracing of the same f within 3 sigma per pixel.  This
    pins f, the pixel map, the clock, the holding-time weight and Resolve's
    k0 / tourCount normalisation on a real scene.  (With the paper's
    stddev = 5e-3 the Cornell image is biased low: the path contribution is
    discontinuous in primary sample space, which the regularity assumption
    of the paper's O(dt) bias analysis, Sec. 5.2, excludes.)
"""
import numpy as np
import pytest

from paper_2605_08916_gb300 import scenes as S


def test_local_dynamics_one_step_moments(oracle):
    O = oracle
    s = 0.05
    c = np.array([0.5, 0.5])
    x = np.array([0.52, 0.47])
    stddev, gt = 0.01, 5e-4
    score = -(x - c) / s ** 2
    n = 40000
    xs = np.stack([O.local_dynamics(x, score, stddev, gt, seed=123, frame=0, step=1, chain=j) for j in range(n)])
    a = 0.5 * stddev ** 2
    J = np.array([[0.0, 1.0], [-1.0, 0.0]])
    mean_exp = x + a * score + gt * (J @ score)
    se = stddev / np.sqrt(n)
    assert np.all(np.abs(xs.mean(0) - mean_exp) < 4 * se), (xs.mean(0), mean_exp)
    # the rotation term is 20 SE away from zero: a sign error fails
    assert abs(gt * (J @ score))[0] > 20 * se
    cov = np.cov((xs - mean_exp).T)
    assert np.allclose(cov, stddev ** 2 * np.eye(2), atol=4 * stddev ** 2 * np.sqrt(2.0 / n))


def test_local_dynamics_wrap_rule(oracle):
    """With stddev = 0 and gamma_tilde = 0 Alg. 4 only wraps x onto the torus
    (x - floor(x)).  A tiny negative coordinate gives 1 - 2^-60, which rounds
    to 1.0 in FP64 and must come back as 0 (the reading for results that
    round to 1); whole periods are removed in both directions."""
    x = np.array([-2.0 ** -60, 1.25, -0.25, 3.5, 0.0, 1.0 - 2.0 ** -53])
    out = oracle.local_dynamics(x, np.zeros_like(x), 0.0, 0.0, seed=1, frame=0, step=1, chain=0)
    assert out.tolist() == [0.0, 0.25, 0.75, 0.5, 0.0, 1.0 - 2.0 ** -53]


@pytest.mark.parametrize("gt_factor", [0.0, 1.0])
def test_stationary_covariance_closed_form(oracle, gt_factor):
    O = oracle
    # s = 0.1 keeps g above the density floor eps everywhere on the torus, so
    # the drift pulls every uniform start into the mode (with s = 0.05 the
    # far field has g < eps and chains random-walk there, as the method says)
    s = 0.1
    mix = S.single_gaussian([0.5, 0.5], s)
    tgt = O.target(mix)
    stddev = 0.04
    gt = gt_factor * 0.5 * stddev ** 2
    prm = O.make_params(L=1, drift="exact", rb=True, stddev=stddev, gamma_tilde=gt, k0=1e-12)
    M, T, burn = 2048, 400, 150
    r = O.restore_run(tgt, prm, seed=7, chain_ids=np.arange(M), n_steps=T, accum=False)
    assert r["tour_count"] == 0
    x = r["x"][burn:] - 0.5
    per_chain = np.einsum("tmi,tmj->mij", x, x) / x.shape[0]
    est = per_chain.mean(0)
    se = per_chain.std(0) / np.sqrt(M)
    a = 0.5 * stddev ** 2 / s ** 2
    b = gt / s ** 2
    var_exp = stddev ** 2 / (1.0 - (1.0 - a) ** 2 - b ** 2)
    for i in range(2):
        assert abs(est[i, i] - var_exp) < 3.5 * se[i, i], (est, var_exp, se)
    assert abs(est[0, 1]) < 3.5 * se[0, 1]
    # the discretisation is visible: the continuous-time variance s^2 is rejected
    assert abs(est[0, 0] - s ** 2) > 3 * se[0, 0]


@pytest.mark.parametrize("rb", [True, False])
def test_constant_target_kill_rate_and_resolve(oracle, rb):
    O = oracle
    c = 2.0
    mix = S.constant_target(d=4, value=c, width=4, height=4)
    tgt = O.target(mix)
    m, dt = 64.0, 1e-5
    k0 = c / (m * dt)
    prm = O.make_params(L=1, drift="exact", rb=rb, k0=k0, m=m, dt=dt)
    M, T = 4096, 200
    r = O.restore_run(tgt, prm, seed=11, chain_ids=np.arange(M), n_steps=T, record=False)
    n = M * (T + 1)
    p_kill = k0 / ((c + 1e-8) / dt + k0)
    assert abs(p_kill - 1.0 / (m + 1.0)) < 1e-6
    frac = r["tour_count"] / n
    assert abs(frac - p_kill) < 4 * np.sqrt(p_kill * (1 - p_kill) / n)
    img = O.resolve(r["accum"], k0, r["tour_count"])
    # each channel's image sums (over pixels) to lambda(f) = c
    tot = img.sum(0)
    assert np.allclose(tot, c, rtol=4 / np.sqrt(r["tour_count"])), tot
    # uniform target: every pixel gets c / (W H) up to noise
    assert np.allclose(img[:, 0], c / 16, rtol=0.1)


def _wrapped_moments_1d(mu, s, n=200001):
    """E[x], E[x^2] on [0,1) of the nearest-image Gaussian (normalised
    numerically), by quadrature."""
    x = (np.arange(n) + 0.5) / n
    dd = x - mu
    dd -= np.round(dd)
    w = np.exp(-0.5 * dd ** 2 / s ** 2)
    w /= w.sum()
    return (w * x).sum(), (w * x * x).sum()


def test_mixture_invariance_moments(oracle):
    O = oracle
    d, K = 4, 3
    rng = np.random.default_rng(5)
    w = rng.uniform(0.5, 1.5, K)
    w /= w.sum()
    mu = rng.uniform(0.3, 0.7, (K, d))
    sig = rng.uniform(0.10, 0.14, K)
    mix = S.Mixture(d, w, mu, sig, 8, 8)
    tgt = O.target(mix)
    # closed-form moments of the mixture (per coordinate quadrature, product form)
    m1 = np.zeros(d)
    m2 = np.zeros((d, d))
    for k in range(K):
        e1 = np.zeros(d)
        e2 = np.zeros(d)
        for i in range(d):
            e1[i], e2[i] = _wrapped_moments_1d(mu[k, i], sig[k])
        mk2 = np.outer(e1, e1)
        np.fill_diagonal(mk2, e2)
        m1 += w[k] * e1
        m2 += w[k] * mk2
    prm = O.make_params(L=1, drift="exact", rb=True, stddev=5e-3, m=64.0)
    # p_lambda = 1 (normalised mixture) -> k0 = p_lambda / (m dt)
    prm.k0 = 1.0 / (64.0 * 1e-5)
    # complete tours are i.i.d.; renewal-reward: pi(g) = E[int g] / E[int 1]
    M = 60000
    r = O.restore_tours(tgt, prm, seed=3, chain_ids=np.arange(M), max_steps=1 << 22)
    assert r["truncated"].sum() == 0
    # E[tour length] = p_lambda / k0 = m dt, i.e. m steps on average (Sec. 6)
    assert abs(r["steps"].mean() / 64.0 - 1.0) < 0.25
    A1, Ag, Agg = r["I1"], r["Ix"], r["Ixx"]
    est1 = Ag.sum(0) / A1.sum()
    est2 = Agg.sum(0) / A1.sum()
    # ratio-estimator standard errors across independent tours
    mA = A1.mean()
    se1 = np.sqrt(np.var(Ag - est1[None, :] * A1[:, None], axis=0) / M) / mA
    se2 = np.sqrt(np.var(Agg - est2[None] * A1[:, None, None], axis=0) / M) / mA
    z1 = np.abs(est1 - m1) / se1
    z2 = np.abs(est2 - m2) / se2
    assert z1.max() < 3.5, (est1, m1, z1)
    assert z2.max() < 3.5, (est2, m2, z2)
    # the check has power: the uniform distribution's moments are rejected
    assert np.max(np.abs(est2 - (np.full((d, d), 0.25) + np.eye(d) / 12.0)) / se2) > 10


def test_discretisation_bias_vanishes_linearly_in_dt(oracle):
    O = oracle
    s = 0.08
    tgt = O.target(S.single_gaussian([0.5, 0.5], s))
    _, var_true = _wrapped_moments_1d(0.5, s)
    var_true -= _wrapped_moments_1d(0.5, s)[0] ** 2
    sigma = 5e-3 / np.sqrt(1e-5)          # the paper's stddev and dt
    M = 1_000_000
    dts = 1.6e-3 / 2.0 ** np.arange(4)
    bias, se = [], []
    for dt in dts:
        prm = O.make_params(L=1, drift="exact", rb=True, stddev=sigma * np.sqrt(dt), dt=dt, m=64.0)
        prm.k0 = 1.0 / (64.0 * dt)         # p_lambda = 1 (normalised density)
        r = O.restore_tours(tgt, prm, seed=11, chain_ids=np.arange(M), max_steps=1 << 22)
        assert r["truncated"].sum() == 0
        A1, Ax, Axx = r["I1"], r["Ix"][:, 0], r["Ixx"][:, 0, 0]
        m1, m2 = Ax.sum() / A1.sum(), Axx.sum() / A1.sum()
        # delta method for the ratio estimators: the variance estimate's
        # influence per tour is (Axx - m2 A1) - 2 m1 (Ax - m1 A1)
        infl = (Axx - m2 * A1) - 2 * m1 * (Ax - m1 * A1)
        bias.append((m2 - m1 * m1) / var_true - 1.0)
        se.append(np.sqrt(np.var(infl) / M) / A1.mean() / var_true)
    b, e = np.array(bias), np.array(se)
    print("relative variance bias", b, "+-", e, "bias / dt", b / dts)
    assert b[0] > 20 * e[0]                        # the check has power
    for k in range(len(dts) - 1):                  # halving dt at least halves the bias
        assert b[k + 1] <= 0.5 * b[k] + 3 * np.sqrt(e[k + 1] ** 2 + 0.25 * e[k] ** 2), (k, b, e)
    assert b[-1] > -3 * e[-1]


def test_cornell_restore_image_matches_path_tracing(oracle):
    O = oracle
    scene = S.cornell_box(1, 16, 16)
    L = 4
    tgt = O.OracleScene(scene)
    xs = np.random.default_rng(11).random((20000, S.pss_dim(L)))
    p_hat = float(np.mean(np.exp(O.evaluate(tgt, xs, L)["logp"])))
    k0 = p_hat / (64 * 1e-5)
    prm = O.make_params(L=L, drift="exact", rb=True, k0=k0, stddev=1e-6)
    M, n_seeds = 4096, 12
    imgs = []
    for s in range(n_seeds):
        r = O.restore_tours(tgt, prm, seed=500 + s, chain_ids=np.arange(M), image=True)
        assert r["truncated"].sum() == 0
        imgs.append(O.resolve(r["accum"], k0, M))
    imgs = np.array(imgs)
    mean = imgs.mean(0)
    var = imgs.var(0, ddof=1) / n_seeds
    ref, ref_var = O.pt_image(tgt, L, 1 << 12, seed=3)
    z = (mean - ref) / np.sqrt(var + ref_var + 1e-300)
    print(f"image sum ratio {mean.sum() / ref.sum():.4f}, |z|<3: {np.mean(np.abs(z) < 3):.3f}, "
          f"mean z^2 {np.mean(z ** 2):.2f}")
    assert abs(mean.sum() / ref.sum() - 1.0) < 0.03
    assert np.mean(np.abs(z) < 3) >= 0.97
    assert np.mean(z ** 2) < 1.6


def test_default_parameters_are_the_papers(oracle):
    """The defaults of both sides are the parameters the paper prints
    (tests/golden/paper_parameters.json, cited there): stddev, dt, m and eps;
    gamma_tilde defaults to stddev^2 / 2 (the reading for the unspecified
    gamma).  The Metropolis entries of the file belong to comparison systems
    that are not built."""
    import json
    import os
    from paper_2605_08916_gb300 import renderer as R
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")) as f:
        g = json.load(f)
    po, pr = oracle.make_params(), R.make_params()
    for key in ("stddev", "dt", "m", "eps"):
        assert getattr(po, key) == g[key], key                        # FP64 fields
        assert getattr(pr, key) == np.float32(g[key]), key            # FP32 fields of the C ABI
    assert po.gamma_tilde == 0.5 * g["stddev"] ** 2
    assert pr.gamma_tilde == np.float32(0.5 * g["stddev"] ** 2)
