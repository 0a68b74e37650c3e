"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or the mathematics
fixes: closed forms, an extended-precision brute force of the textbook
Bernoulli likelihood, central finite differences, symmetries, invariances,
library routines (scipy, numpy, torch dtype conversions) and quadrature.
They are chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _data(n, p, seed, intercept=True):
    d = synth.make_glm(n, p, seed, dtype=np.float64, intercept=intercept)
    return d.X, d.y, d.beta_star


# --- closed forms -----------------------------------------------------------

@pytest.mark.parametrize("n,p,sigma", [(1, 1, 10.0), (37, 5, 10.0), (1000, 50, 3.0)])
def test_beta_zero_closed_form(n, p, sigma):
    """f(0) = -N log 2 - (P/2) log(2 pi s^2);  g(0) = X^t (y - 1/2)."""
    X, y, _ = _data(n, p, 11 + n)
    f, g = oracle.logpost_grad(X, y, np.zeros(p), prior_sigma=sigma)
    f_exact = -n * math.log(2.0) - 0.5 * p * math.log(2.0 * math.pi * sigma * sigma)
    assert f[0] == pytest.approx(f_exact, rel=1e-13, abs=1e-12)
    g_exact = X.T @ (y.astype(np.float64) - 0.5)
    np.testing.assert_allclose(g[0], g_exact, rtol=1e-12, atol=1e-10)


def test_intercept_only_closed_form():
    """P = 1, x_n = 1: f(b) = n1 log s(b) + n0 log s(-b) + log N(b|0,s^2), g = n1 - N s(b) - b/s^2."""
    from scipy.special import expit, log_expit
    from scipy.stats import norm
    n = 333
    rng = np.random.default_rng(5)
    y = (rng.random(n) < 0.3).astype(np.uint8)
    X = np.ones((n, 1))
    n1 = int(y.sum())
    n0 = n - n1
    for b in (-3.0, -0.2, 0.0, 0.7, 4.5, 40.0, -40.0):
        f, g = oracle.logpost_grad(X, y, np.array([b]), prior_sigma=10.0)
        f_ref = n1 * log_expit(b) + n0 * log_expit(-b) + norm.logpdf(b, 0.0, 10.0)
        g_ref = n1 - n * expit(b) - b / 100.0
        assert f[0] == pytest.approx(f_ref, rel=1e-12, abs=1e-10)
        assert g[0, 0] == pytest.approx(g_ref, rel=1e-10, abs=1e-9)


def test_prior_only_equals_gaussian_logpdf():
    """With no rows the log-posterior is the N(0, s^2 I) log-density and g = -b/s^2."""
    from scipy.stats import multivariate_normal
    rng = np.random.default_rng(2)
    for p, sigma in ((1, 10.0), (7, 2.5), (50, 10.0)):
        b = rng.standard_normal(p) * 3
        X = np.zeros((0, p))
        y = np.zeros(0, dtype=np.uint8)
        f, g = oracle.logpost_grad(X, y, b, prior_sigma=sigma)
        ref = multivariate_normal(np.zeros(p), sigma * sigma * np.eye(p)).logpdf(b)
        assert f[0] == pytest.approx(ref, rel=1e-12)
        np.testing.assert_allclose(g[0], -b / sigma**2, rtol=1e-14)


# --- extended-precision brute force -----------------------------------------

def _mp_bernoulli_logpost(mp, X, y, b, sigma):
    """Textbook form: sum_n [y log p_n + (1-y) log(1-p_n)] + Gaussian log-density."""
    tot = mp.mpf(0)
    for n in range(X.shape[0]):
        eta = mp.fsum(mp.mpf(float(X[n, j])) * b[j] for j in range(X.shape[1]))
        pn = 1 / (1 + mp.exp(-eta))
        tot += mp.log(pn) if y[n] else mp.log(1 - pn)
    s2 = mp.mpf(sigma) ** 2
    P = X.shape[1]
    tot += -mp.fsum(bj * bj for bj in b) / (2 * s2) - mp.mpf(P) / 2 * mp.log(2 * mp.pi * s2)
    return tot


@pytest.mark.parametrize("n,p,seed", [(1, 1, 0), (9, 3, 1), (64, 8, 2), (40, 5, 3)])
def test_bruteforce_mpmath(n, p, seed):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    X, y, bs = _data(n, p, 100 + seed)
    rng = np.random.default_rng(seed)
    beta = bs + 0.7 * rng.standard_normal(p)
    f, g = oracle.logpost_grad(X, y, beta, prior_sigma=10.0)
    bm = [mp.mpf(float(v)) for v in beta]
    fref = _mp_bernoulli_logpost(mp, X, y, bm, 10.0)
    assert abs(f[0] - float(fref)) <= 1e-13 * max(1.0, abs(float(fref)))
    # gradient by high-precision numerical differentiation of the textbook form
    for j in range(p):
        def fj(t, j=j):
            bb = list(bm)
            bb[j] = t
            return _mp_bernoulli_logpost(mp, X, y, bb, 10.0)
        dref = mp.diff(fj, bm[j])
        assert abs(g[0, j] - float(dref)) <= 1e-11 * max(1.0, abs(float(dref)))


def test_central_finite_differences():
    X, y, bs = _data(500, 12, 7)
    beta = bs + 0.3
    f, g = oracle.logpost_grad(X, y, beta)
    for j in range(12):
        h = 1e-5 * max(1.0, abs(beta[j]))
        bp = beta.copy(); bp[j] += h
        bm = beta.copy(); bm[j] -= h
        fd = (oracle.logpost_grad(X, y, bp)[0][0] - oracle.logpost_grad(X, y, bm)[0][0]) / (2 * h)
        assert g[0, j] == pytest.approx(fd, rel=1e-6, abs=1e-5)


# --- symmetries and invariances ---------------------------------------------

def test_label_sign_symmetry():
    """f(b; y) = f(-b; 1-y) and g(b; y) = -g(-b; 1-y)."""
    X, y, bs = _data(300, 6, 8)
    beta = bs + 0.5
    f1, g1 = oracle.logpost_grad(X, y, beta)
    f2, g2 = oracle.logpost_grad(X, (1 - y).astype(np.uint8), -beta)
    assert f1[0] == pytest.approx(f2[0], rel=1e-13)
    np.testing.assert_allclose(g1[0], -g2[0], rtol=1e-11, atol=1e-11)


def test_row_permutation_and_duplication():
    X, y, bs = _data(200, 4, 9)
    beta = bs - 0.2
    s = 1e9  # flat prior isolates the likelihood
    f, g = oracle.logpost_grad(X, y, beta, prior_sigma=s)
    perm = np.random.default_rng(1).permutation(200)
    fp, gp = oracle.logpost_grad(X[perm], y[perm], beta, prior_sigma=s)
    assert fp[0] == pytest.approx(f[0], rel=1e-12)
    np.testing.assert_allclose(gp[0], g[0], rtol=1e-10, atol=1e-10)
    fl, gl = oracle.loglik_partial(X, y, beta, 0, 200)
    fd, gd = oracle.loglik_partial(np.vstack([X, X]), np.concatenate([y, y]), beta, 0, 400)
    assert fd[0] == pytest.approx(2 * fl[0], rel=1e-13)
    np.testing.assert_allclose(gd[0], 2 * gl[0], rtol=1e-12, atol=1e-12)


def test_row_shards_sum_to_whole():
    """The per-worker partial sums over any row split add up to the whole likelihood."""
    X, y, bs = _data(1001, 9, 10)
    beta = np.vstack([bs, bs + 0.1])
    f_all, g_all = oracle.loglik_partial(X, y, beta, 0, 1001)
    cuts = [0, 1, 250, 251, 700, 1001]
    fs = np.zeros(2)
    gs = np.zeros((2, 9))
    for a, b in zip(cuts[:-1], cuts[1:]):
        f, g = oracle.loglik_partial(X, y, beta, a, b)
        fs += f
        gs += g
    np.testing.assert_allclose(fs, f_all, rtol=1e-13)
    np.testing.assert_allclose(gs, g_all, rtol=1e-11, atol=1e-11)
    # and the prior is added once on top
    f_post, g_post = oracle.logpost_grad(X, y, beta, prior_sigma=10.0)
    from scipy.stats import norm
    prior = norm.logpdf(beta, 0, 10.0).sum(axis=1)
    np.testing.assert_allclose(f_post, f_all + prior, rtol=1e-13)
    np.testing.assert_allclose(g_post, g_all - beta / 100.0, rtol=1e-12, atol=1e-12)


def test_multi_beta_columns_independent():
    """Row k of the batched result equals the single-vector result at beta_k."""
    X, y, bs = _data(150, 5, 12)
    B = bs[None, :] + np.random.default_rng(3).standard_normal((4, 5))
    f, g = oracle.logpost_grad(X, y, B)
    for k in range(4):
        fk, gk = oracle.logpost_grad(X, y, B[k])
        assert f[k] == fk[0]
        np.testing.assert_array_equal(g[k], gk[0])


def test_padded_stride_ignored():
    X, y, bs = _data(64, 5, 13)
    Xp = synth.pad_columns(X, 8)
    Xp[:, 5:] = 123.0  # padding must not be read
    f1, g1 = oracle.logpost_grad(X, y, bs)
    f2, g2 = oracle.logpost_grad(Xp, y, bs, p=5)
    assert f1[0] == f2[0]
    np.testing.assert_array_equal(g1, g2)


def test_large_eta_stable():
    """|eta| = 1000: ell = -|eta| on a wrong label, 0 on a right one; residual in {0, +-1}."""
    X = np.ones((4, 1))
    y = np.array([1, 0, 1, 0], dtype=np.uint8)
    s = 1e9
    for b in (1000.0, -1000.0):
        f, g = oracle.loglik_partial(X, y, np.array([b]), 0, 4)
        assert np.isfinite(f[0]) and np.isfinite(g[0, 0])
        assert f[0] == pytest.approx(-2 * 1000.0, rel=1e-15)
        # residuals: y - s(b) = y - 1 or y - 0
        r = (y - (1.0 if b > 0 else 0.0)).sum()
        assert g[0, 0] == pytest.approx(r, abs=0)
    f, _ = oracle.logpost_grad(X, y, np.array([1000.0]), prior_sigma=s)
    assert np.isfinite(f[0])


def test_concavity():
    """The log-posterior is concave: second differences along any direction are <= 0."""
    X, y, bs = _data(400, 6, 14)
    rng = np.random.default_rng(4)
    for _ in range(10):
        b = bs + rng.standard_normal(6)
        d = rng.standard_normal(6)
        h = 0.05
        f0 = oracle.logpost_grad(X, y, b)[0][0]
        fp = oracle.logpost_grad(X, y, b + h * d)[0][0]
        fm = oracle.logpost_grad(X, y, b - h * d)[0][0]
        assert fp + fm - 2 * f0 <= 1e-9


# --- hierarchical (grouped) form --------------------------------------------

def test_grouped_equals_per_group_plus_prior():
    from scipy.stats import norm
    gd = synth.make_grouped(6, 4, 21, dtype=np.float64, sizes=np.array([20, 1, 0, 57, 3, 100]))
    f, g = oracle.logpost_grad_grouped(gd.X, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau)
    for m in range(6):
        a, b = gd.offsets[m], gd.offsets[m + 1]
        fl, gl = oracle.loglik_partial(gd.X, gd.y, gd.beta[m], a, b)
        prior = norm.logpdf(gd.beta[m], gd.mu, gd.tau).sum()
        assert f[m] == pytest.approx(fl[0] + prior, rel=1e-13, abs=1e-12)
        np.testing.assert_allclose(g[m], gl[0] - (gd.beta[m] - gd.mu) / gd.tau**2,
                                   rtol=1e-12, atol=1e-12)


def test_grouped_beta_zero_closed_form():
    """Each group at b_m = 0, mu = 0: f_m = -n_m log 2 + log N(0|0,tau^2 I); g_m = X_m^t (y_m - 1/2)."""
    gd = synth.make_grouped(5, 3, 22, dtype=np.float64, sizes=np.array([4, 9, 20, 1, 33]))
    zeros = np.zeros_like(gd.beta)
    f, g = oracle.logpost_grad_grouped(gd.X, gd.y, gd.offsets, zeros, np.zeros(3), 0.5)
    for m in range(5):
        a, b = gd.offsets[m], gd.offsets[m + 1]
        fe = -(b - a) * math.log(2) - 1.5 * math.log(2 * math.pi * 0.25)
        assert f[m] == pytest.approx(fe, rel=1e-13)
        np.testing.assert_allclose(g[m], gd.X[a:b].T @ (gd.y[a:b] - 0.5), rtol=1e-12, atol=1e-12)


# --- random-walk Metropolis consumer ----------------------------------------

def test_rwm_replay_and_decisions():
    X, y, bs = _data(300, 4, 30)
    z, lu = synth.rwm_streams(50, 2, 4, 31)
    b0 = np.vstack([bs, bs]).astype(np.float32)
    step = 0.05
    r1 = oracle.rwm(X, y, b0, z, lu, step)
    r2 = oracle.rwm(X, y, b0, z, lu, step)
    np.testing.assert_array_equal(r1["samples"], r2["samples"])
    np.testing.assert_array_equal(r1["accept"], r2["accept"])
    # every decision is log u < log alpha, and the state follows it
    assert np.array_equal(r1["accept"].astype(bool), lu < r1["log_alpha"])
    prev = b0.copy()
    for t in range(50):
        prop = (np.float32(step) * z[t] + prev).astype(np.float32)
        for k in range(2):
            exp_state = prop[k] if r1["accept"][t, k] else prev[k]
            # fmaf(step, z, b) is within one rounding of the two-rounding form
            np.testing.assert_allclose(r1["samples"][t, k], exp_state, rtol=2e-7, atol=1e-12)
        prev = r1["samples"][t].copy()
    # logpost trace equals an independent evaluation at the recorded states
    for t in (0, 17, 49):
        f, _ = oracle.logpost_grad(X, y, r1["samples"][t].astype(np.float64))
        np.testing.assert_allclose(r1["logpost"][t], f, rtol=1e-14)


def test_rwm_posterior_mean_matches_quadrature():
    """Intercept-only model: the chain mean agrees with the quadrature posterior mean."""
    from scipy import integrate
    from scipy.special import log_expit
    n = 40
    y = np.zeros(n, dtype=np.uint8)
    y[:12] = 1
    X = np.ones((n, 1))
    sigma = 10.0

    def logp(b):
        return 12 * log_expit(b) + 28 * log_expit(-b) - b * b / (2 * sigma**2)
    mode = math.log(12 / 28)
    Z = integrate.quad(lambda b: math.exp(logp(b) - logp(mode)), -10, 10, limit=200)[0]
    mean = integrate.quad(lambda b: b * math.exp(logp(b) - logp(mode)), -10, 10, limit=200)[0] / Z
    var = integrate.quad(lambda b: (b - mean) ** 2 * math.exp(logp(b) - logp(mode)),
                         -10, 10, limit=200)[0] / Z
    T = 40000
    z, lu = synth.rwm_streams(T, 1, 1, 77)
    res = oracle.rwm(X, y, np.array([[mode]], dtype=np.float32), z, lu, step=0.9, prior_sigma=sigma)
    s = res["samples"][2000:, 0, 0].astype(np.float64)
    # batch-means Monte Carlo standard error
    nb = 50
    bm = s[: len(s) // nb * nb].reshape(nb, -1).mean(axis=1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(s.mean() - mean) < 5 * se + 1e-3
    assert abs(s.var() - var) / var < 0.15
    assert 0.2 < res["accept"].mean() < 0.9
