"""Pins of the oracle's univariate slice sampler (Neal 2003, stepping out then
shrinkage) and its Gibbs sweeps over GLM coefficients (§3.4.4), against
closed forms, invariants and quadrature rather than against itself."""
import math

import numpy as np

import oracle
import synth


def _chain(logdens, x0, n, seed, w=1.0, m=4, s_max=30):
    lu, uni = synth.slice_streams(n, 1, s_max, seed)
    x = np.float32(x0)
    g = logdens(x)
    out = np.empty(n)
    for t in range(n):
        x, g, _, _, _ = oracle.slice_step(logdens, x, g, lu[t, 0], uni[t, 0], w, m, s_max)
        out[t] = x
    return out


def test_slice_step_samples_a_standard_normal():
    """A long chain on log N(0, 1): mean 0 and variance 1 within Monte-Carlo error."""
    s = _chain(lambda x: -0.5 * float(x) ** 2, 0.0, 20000, 11)
    nb = 40
    bm = s.reshape(nb, -1).mean(axis=1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(s.mean()) < 5 * se + 1e-3
    assert abs(s.var() - 1.0) < 0.06


def test_slice_step_interval_on_a_flat_density():
    """Constant log density: stepping out never stops early, so the interval is
    exactly [L0 - J w, R0 + K w] with L0 = x0 - w U, R0 = L0 + w, J = floor(m V),
    K = m - 1 - J (each operation rounded to FP32), and the first shrinkage
    proposal is accepted: x1 = L + U1 (R - L)."""
    f32 = np.float32
    rng = np.random.default_rng(3)
    for _ in range(200):
        x0 = f32(rng.normal())
        w = f32(rng.uniform(0.1, 3.0))
        m = int(rng.integers(1, 9))
        uni = rng.random(5).astype(np.float32)
        evals = []

        def flat(x):
            evals.append(x)
            return 0.0
        x1, g1, nsh, nev, moved = oracle.slice_step(flat, x0, 0.0, math.log(0.3), uni, w, m, 3)
        L0 = f32(x0 - f32(w * uni[0]))
        R0 = f32(L0 + w)
        J = int(math.floor(f32(f32(m) * uni[1])))
        K = m - 1 - J
        L = f32(L0 - f32(f32(J) * w))
        R = f32(R0 + f32(f32(K) * w))
        assert x1 == f32(L + f32(uni[2] * f32(R - L)))
        assert moved and nsh == 0 and nev == J + K + 1 and g1 == 0.0


def test_slice_step_stays_inside_a_hard_support():
    """Density zero outside [-1, 2]: accepted points stay inside, and a chain
    covers the support uniformly (mean 0.5, variance 9/12)."""
    def box(x):
        return 0.0 if -1.0 <= float(x) <= 2.0 else -1e300
    s = _chain(box, 0.3, 20000, 5, w=0.7, m=6)
    assert s.min() >= -1.0 and s.max() <= 2.0
    assert abs(s.mean() - 0.5) < 0.05
    assert abs(s.var() - 0.75) < 0.05


def test_slice_gibbs_records_the_plain_log_posterior():
    """After every coordinate update the recorded log-posterior equals the plain
    definition at the recorded state, and every update's level test holds."""
    d = synth.make_glm(300, 4, 21, dtype=np.float64)
    lu, uni = synth.slice_streams(3, 4, 30, 22)
    res = oracle.slice_gibbs(d.X, d.y, d.beta_star.astype(np.float32), lu, uni, w=0.5, m=4)
    beta = d.beta_star.astype(np.float32).copy()
    g_prev = res["f0"]
    for s in range(3):
        for k in range(4):
            beta[k] = res["xk"][s, k]
            f, _ = oracle.logpost_grad(d.X, d.y, beta.astype(np.float64))
            assert abs(res["gk"][s, k] - f[0]) <= 1e-9 * abs(f[0])
            assert g_prev + lu[s, k] < res["gk"][s, k]        # inside the slice
            g_prev = res["gk"][s, k]


def test_slice_gibbs_posterior_moments_match_quadrature():
    """Intercept-only model: Gibbs-slice chain mean and variance agree with the
    quadrature posterior."""
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
    S = 6000
    lu, uni = synth.slice_streams(S, 1, 30, 31)
    res = oracle.slice_gibbs(X, y, np.array([mode], dtype=np.float32), lu, uni, w=0.5, m=4,
                             prior_sigma=sigma)
    s = res["xk"][200:, 0].astype(np.float64)
    nb = 40
    bm = s[: len(s) // nb * nb].reshape(nb, -1).mean(axis=1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(s.mean() - mean) < 5 * se + 1e-3
    assert abs(s.var() - var) / var < 0.12


def test_slice_step_shrinks_toward_the_current_point():
    """Shrinkage keeps x0 inside the interval: each proposal lies between the
    closest rejected proposals on either side of x0 (and inside the initial
    interval), whatever the random numbers."""
    f32 = np.float32
    rng = np.random.default_rng(17)
    for trial in range(300):
        x0 = f32(rng.uniform(-0.2, 0.2))
        lo, hi = -0.25, 0.25                         # the slice: a narrow box
        pts = []

        def box(x):
            pts.append(float(x))
            return 0.0 if lo <= float(x) <= hi else -1e300
        uni = rng.random(2 + 20).astype(np.float32)
        w = f32(rng.uniform(2.0, 8.0))               # wide: several rejections
        x1, g1, nsh, nev, moved = oracle.slice_step(box, x0, 0.0, math.log(0.5), uni, w, 1, 20)
        L0 = f32(x0 - f32(w * uni[0]))
        R0 = f32(L0 + w)
        left, right = float(L0), float(R0)
        for x in pts:                                # m = 1: only shrinkage proposals
            assert left <= x <= right, (trial, x, left, right)
            if lo <= x <= hi:
                break
            if x < x0:
                left = x
            else:
                right = x
        assert moved and lo <= x1 <= hi
