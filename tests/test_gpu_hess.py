"""GPU parity of the one-pass log-posterior, gradient and Hessian (§4.2's
derivatives one order further, §5.2) against the FP64 oracle on the same FP32
X: |f - f_o| / |f_o| <= 1e-5, ||g - g_o|| / ||g_o|| <= 1e-4 and
||H - H_o||_F / ||H_o||_F <= 1e-4 (the contraction on the tensor cores from
BF16 hi/lo terms with FP32 accumulation over up to N / 152 rows per partial,
then a fixed-order FP32 sum of the partials). H is exactly symmetric and the
result bitwise reproducible."""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import to_dev, torch

pytestmark = pytest.mark.gpu


def _eval(Xs, y, beta, n, p, ld, sigma=10.0):
    t = torch()
    h = glm.glm_hess_create(n, p, ld, sigma)
    try:
        Xd = to_dev(Xs) if n > 0 else None
        yd = to_dev(y) if n > 0 else None
        bd = to_dev(np.asarray(beta, dtype=np.float32))
        f = t.empty(1, dtype=t.float64, device="cuda")
        g = t.empty(p, dtype=t.float32, device="cuda")
        H = t.empty((p, p), dtype=t.float32, device="cuda")
        glm.glm_hess_eval(h, Xd, yd, bd, f, g, H)
        assert glm.glm_hess_sync(h) == glm.GLM_OK
        return float(f.cpu().numpy()[0]), g.cpu().numpy(), H.cpu().numpy()
    finally:
        glm.glm_hess_destroy(h)


def _case(n, p, seed):
    d = synth.make_glm(max(n, 1), p, seed, dtype=np.float32)
    ld = (p + 3) // 4 * 4
    Xs = synth.pad_columns(d.X[:n], ld) if n > 0 else np.zeros((0, ld), np.float32)
    return d, Xs, ld


@pytest.mark.parametrize("n,p", [(0, 4), (1, 1), (63, 5), (64, 8), (65, 17), (1000, 33),
                                 (20011, 64), (100003, 50)])
def test_hessian_matches_oracle(n, p):
    d, Xs, ld = _case(n, p, 1200 + n + p)
    rng = np.random.default_rng(n + 7)
    beta = (d.beta_star + 0.1 * rng.standard_normal(p)).astype(np.float32)
    f, g, H = _eval(Xs, d.y[:n], beta, n, p, ld)
    fo, go, Ho = oracle.logpost_grad_hess(d.X[:n].astype(np.float64), d.y[:n], beta.astype(np.float64))
    assert abs(f - fo) <= 1e-5 * abs(fo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    assert np.linalg.norm(H - Ho) <= 1e-4 * np.linalg.norm(Ho)
    assert np.array_equal(H, H.T)


def test_hessian_is_deterministic_and_agrees_with_the_fused_pass():
    n, p = 50000, 40
    d, Xs, ld = _case(n, p, 1300)
    beta = d.beta_star.astype(np.float32)
    a = _eval(Xs, d.y, beta, n, p, ld)
    b = _eval(Xs, d.y, beta, n, p, ld)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    t = torch()
    hh = glm.glm_create(n, p, ld, 1, glm.GLM_X_F32, 10.0)
    try:
        f = t.empty(1, dtype=t.float64, device="cuda")
        g = t.empty((1, p), dtype=t.float32, device="cuda")
        glm.glm_logpost_grad(hh, to_dev(Xs), None, to_dev(d.y), to_dev(beta[None, :]), 1, f, g)
        assert glm.glm_sync(hh) == glm.GLM_OK
        assert abs(float(f.cpu()[0]) - a[0]) <= 1e-6 * abs(a[0])
        assert np.linalg.norm(g.cpu().numpy()[0] - a[1]) <= 1e-5 * np.linalg.norm(a[1])
    finally:
        glm.glm_destroy(hh)


def test_hessian_at_zero_and_extreme_coefficients():
    """beta = 0: H = -X^T X / 4 - I / s^2 exactly in the oracle; large |eta|
    (w -> 0) stays finite."""
    n, p = 4096, 16
    d, Xs, ld = _case(n, p, 1400)
    for beta in (np.zeros(p, np.float32), (40.0 * d.beta_star).astype(np.float32)):
        f, g, H = _eval(Xs, d.y, beta, n, p, ld, sigma=3.0)
        fo, go, Ho = oracle.logpost_grad_hess(d.X.astype(np.float64), d.y, beta.astype(np.float64),
                                              prior_sigma=3.0)
        assert np.isfinite(H).all() and np.isfinite(f)
        assert np.linalg.norm(H - Ho) <= 1e-4 * np.linalg.norm(Ho)
        assert abs(f - fo) <= 1e-5 * abs(fo)


def test_full_size_hessian_workload():
    """N = 2,000,000, P = 64 FP32 (the benchmark workload)."""
    n, p = 2_000_000, 64
    d = synth.make_glm(n, p, synth.seed_for(6), dtype=np.float32)
    beta = d.beta_star.astype(np.float32)
    f, g, H = _eval(d.X, d.y, beta, n, p, 64)
    fo, go, Ho = oracle.logpost_grad_hess(d.X.astype(np.float64), d.y, beta.astype(np.float64))
    assert abs(f - fo) <= 1e-5 * abs(fo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    assert np.linalg.norm(H - Ho) <= 1e-4 * np.linalg.norm(Ho)
