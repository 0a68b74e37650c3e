"""Pins of the oracle's Hessian of the logistic log-posterior against finite
differences of the (separately pinned) gradient, the beta = 0 closed form,
symmetry and negative definiteness."""
import numpy as np

import oracle
import synth


def test_hessian_matches_finite_differences_of_the_gradient():
    d = synth.make_glm(400, 6, 31, dtype=np.float64)
    b = d.beta_star + 0.1
    _, g0, H = oracle.logpost_grad_hess(d.X, d.y, b)
    h = 1e-5
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        _, gp = oracle.logpost_grad(d.X, d.y, (b + e)[None, :])
        _, gm = oracle.logpost_grad(d.X, d.y, (b - e)[None, :])
        col = (gp[0] - gm[0]) / (2 * h)
        assert np.allclose(col, H[:, j], rtol=1e-6, atol=1e-6 * np.abs(H).max())


def test_hessian_at_zero_is_quarter_gram_matrix():
    """beta = 0: every mu = 1/2, so H = -X^T X / 4 - I / sigma^2."""
    d = synth.make_glm(300, 5, 32, dtype=np.float64)
    _, _, H = oracle.logpost_grad_hess(d.X, d.y, np.zeros(5), prior_sigma=3.0)
    want = -(d.X.T @ d.X) / 4.0 - np.eye(5) / 9.0
    assert np.allclose(H, want, rtol=1e-13, atol=1e-12)


def test_hessian_is_symmetric_negative_definite_and_consistent():
    d = synth.make_glm(500, 8, 33, dtype=np.float64)
    f, g, H = oracle.logpost_grad_hess(d.X, d.y, d.beta_star)
    assert np.array_equal(H, H.T) or np.allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).max() < 0
    f2, g2 = oracle.logpost_grad(d.X, d.y, d.beta_star[None, :])
    assert f == f2[0] and np.array_equal(g, g2[0])
