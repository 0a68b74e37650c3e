"""GPU parity of the Gibbs-slice sampler with the differential update of X beta
(§3.4.4) against the FP64 oracle, which evaluates every point with the plain
log-posterior.

Evaluations: |f - f_o|/|f_o| <= 1e-5 on the same FP32 X and beta. Chains: the
device's coordinate values equal the oracle's until the first differing
decision, which must be a near tie (the slice level within 2e-5 |f| + 1e-6
of an evaluated log-posterior), and every device update replayed in the
oracle from the device's own state gives the same value except at near ties.
"""
import math

import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import to_dev, torch

pytestmark = pytest.mark.gpu


class Chain:
    """Device copies of one column-major dataset and a sampler for it."""

    def __init__(self, n, p, seed, w=0.5, m=4, s_max=30, spec=0):
        d = synth.make_glm(n, p, seed, dtype=np.float32)
        self.d, self.n, self.p = d, n, p
        self.ld = (n + 3) // 4 * 4
        Xt = np.zeros((p, self.ld), dtype=np.float32)
        Xt[:, :n] = d.X.T
        self.Xt_host = Xt
        self.X64 = d.X.astype(np.float64)
        self.Xt = to_dev(Xt)
        self.y = to_dev(d.y)
        self.w, self.m, self.s_max = w, m, s_max
        self.s = glm.glm_slice_create(n, p, self.ld, w=w, m=m, s_max=s_max, spec=spec)

    def close(self):
        glm.glm_slice_destroy(self.s)

    def eta_of(self, beta):
        t = torch()
        b = to_dev(np.asarray(beta, dtype=np.float32))
        eta = t.empty(self.n, dtype=t.float32, device="cuda")
        glm.glm_slice_eta(self.s, self.Xt, b, eta)
        assert glm.glm_slice_sync(self.s) == glm.GLM_OK
        return eta, b

    def f_oracle(self, beta):
        f, _ = oracle.logpost_grad(self.X64, self.d.y, np.asarray(beta, np.float64)[None, :])
        return float(f[0])

    def run(self, beta0, lu, uni, init=True, state=None):
        t = torch()
        S = lu.shape[0]
        if state is None:
            eta, b = self.eta_of(beta0)
            fs = t.zeros(1, dtype=t.float64, device="cuda")
        else:
            eta, b, fs = state
        xk = t.empty((S, self.p), dtype=t.float32, device="cuda")
        gk = t.empty((S, self.p), dtype=t.float64, device="cuda")
        ns = t.empty((S, self.p), dtype=t.int32, device="cuda")
        glm.glm_slice_run(self.s, self.Xt, self.y, eta, b, fs, 1 if init else 0, S, to_dev(lu),
                          to_dev(uni), xk, gk, ns)
        assert glm.glm_slice_sync(self.s) == glm.GLM_OK
        return (xk.cpu().numpy(), gk.cpu().numpy(), ns.cpu().numpy(), b.cpu().numpy(),
                fs.cpu().numpy()[0], eta, (eta, b, fs))


def test_eta_and_coordinate_evaluations_match_oracle():
    c = Chain(20011, 7, 601)
    try:
        rng = np.random.default_rng(602)
        beta = (c.d.beta_star + 0.3 * rng.standard_normal(7)).astype(np.float32)
        eta, b = c.eta_of(beta)
        eta_ref = c.X64 @ beta.astype(np.float64)
        assert np.max(np.abs(eta.cpu().numpy() - eta_ref)) <= 1e-5 * (1 + np.abs(eta_ref).max())
        t = torch()
        for k in (0, 3, 6):
            xs = (beta[k] + np.linspace(-2.0, 2.0, 16)).astype(np.float32)
            f = t.empty(16, dtype=t.float64, device="cuda")
            glm.glm_slice_coord_logpost(c.s, c.Xt, c.y, eta, b, k, to_dev(xs), 16, f)
            assert glm.glm_slice_sync(c.s) == glm.GLM_OK
            f = f.cpu().numpy()
            for j in range(16):
                bj = beta.copy()
                bj[k] = xs[j]
                fo = c.f_oracle(bj)
                assert abs(f[j] - fo) <= 1e-5 * abs(fo), (k, j, f[j], fo)
    finally:
        c.close()


def _replay(c, beta_before, k, x_dev, lu, un):
    """Oracle update of coordinate k from the device's state; returns the
    oracle's value and the smallest gap between the slice level and an
    evaluated log-posterior (near-tie measure)."""
    gaps = []
    g0 = c.f_oracle(beta_before)
    log_y = g0 + lu

    def dens(x):
        b = beta_before.copy()
        b[k] = x
        g = c.f_oracle(b)
        gaps.append(abs(g - log_y))
        return g
    x1, g1, _, _, _ = oracle.slice_step(dens, beta_before[k], g0, lu, un, c.w, c.m, c.s_max)
    return x1, g1, (min(gaps) if gaps else math.inf), abs(g0)


@pytest.mark.parametrize("n,p,sweeps", [(3000, 5, 6), (20011, 8, 3), (131, 3, 10)])
def test_slice_chain_matches_oracle(n, p, sweeps):
    c = Chain(n, p, 700 + n + p)
    try:
        lu, uni = synth.slice_streams(sweeps, p, c.s_max, 701 + n)
        beta0 = c.d.beta_star.astype(np.float32)
        xk, gk, ns, beta_end, f_end, eta, _ = c.run(beta0, lu, uni)
        ref = oracle.slice_gibbs(c.X64, c.d.y, beta0, lu, uni, c.w, c.m)
        # identical until the first differing decision, which must be a near tie
        same = xk == ref["xk"]
        flat = same.reshape(-1)
        first = int(np.argmin(flat)) if not flat.all() else flat.size
        # per-update replay from the device's own state
        beta = beta0.copy()
        near_ties = 0
        for u in range(sweeps * p):
            s_, k = divmod(u, p)
            x1, g1, gap, fabs = _replay(c, beta, k, xk[s_, k], lu[s_, k], uni[s_, k])
            tie = gap < 2e-5 * fabs + 1e-6
            if x1 != xk[s_, k]:
                assert tie, (u, x1, xk[s_, k], gap)
                near_ties += 1
            else:
                assert abs(gk[s_, k] - g1) <= 1e-5 * abs(g1), (u, gk[s_, k], g1)
            if u == first and first < flat.size:
                assert tie, (u, gap)
            beta[k] = xk[s_, k]
        assert np.array_equal(beta, beta_end)
        assert abs(f_end - c.f_oracle(beta_end)) <= 1e-5 * abs(f_end)
        # eta kept by differential updates still equals X beta
        eta_ref = c.X64 @ beta_end.astype(np.float64)
        assert np.max(np.abs(eta.cpu().numpy() - eta_ref)) <= 1e-4 * (1 + np.abs(eta_ref).max())
        print(f"N={n} P={p}: {sweeps * p} updates, identical prefix {first}, near ties {near_ties}")
    finally:
        c.close()


def test_slice_run_is_deterministic_and_resumable():
    c = Chain(5000, 6, 801)
    try:
        lu, uni = synth.slice_streams(6, 6, c.s_max, 802)
        beta0 = c.d.beta_star.astype(np.float32)
        a = c.run(beta0, lu, uni)
        b = c.run(beta0, lu, uni)
        for x, y in zip(a[:5], b[:5]):
            np.testing.assert_array_equal(x, y)
        # 2 sweeps, then 4 more from the device state, equals 6 in one run
        first = c.run(beta0, lu[:2], uni[:2])
        second = c.run(None, lu[2:], uni[2:], init=False, state=first[6])
        np.testing.assert_array_equal(np.concatenate([first[0], second[0]]), a[0])
        np.testing.assert_array_equal(np.concatenate([first[1], second[1]]), a[1])
        np.testing.assert_array_equal(second[3], a[3])
    finally:
        c.close()


@pytest.mark.parametrize("m", [1, 4, 9])
def test_speculative_shrinkage_equals_one_proposal_per_pass(m):
    """Evaluating several shrinkage proposals per pass is exact: every spec
    gives bitwise the same chain as spec = 1 (one proposal per pass), with
    wide intervals (many shrinkage steps) and s_max small enough to be hit."""
    n, p, sweeps, s_max = 7001, 5, 4, 6
    lu, uni = synth.slice_streams(sweeps, p, s_max, 950 + m)
    out = {}
    for spec in (1, 2, 3, 7, 16):
        c = Chain(n, p, 951, w=2.0, m=m, s_max=s_max, spec=spec)
        try:
            r = c.run(c.d.beta_star.astype(np.float32), lu, uni)
            out[spec] = r[:5] + (r[5].cpu().numpy(),)
        finally:
            c.close()
    for spec in (2, 3, 7, 16):
        for a, b in zip(out[1], out[spec]):
            np.testing.assert_array_equal(a, b)
    assert (out[1][2] == s_max).any() or out[1][2].max() >= 3


def test_slice_full_size_big_workload():
    """N=2,000,000, P=100 column-major FP32: one sweep; the final state's
    log-posterior and eta against the oracle, and a sample of updates
    replayed from the device state."""
    n, p = 2_000_000, 100
    c = Chain(n, p, synth.seed_for(1))
    try:
        lu, uni = synth.slice_streams(1, p, c.s_max, synth.seed_for(1) + 5)
        beta0 = c.d.beta_star.astype(np.float32)
        xk, gk, ns, beta_end, f_end, eta, _ = c.run(beta0, lu, uni)
        assert abs(f_end - c.f_oracle(beta_end)) <= 1e-5 * abs(f_end)
        eta_ref = c.X64 @ beta_end.astype(np.float64)
        assert np.max(np.abs(eta.cpu().numpy() - eta_ref)) <= 1e-4 * (1 + np.abs(eta_ref).max())
        beta = beta0.copy()
        for k in range(p):
            if k in (0, 1, 50, 99):
                x1, g1, gap, fabs = _replay(c, beta, k, xk[0, k], lu[0, k], uni[0, k])
                if x1 != xk[0, k]:
                    assert gap < 2e-5 * fabs + 1e-6
            beta[k] = xk[0, k]
        print(f"big: mean shrink steps {ns.mean():.2f}, f {f_end:.3f}")
    finally:
        c.close()


def test_slice_argument_errors_and_size_limit():
    with pytest.raises(glm.GLMError) as e:
        glm.glm_slice_create(10_000_000, 10, 10_000_000)
    assert e.value.status == glm.GLM_ERR_UNSUPPORTED
    c = Chain(1000, 4, 901)
    try:
        t = torch()
        eta, b = c.eta_of(c.d.beta_star.astype(np.float32))
        f = t.empty(16, dtype=t.float64, device="cuda")
        xs = to_dev(np.zeros(17, np.float32))
        for k, M in [(-1, 1), (4, 1), (0, 0), (0, 17)]:
            with pytest.raises(glm.GLMError):
                glm.glm_slice_coord_logpost(c.s, c.Xt, c.y, eta, b, k, xs, M, f)
    finally:
        c.close()
