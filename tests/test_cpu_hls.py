"""The multi-core FP64 CPU baseline (oracle/cpu_hls.c: partial loop fusion,
cache fusion and one combine per thread, §3.4.1, §4.2.1, §4.2.2) against the
plain oracle. Only the summation order differs, so the two agree to FP64
rounding; the baseline's timing is only meaningful if it computes the same
f and g."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n,p,ld,k,threads", [
    (0, 3, 3, 1, 4),            # no rows: the prior alone
    (1, 1, 1, 1, 1),
    (127, 5, 8, 2, 3),          # one ragged chunk, more threads than chunks
    (1_001, 50, 52, 3, 8),      # ragged chunks and thread blocks, padded stride
    (20_000, 100, 100, 1, 5),
])
def test_hls_equals_oracle(n, p, ld, k, threads):
    d = synth.make_glm(max(n, 1), p, 900 + n + p, dtype=np.float64)
    X = synth.pad_columns(d.X[:n], ld) if n else np.zeros((0, ld))
    y = d.y[:n]
    rng = np.random.default_rng(n + k)
    B = d.beta_star[None, :] + 0.3 * rng.standard_normal((k, p))
    f_o, g_o = oracle.logpost_grad(X, y, B, p=p)
    f, g = oracle.hls_logpost_grad(X, y, B, p=p, threads=threads)
    np.testing.assert_allclose(f, f_o, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(g, g_o, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(g_o).max()))


def test_hls_thread_count_does_not_change_the_result_beyond_rounding():
    d = synth.make_glm(5_000, 20, 4, dtype=np.float64)
    res = [oracle.hls_logpost_grad(d.X, d.y, d.beta_star, threads=t) for t in (1, 2, 7)]
    for f, g in res[1:]:
        np.testing.assert_allclose(f, res[0][0], rtol=1e-13)
        np.testing.assert_allclose(g, res[0][1], rtol=1e-10, atol=1e-10)
    assert oracle.hls_max_threads() >= 1
