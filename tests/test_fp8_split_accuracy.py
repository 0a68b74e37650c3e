"""Accuracy of the FP8 tensor-core pass's operand splitting, checked on the CPU
against the FP64 oracle before any GPU run.

With X stored as FP8 E4M3 (4 significant bits) the tensor-core pass takes the
MMA operands in E4M3 as well, so the other operands are written as sums of
E4M3 terms:
- the coefficients v_j = s_j beta_kj as four terms, term t scaled by
  2^(e_k + 4t), where 2^e_k brings max_j |v_j| into [128, 256);
- the residual r = y - sigma(eta) as five terms in two blocks: v = 2^8 r
  rounded to FP16 and split exactly into three terms (scale 2^8), and the
  FP32 remainder v - fp16(v) rounded to FP16, scaled by 2^12 and split into
  two (scale 2^20): about 20 bits, which the near-cancelling sums g = X^t r
  near the mode need.
Products of E4M3 values are exact in FP32 and the MMAs accumulate in FP32.
This emulation follows those steps (NumPy; the FP32 sums use BLAS in another
order than the tensor cores, which is within FP32 rounding) and must meet the
tolerance of reduced-precision storage, 1e-4 on f and g, against the oracle
on the same E4M3 X (the precision contract, §3.3.1 roofline reasoning for
why the bytes of X matter). The N = 1e5 rows here are fewer than the
batched workload's 1e6, which makes the random part of the error larger,
not smaller.
"""
import numpy as np
import pytest

import oracle
import synth

RTOL = 1e-4


def e4m3_round(v):
    """Nearest OCP E4M3 value (ties to even), saturating at 448."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -10)))
    q = 2.0 ** (np.maximum(e, -6) - 3)          # normal: 3 fraction bits; subnormal: 2^-9
    r = np.minimum(np.round(a / q) * q, 448.0)
    return np.sign(v) * r


def coefficient_terms(B, sc, per_term=True):
    """The four E4M3 coefficient terms; term t is stored at scale 16^t
    (per_term=False: all four at the vector's one scale)."""
    v = B.astype(np.float64) * sc[None, :].astype(np.float64)
    m = np.abs(v).max(axis=1)
    ex = np.where(m > 0, np.floor(np.log2(np.where(m > 0, m, 1.0))) + 1, 0)
    e = np.where(m > 0, 8 - ex, 0)               # max |v 2^e| in [128, 256)
    rem = v * (2.0 ** e)[:, None]
    terms = []
    for t in range(4):
        st = 16.0 ** t if per_term else 1.0
        code = e4m3_round(rem * st)
        terms.append(code * (16.0 ** t / st))    # the stored E4M3 values, at scale 16^t
        rem = rem - code / st
    return terms, e


def _f16_terms(a, n):
    """Exact split of FP16 values into n E4M3 terms (differences in FP16)."""
    out = []
    for _ in range(n):
        t = e4m3_round(a.astype(np.float64))
        out.append(t)
        a = (a.astype(np.float64) - t).astype(np.float16)   # exact in FP16
    return out


def residual_terms(r):
    """Block A (scale 2^8): v = 2^8 r rounded to FP16, split into three terms;
    block B (scale 2^20): v - fp16(v), exact in FP32, rounded to FP16, scaled
    by 2^12 and split into two terms."""
    v = np.asarray(r, dtype=np.float32) * np.float32(256.0)
    a16 = v.astype(np.float16)
    d16 = (v - a16.astype(np.float32)).astype(np.float16) * np.float16(4096.0)   # exact scaling
    return _f16_terms(a16, 3), _f16_terms(d16, 2)


def emulate(Q, sc, y, B, per_term=True):
    """f and g as the FP8 tensor-core pass computes them."""
    qv = (oracle.dequantize_e4m3(Q, sc) / sc[None, :].astype(np.float64)).astype(np.float32)
    terms, e = coefficient_terms(B, sc, per_term)
    acc = [qv @ t.T.astype(np.float32) for t in terms]          # FP32 accumulation
    eta_s = acc[0] + (acc[1] + (acc[2] + acc[3] / 16) / 16) / 16
    eta = eta_s.astype(np.float64) * (2.0 ** -e)[None, :]
    yy = y.astype(np.float64)[:, None]
    ell = yy * eta - (np.maximum(eta, 0) + np.log1p(np.exp(-np.abs(eta))))
    with np.errstate(over="ignore"):
        r = yy - 1.0 / (1.0 + np.exp(-eta))
    ta, tb = residual_terms(r)
    ga = np.zeros(B.shape, dtype=np.float32)
    gb = np.zeros(B.shape, dtype=np.float32)
    for t in ta:
        ga += t.T.astype(np.float32) @ qv
    for t in tb:
        gb += t.T.astype(np.float32) @ qv
    P = B.shape[1]
    s2 = 100.0
    g = (ga.astype(np.float64) / 256.0 + gb.astype(np.float64) / 2.0 ** 20) * sc[None, :] - B / s2
    f = ell.sum(0) - (B.astype(np.float64) ** 2).sum(1) / (2 * s2) - 0.5 * P * np.log(2 * np.pi * s2)
    return f, g


def _check(Q, sc, y, B, p, what):
    f, g = emulate(Q, sc, y, B)
    f_o, g_o = oracle.logpost_grad(oracle.dequantize_e4m3(Q, sc), y, B.astype(np.float64), p=p)
    ef = np.abs(f - f_o) / np.abs(f_o)
    eg = np.linalg.norm(g - g_o, axis=1) / np.linalg.norm(g_o, axis=1)
    assert ef.max() <= RTOL and eg.max() <= RTOL, f"{what}: f {ef.max():.2e} g {eg.max():.2e}"
    return ef.max(), eg.max()


def test_e4m3_round_matches_the_oracle_encoder():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.uniform(-4, 2.6, 2000),
                        [0.0, 448.0, 464.0, -500.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -10]])
    want = np.array([oracle.e4m3_value(oracle.e4m3_from_f64(float(x))) for x in v])
    np.testing.assert_array_equal(e4m3_round(v), want)


def test_split_accuracy_at_the_batched_shape():
    """P = 256, K = 64 vectors ~ N(beta*, 0.05^2), X FP8 with column scales."""
    n, p, k = 100_000, 256, 64
    d = synth.make_glm(n, p, synth.seed_for(2), dtype=np.float32)
    rng = np.random.default_rng(synth.seed_for(2) + 1)
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    Q, sc = oracle.quantize_e4m3(d.X, p, p)
    ef, eg = _check(Q, sc, d.y, B, p, "batched shape")
    assert eg < 2e-5          # well inside the tolerance, not at its edge


def test_split_accuracy_with_subnormal_codes_and_wide_coefficient_range():
    """Columns quantised to E4M3 subnormal codes carrying coefficients 10^4
    times the others: per-term scaling keeps the small coefficients exact
    enough (a single scale for all four terms would not)."""
    n, p, k = 6000, 32, 16
    d = synth.make_glm(n, p, 71, dtype=np.float32)
    X = d.X.copy()
    rng = np.random.default_rng(72)
    for j in (3, 7, 11):
        X[:, j] = 3e-4 * rng.standard_normal(n)
        X[0, j] = 10.0
    Q, sc = oracle.quantize_e4m3(X, p, synth.padded_ld(p, 1))
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    B[:, [3, 7, 11]] = 500.0 * rng.standard_normal((k, 3))
    _check(Q, sc, d.y, B, p, "subnormal codes")


def test_split_accuracy_with_wild_column_scales_and_extreme_coefficients():
    n, p, k = 9000, 64, 24
    d = synth.make_glm(n, p, 61, dtype=np.float32)
    X = d.X.copy()
    X[:, 2] *= 1000.0
    X[:, 3] = 0.0
    X[:, 4] *= 1e-3
    Q, sc = oracle.quantize_e4m3(X, p, synth.padded_ld(p, 1))
    rng = np.random.default_rng(62)
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    B[0, :] = 0.0
    B[1, 0] = 40.0
    B[2, :] *= 30.0
    B[3, :] *= 1e-6
    _check(Q, sc, d.y, B, p, "wild scales")


@pytest.mark.parametrize("n,p,k", [(1, 8, 16), (127, 64, 16), (256, 1, 16), (3000, 5, 64),
                                   (20011, 256, 64)])
def test_split_accuracy_on_the_gpu_test_shapes(n, p, k):
    """The shapes of the GPU parity tests, including the intercept-only case
    where g is a sum that nearly cancels (a residual split of 16 bits misses
    the tolerance there)."""
    d = synth.make_glm(n, p, 500 + n + p + k, dtype=np.float32)
    Q, sc = oracle.quantize_e4m3(d.X, p, synth.padded_ld(p, 1))
    rng = np.random.default_rng(500 + n + p + k + 1)
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    _check(Q, sc, d.y, B, p, f"N={n} P={p} K={k}")


def test_a_single_scale_for_all_terms_would_fail():
    """The reading that needs per-term scales: with one scale 2^e_k for all
    four coefficient terms, the subnormal-code case misses the tolerance by
    orders of magnitude (planted on the CPU; the kernel never does this)."""
    n, p, k = 6000, 32, 16
    d = synth.make_glm(n, p, 71, dtype=np.float32)
    X = d.X.copy()
    rng = np.random.default_rng(72)
    for j in (3, 7, 11):
        X[:, j] = 3e-4 * rng.standard_normal(n)
        X[0, j] = 10.0
    Q, sc = oracle.quantize_e4m3(X, p, synth.padded_ld(p, 1))
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    B[:, [3, 7, 11]] = 500.0 * rng.standard_normal((k, 3))
    f_o, g_o = oracle.logpost_grad(oracle.dequantize_e4m3(Q, sc), d.y, B.astype(np.float64), p=p)
    _, g = emulate(Q, sc, d.y, B, per_term=False)
    eg = np.linalg.norm(g - g_o, axis=1) / np.linalg.norm(g_o, axis=1)
    assert eg.max() > 100 * RTOL
