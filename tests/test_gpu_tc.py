"""GPU parity of the tcgen05 tensor-core batched pass (K >= 16 vectors, BF16 X).

The oracle runs on the same BF16-rounded X (promoted exactly to FP64) and the
same FP32 beta: |f - f_o|/|f_o| <= 1e-4 and ||g - g_o||/||g_o|| <= 1e-4.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import Handle, assert_close, rel_errors

pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _bf16_case(n, p, k, seed, spread=0.05):
    d = synth.make_glm(n, p, seed, dtype=np.float32)
    ld = synth.padded_ld(p, 2)
    Xs = synth.pad_columns(d.X, ld)
    q = oracle.bf16_from_f32(Xs)
    Xr = oracle.bf16_to_f64(q)
    rng = np.random.default_rng(seed + 1)
    B = (d.beta_star[None, :] + spread * rng.standard_normal((k, p))).astype(np.float32)
    return q, Xr, d.y, B, d


def _tc_handle(q, y, p, k):
    h = Handle(q, y, p, xtype=glm.GLM_X_BF16, k_max=k)
    info = h.info()
    assert info["tc_enabled"] == 1 and k >= info["tc_min_k"], info
    return h


@pytest.mark.parametrize("n,p,k", [
    (20011, 256, 64), (1, 8, 16), (127, 64, 16), (128, 100, 17), (129, 128, 32), (5000, 200, 33),
    (3000, 5, 64), (4097, 256, 65), (777, 256, 100), (256, 1, 16), (70000, 256, 64),
])
def test_tc_matches_oracle(n, p, k):
    q, Xr, y, B, _ = _bf16_case(n, p, k, 300 + n + p + k)
    h = _tc_handle(q, y, p, k)
    f, g = h.eval(B)
    f_o, g_o = oracle.logpost_grad(Xr, y, B.astype(np.float64), p=p)
    ef, eg = assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what=f"tc N={n} P={p} K={k}")
    print(f"tc N={n} P={p} K={k}: f {ef:.2e} g {eg:.2e}")


def test_tc_matches_cuda_core_path_and_is_deterministic():
    n, p, k = 30011, 256, 64
    q, Xr, y, B, _ = _bf16_case(n, p, k, 41)
    h = _tc_handle(q, y, p, k)
    f1, g1 = h.eval(B)
    f2, g2 = h.eval(B)
    np.testing.assert_array_equal(f1, f2)
    np.testing.assert_array_equal(g1, g2)
    hc = Handle(q, y, p, xtype=glm.GLM_X_BF16, k_max=k, flags=glm.GLM_FLAG_NO_TENSOR_CORES)
    fc, gc = hc.eval(B)
    assert_close(f1, g1, fc, gc, f_rtol=RTOL, g_rtol=RTOL, what="tc vs cuda cores")


def test_tc_large_eta_and_separated_rows():
    n, p, k = 9000, 64, 16
    q, Xr, y, B, _ = _bf16_case(n, p, k, 57)
    B[0, :] = 0.0
    B[1, 0] = 40.0
    B[2, :] *= 30.0
    h = _tc_handle(q, y, p, k)
    f, g = h.eval(B)
    assert np.isfinite(f).all() and np.isfinite(g).all()
    f_o, g_o = oracle.logpost_grad(Xr, y, B.astype(np.float64), p=p)
    assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what="tc large eta")


def test_tc_batched_workload_full_size_sampled():
    """N=1,000,000, P=256, K=64 chains, X BF16: every f and g against the
    oracle on the same rounded X for a sample of the 64 vectors."""
    n, p, k = 1_000_000, 256, 64
    q, Xr, y, B, d = _bf16_case(n, p, k, synth.seed_for(2))
    h = _tc_handle(q, y, p, k)
    f, g = h.eval(B)
    f2, g2 = h.eval(B)
    np.testing.assert_array_equal(f, f2)
    for kk in (0, 17, 40, 63):
        f_o, g_o = oracle.logpost_grad(Xr, y, B[kk].astype(np.float64), p=p)
        ef, eg = assert_close(f[kk:kk + 1], g[kk:kk + 1], f_o, g_o, f_rtol=RTOL, g_rtol=RTOL,
                              what=f"full size k={kk}")
        fu, gu = oracle.logpost_grad(d.X.astype(np.float64), y, B[kk].astype(np.float64))
        eu, gu_ = rel_errors(f[kk:kk + 1], g[kk:kk + 1], fu, gu)
        print(f"k={kk}: vs rounded X f {ef:.2e} g {eg:.2e}; vs FP32 X f {eu.max():.2e} "
              f"g {gu_.max():.2e}")


# ---- FP8 E4M3 storage: E4M3 tiles converted to FP16 on chip ------------------

def _fp8_case(n, p, k, seed, spread=0.05, wild_columns=False):
    d = synth.make_glm(n, p, seed, dtype=np.float32)
    X = d.X.copy()
    if wild_columns and p >= 5:
        X[:, 2] *= 1000.0          # large column scale
        X[:, 3] = 0.0              # all-zero column
        X[:, 4] *= 1e-3            # tiny column scale
    ld = synth.padded_ld(p, 1)
    Q, sc = oracle.quantize_e4m3(X, p, ld)
    Xr = oracle.dequantize_e4m3(Q, sc)
    rng = np.random.default_rng(seed + 1)
    B = (d.beta_star[None, :] + spread * rng.standard_normal((k, p))).astype(np.float32)
    return Q, sc, Xr, d.y, B, d


def _tc_fp8_handle(Q, sc, y, p, k):
    h = Handle(Q, y, p, xtype=glm.GLM_X_FP8E4M3, k_max=k, x_scale=sc)
    info = h.info()
    assert info["tc_enabled"] == 1 and k >= info["tc_min_k"], info
    return h


@pytest.mark.parametrize("n,p,k", [
    (20011, 256, 64), (1, 8, 16), (127, 64, 16), (128, 100, 17), (129, 128, 32), (5000, 200, 33),
    (3000, 5, 64), (4097, 256, 65), (777, 256, 100), (256, 1, 16), (70000, 256, 64),
])
def test_tc_fp8_matches_oracle(n, p, k):
    Q, sc, Xr, y, B, _ = _fp8_case(n, p, k, 500 + n + p + k)
    h = _tc_fp8_handle(Q, sc, y, p, k)
    f, g = h.eval(B)
    f_o, g_o = oracle.logpost_grad(Xr, y, B.astype(np.float64), p=p)
    ef, eg = assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what=f"tc fp8 N={n} P={p} K={k}")
    print(f"tc fp8 N={n} P={p} K={k}: f {ef:.2e} g {eg:.2e}")


def test_tc_fp8_wild_column_scales_and_extreme_coefficients():
    n, p, k = 9000, 64, 24
    Q, sc, Xr, y, B, _ = _fp8_case(n, p, k, 61, wild_columns=True)
    B[0, :] = 0.0
    B[1, 0] = 40.0
    B[2, :] *= 30.0
    B[3, :] *= 1e-6
    h = _tc_fp8_handle(Q, sc, y, p, k)
    f, g = h.eval(B)
    assert np.isfinite(f).all() and np.isfinite(g).all()
    f_o, g_o = oracle.logpost_grad(Xr, y, B.astype(np.float64), p=p)
    assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what="tc fp8 wild scales")


def test_tc_fp8_matches_cuda_core_path_and_is_deterministic():
    n, p, k = 30011, 200, 48
    Q, sc, Xr, y, B, _ = _fp8_case(n, p, k, 43)
    h = _tc_fp8_handle(Q, sc, y, p, k)
    f1, g1 = h.eval(B)
    f2, g2 = h.eval(B)
    np.testing.assert_array_equal(f1, f2)
    np.testing.assert_array_equal(g1, g2)
    hc = Handle(Q, y, p, xtype=glm.GLM_X_FP8E4M3, k_max=k, x_scale=sc,
                flags=glm.GLM_FLAG_NO_TENSOR_CORES)
    fc, gc = hc.eval(B)
    assert_close(f1, g1, fc, gc, f_rtol=RTOL, g_rtol=RTOL, what="tc fp8 vs cuda cores")


def test_tc_fp8_batched_workload_full_size_sampled():
    """N=1,000,000, P=256, K=64 chains, X FP8 E4M3 with column scales: f and
    g of a sample of the 64 vectors against the oracle on the same E4M3 X."""
    n, p, k = 1_000_000, 256, 64
    Q, sc, Xr, y, B, _ = _fp8_case(n, p, k, synth.seed_for(2))
    h = _tc_fp8_handle(Q, sc, y, p, k)
    f, g = h.eval(B)
    f2, _ = h.eval(B)
    np.testing.assert_array_equal(f, f2)
    for kk in (0, 21, 63):
        f_o, g_o = oracle.logpost_grad(Xr, y, B[kk].astype(np.float64), p=p)
        ef, eg = assert_close(f[kk:kk + 1], g[kk:kk + 1], f_o, g_o, f_rtol=RTOL, g_rtol=RTOL,
                              what=f"fp8 full size k={kk}")
        print(f"fp8 k={kk}: f {ef:.2e} g {eg:.2e}")


def test_tc_fp8_subnormal_codes():
    """Columns whose values sit far below their column maximum quantise to
    E4M3 subnormal codes (|q| < 2^-6); their FP16 images are exact and must
    enter both contractions unchanged."""
    n, p, k = 6000, 32, 16
    d = synth.make_glm(n, p, 71, dtype=np.float32)
    X = d.X.copy()
    rng = np.random.default_rng(72)
    for j in (3, 7, 11):
        X[:, j] = 3e-4 * rng.standard_normal(n)
        X[0, j] = 10.0
    ld = synth.padded_ld(p, 1)
    Q, sc = oracle.quantize_e4m3(X, p, ld)
    codes = Q[1:, [3, 7, 11]]
    subnormal = ((codes & 0x78) == 0) & ((codes & 0x07) != 0)
    assert subnormal.mean() > 0.5, subnormal.mean()
    Xr = oracle.dequantize_e4m3(Q, sc)
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    B[:, [3, 7, 11]] = 500.0 * rng.standard_normal((k, 3))   # make those columns matter
    h = _tc_fp8_handle(Q, sc, d.y, p, k)
    f, g = h.eval(B)
    f_o, g_o = oracle.logpost_grad(Xr, d.y, B.astype(np.float64), p=p)
    assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what="tc fp8 subnormal codes")
    # the subnormal columns of g on their own
    cols = [3, 7, 11]
    num = np.linalg.norm(g[:, cols] - g_o[:, cols], axis=1)
    den = np.linalg.norm(g_o[:, cols], axis=1)
    assert (num <= 1e-4 * den + 1e-6 * np.linalg.norm(g_o, axis=1)).all()
