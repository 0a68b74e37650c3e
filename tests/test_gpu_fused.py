"""GPU parity of the fused single-pass kernel against the FP64 oracle.

Every case runs the CUDA path through the C ABI and compares f and g with the
oracle evaluated on the same stored X (FP32, or the BF16/FP8 values promoted
exactly) and the same FP32 beta: |f - f_o|/|f_o| <= 1e-5 and
||g - g_o||/||g_o|| <= 1e-4.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import Handle, assert_close, rel_errors, to_dev, torch

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_glm.json")


def _f32_case(n, p, seed, ld=None):
    d = synth.make_glm(n, p, seed, dtype=np.float32)
    ld = ld or synth.padded_ld(p, 4)
    return synth.pad_columns(d.X, ld), d.y, d.beta_star


def _oracle(Xs, y, beta, p, sigma=10.0):
    return oracle.logpost_grad(Xs.astype(np.float64), y, np.atleast_2d(beta).astype(np.float64),
                               prior_sigma=sigma, p=p)


def test_golden_tiny():
    gd = json.load(open(GOLDEN))
    n, p, k = gd["n"], gd["p"], gd["k"]
    X = np.array(gd["X"], dtype=np.float32).reshape(n, p)
    Xs = synth.pad_columns(X, synth.padded_ld(p, 4))
    y = np.array(gd["y"], dtype=np.uint8)
    beta = np.array(gd["beta"], dtype=np.float32).reshape(k, p)
    h = Handle(Xs, y, p, k_max=k)
    f, g = h.eval(beta)
    assert_close(f, g, np.array(gd["f"]), np.array(gd["g"]).reshape(k, p), what="golden")


def test_small_workload_100_points():
    """N=10,000, P=50, FP64 data stored FP32; 100 beta ~ N(beta*, 0.1^2)."""
    d = synth.make_glm(10_000, 50, synth.seed_for(0), dtype=np.float64)
    X32 = d.X.astype(np.float32)
    Xs = synth.pad_columns(X32, 52)
    B = synth.eval_points(d.beta_star, 100, 0.1, synth.seed_for(0) + 1).astype(np.float32)
    h = Handle(Xs, d.y, 50, k_max=100)
    f, g = h.eval(B)
    f_o, g_o = _oracle(Xs, d.y, B, 50)
    ef, eg = assert_close(f, g, f_o, g_o, what="small workload")
    # reported, not asserted: error against the unrounded FP64 data
    f64, g64 = oracle.logpost_grad(d.X, d.y, B.astype(np.float64))
    ef64, eg64 = rel_errors(f, g, f64, g64)
    print(f"small: vs same-rounded f {ef:.2e} g {eg:.2e}; vs FP64 X f {ef64.max():.2e} "
          f"g {eg64.max():.2e}")


SHAPES = [
    # (N, P, K)
    (0, 5, 1), (1, 1, 1), (1, 50, 3), (31, 3, 2), (32, 4, 1), (33, 5, 5), (127, 100, 1),
    (129, 100, 2), (255, 7, 8), (257, 64, 9), (1000, 50, 4), (4099, 31, 3), (20011, 100, 1),
    (5003, 256, 2), (3001, 513, 1), (777, 16, 16), (50000, 12, 1), (100003, 100, 8),
]


@pytest.mark.parametrize("n,p,k", SHAPES)
def test_shapes_f32(n, p, k):
    Xs, y, bs = _f32_case(n, p, 1000 + n + p)
    rng = np.random.default_rng(n + 7 * p + k)
    B = (bs[None, :] + 0.3 * rng.standard_normal((k, p))).astype(np.float32)
    h = Handle(Xs, y, p, k_max=k)
    f, g = h.eval(B)
    f_o, g_o = _oracle(Xs, y, B, p)
    assert_close(f, g, f_o, g_o, what=f"N={n} P={p} K={k}")


def test_wider_stride_than_needed():
    """ld well above P: padding columns are finite and must not leak into f or g."""
    Xs, y, bs = _f32_case(3000, 10, 5, ld=40)
    Xs[:, 10:] = 7.0
    h = Handle(Xs, y, 10, k_max=2)
    B = np.stack([bs, -bs]).astype(np.float32)
    f, g = h.eval(B)
    f_o, g_o = _oracle(Xs, y, B, 10)
    assert_close(f, g, f_o, g_o, what="wide stride")


def test_deterministic_and_batch_invariant():
    Xs, y, bs = _f32_case(60000, 50, 9)
    rng = np.random.default_rng(3)
    B = (bs[None, :] + 0.2 * rng.standard_normal((8, 50))).astype(np.float32)
    h = Handle(Xs, y, 50, k_max=8)
    f1, g1 = h.eval(B)
    f2, g2 = h.eval(B)
    np.testing.assert_array_equal(f1, f2)
    np.testing.assert_array_equal(g1, g2)
    for k in (0, 5):
        fk, gk = h.eval(B[k])
        assert_close(fk, gk, f1[k:k + 1], g1[k:k + 1], f_rtol=1e-12, g_rtol=1e-6, what="alone vs batch")


def test_large_eta_is_finite():
    n, p = 4096, 8
    Xs, y, _ = _f32_case(n, p, 11)
    B = np.array([[300.0] + [0.0] * 7, [-300.0] + [0.0] * 7, [0.0] * 7 + [120.0]], dtype=np.float32)
    h = Handle(Xs, y, p, k_max=3)
    f, g = h.eval(B)
    assert np.isfinite(f).all() and np.isfinite(g).all()
    f_o, g_o = _oracle(Xs, y, B, p)
    assert_close(f, g, f_o, g_o, what="large |eta|")


def test_beta_zero_closed_form_on_gpu():
    Xs, y, _ = _f32_case(30000, 20, 12)
    h = Handle(Xs, y, 20, k_max=1)
    f, g = h.eval(np.zeros(20, dtype=np.float32))
    f_exact = -30000 * math.log(2.0) - 10 * math.log(2 * math.pi * 100.0)
    assert abs(f[0] - f_exact) / abs(f_exact) <= 1e-6
    g_exact = Xs[:, :20].astype(np.float64).T @ (y - 0.5)
    assert np.linalg.norm(g[0] - g_exact) / np.linalg.norm(g_exact) <= 1e-5


def test_host_entry_point_matches_device_entry_point():
    Xs, y, bs = _f32_case(20000, 50, 13)
    B = np.stack([bs, bs * 0.5, bs - 0.1]).astype(np.float32)
    h = Handle(Xs, y, 50, k_max=3)
    f_dev, g_dev = h.eval(B)
    f_host = np.zeros(3, dtype=np.float64)
    g_host = np.zeros((3, 50), dtype=np.float32)
    glm.glm_logpost_grad_host(h.h, h.X, None, h.y, B, 3, f_host, g_host)
    np.testing.assert_array_equal(f_host, f_dev)
    np.testing.assert_array_equal(g_host, g_dev)


def test_argument_errors_launch_nothing():
    t = torch()
    Xs, y, bs = _f32_case(1000, 8, 14)
    h = Handle(Xs, y, 8, k_max=2)
    bd = to_dev(np.atleast_2d(bs).astype(np.float32))
    f = t.full((2,), 123.0, dtype=t.float64, device="cuda")
    g = t.full((2, 8), 5.0, dtype=t.float32, device="cuda")
    raw = t.zeros(Xs.size + 8, dtype=t.float32, device="cuda")
    cases = [
        dict(X=raw.data_ptr() + 4, K=1),                  # misaligned X
        dict(X=h.X, K=3),                                 # K > k_max
        dict(X=h.X, K=0),
        dict(X=h.X, K=1, x_scale=bd),                     # scales for FP32 X
    ]
    for c in cases:
        with pytest.raises(glm.GLMError) as e:
            glm.glm_logpost_grad(h.h, c["X"], c.get("x_scale"), h.y, bd, c["K"], f, g)
        assert e.value.status == glm.GLM_ERR_INVALID_ARG
    t.cuda.synchronize()
    assert (f == 123.0).all() and (g == 5.0).all()


def test_bounded_wait_reports_timeout_and_context_survives():
    Xs, y, bs = _f32_case(2000, 8, 15)
    h = Handle(Xs, y, 8, k_max=1)
    glm.glm_selftest_wait_timeout(h.h, 2000)
    assert glm.glm_sync(h.h) == glm.GLM_ERR_TIMEOUT
    assert glm.glm_sync(h.h) == glm.GLM_OK          # the status word was cleared
    f, g = h.eval(bs)                               # and the context still works
    f_o, g_o = _oracle(Xs, y, bs, 8)
    assert_close(f, g, f_o, g_o, what="after timeout")


def test_big_workload_full_size():
    """N=2,000,000, P=100, FP32 X, K=1 — the benchmark's launch configuration."""
    d = synth.make_glm(2_000_000, 100, synth.seed_for(1), dtype=np.float32)
    B = synth.eval_points(d.beta_star, 2, 0.1, synth.seed_for(1) + 1).astype(np.float32)
    h = Handle(d.X, d.y, 100, k_max=1)
    for k in range(2):
        f, g = h.eval(B[k])
        f_o, g_o = _oracle(d.X, d.y, B[k], 100)
        ef, eg = assert_close(f, g, f_o, g_o, what="big workload")
        print(f"big: f rel {ef:.2e} g rel {eg:.2e}")


@pytest.mark.parametrize("xtype", [glm.GLM_X_F32, glm.GLM_X_BF16, glm.GLM_X_FP8E4M3])
def test_every_row_width_configures_and_launches(xtype):
    """Row widths from 1 to 520 columns at the largest CUDA-core chunk
    (8 vectors; 4 for FP8): the configurator's tile, stage and split choice
    must fit the per-block shared-memory limit together with the kernel's
    static shared arrays, and the results must match the oracle on the same
    stored X (rounded by the oracle's own BF16 / E4M3 encoders)."""
    t = torch()
    es = glm.ELEM_BYTES[xtype]
    k = 4 if xtype == glm.GLM_X_FP8E4M3 else 8
    n = 300
    for p in list(range(1, 80)) + list(range(80, 521, 9)):
        d = synth.make_glm(n, p, 4000 + p, dtype=np.float32)
        ld = synth.padded_ld(p, es)
        Xs = synth.pad_columns(d.X, ld)
        xs = None
        if xtype == glm.GLM_X_F32:
            Xstore, Xr = Xs, Xs.astype(np.float64)
        elif xtype == glm.GLM_X_BF16:
            Xstore = oracle.bf16_from_f32(Xs)
            Xr = oracle.bf16_to_f64(Xstore)
        else:
            Xstore, sc = oracle.quantize_e4m3(d.X, p, ld)
            Xr = oracle.dequantize_e4m3(Xstore, sc)
            xs = sc
        h = Handle(Xstore, d.y, p, xtype=xtype, k_max=k, x_scale=xs,
                   flags=glm.GLM_FLAG_NO_TENSOR_CORES)
        try:
            rng = np.random.default_rng(p)
            # a spread well away from the mode, so that g is not a near-zero
            # difference of large sums (P = 1 is the intercept alone)
            B = (d.beta_star[None, :] + 0.5 * rng.standard_normal((k, p))).astype(np.float32)
            f, g = h.eval(B)
            f_o, g_o = oracle.logpost_grad(Xr, d.y, B.astype(np.float64), p=p)
            # FP32 storage meets the FP32 contract (f 1e-5); BF16 / FP8
            # storage meets 1e-4 against the oracle on the same rounded X
            f_rtol = 1e-5 if xtype == glm.GLM_X_F32 else 1e-4
            assert_close(f, g, f_o, g_o, f_rtol=f_rtol, g_rtol=1e-4,
                         what=f"xtype={xtype} P={p} ld={ld}")
        finally:
            h.close()
