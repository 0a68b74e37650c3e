"""GPU parity of reduced-precision storage: the quantiser is bit-exact against
the oracle's quantisers, and evaluations on BF16 / FP8-stored X match the
oracle run on the same rounded X (<= 1e-4 on f and g)."""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import Handle, assert_close, rel_errors, to_dev, torch

pytestmark = pytest.mark.gpu

RTOL_LOWP = 1e-4


def _quantize_on_gpu(X32, p, xtype):
    t = torch()
    n = X32.shape[0]
    es = glm.ELEM_BYTES[xtype]
    ld = synth.padded_ld(p, es)
    h = glm.glm_create(n, p, ld, 1, xtype, 10.0, 0, 0)
    try:
        Xd = to_dev(X32)
        if xtype == glm.GLM_X_BF16:
            Xq = t.empty((n, ld), dtype=t.int16, device="cuda")
            glm.glm_quantize(h, Xd, X32.shape[1], Xq, None)
            sc = None
        else:
            Xq = t.empty((n, ld), dtype=t.uint8, device="cuda")
            sc = t.empty(p, dtype=t.float32, device="cuda")
            glm.glm_quantize(h, Xd, X32.shape[1], Xq, sc)
        assert glm.glm_sync(h) == glm.GLM_OK
        q = Xq.cpu().numpy()
        if xtype == glm.GLM_X_BF16:
            q = q.view(np.uint16)
        return q, (None if sc is None else sc.cpu().numpy())
    finally:
        glm.glm_destroy(h)


@pytest.mark.parametrize("n,p", [(1, 1), (1000, 7), (4097, 50), (30000, 256)])
def test_bf16_quantiser_bit_exact(n, p):
    d = synth.make_glm(n, p, 50 + p, dtype=np.float32)
    X = d.X.copy()
    X[0, -1] = 3.0e38 if p > 1 else X[0, -1]
    q, _ = _quantize_on_gpu(X, p, glm.GLM_X_BF16)
    ld = q.shape[1]
    ref = oracle.bf16_from_f32(X)
    np.testing.assert_array_equal(q[:, :p], ref)
    assert (q[:, p:ld] == 0).all()


@pytest.mark.parametrize("n,p", [(1, 1), (999, 5), (4097, 50), (30000, 256)])
def test_fp8_quantiser_bit_exact(n, p):
    d = synth.make_glm(n, p, 70 + p, dtype=np.float32)
    X = d.X.copy()
    if p >= 5:
        X[:, 2] *= 1000.0
        X[:, 3] = 0.0
        X[:, 4] *= 1e-3
    q, sc = _quantize_on_gpu(X, p, glm.GLM_X_FP8E4M3)
    Qo, so = oracle.quantize_e4m3(X, ld_q=q.shape[1])
    np.testing.assert_array_equal(sc, so)
    np.testing.assert_array_equal(q, Qo)


@pytest.mark.parametrize("xtype", [glm.GLM_X_BF16, glm.GLM_X_FP8E4M3])
@pytest.mark.parametrize("n,p,k", [(1, 3, 1), (1000, 50, 3), (20011, 256, 4), (5000, 100, 8),
                                   (3001, 513, 1)])
def test_lowp_eval_vs_oracle_on_rounded_x(xtype, n, p, k):
    d = synth.make_glm(n, p, 90 + n + p, dtype=np.float32)
    q, sc = _quantize_on_gpu(d.X, p, xtype)
    if xtype == glm.GLM_X_BF16:
        Xr = oracle.bf16_to_f64(q)
    else:
        Xr = oracle.dequantize_e4m3(q, sc, p=p)
        Xr = synth.pad_columns(Xr, q.shape[1])
    rng = np.random.default_rng(k + n)
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    h = Handle(q, d.y, p, xtype=xtype, k_max=k, x_scale=sc, flags=glm.GLM_FLAG_NO_TENSOR_CORES)
    f, g = h.eval(B)
    f_o, g_o = oracle.logpost_grad(Xr, d.y, B.astype(np.float64), p=p)
    assert_close(f, g, f_o, g_o, f_rtol=RTOL_LOWP, g_rtol=RTOL_LOWP, what=f"xtype={xtype}")
    # reported: error against the unrounded X
    fu, gu = oracle.logpost_grad(d.X.astype(np.float64), d.y, B.astype(np.float64))
    ef, eg = rel_errors(f, g, fu, gu)
    print(f"xtype {xtype} N={n} P={p}: vs unrounded X f {ef.max():.2e} g {eg.max():.2e}")
