"""The allocation-free entry point (glm_logpost_grad_noalloc) against the
handle entry point (glm_logpost_grad) and the FP64 oracle.

glm_logpost_grad_noalloc serves callers that cannot allocate device memory
while they evaluate (memory pools that own all device memory, real-time loops,
plugins whose host forbids allocation): it keeps its scratch in a fixed device
array inside the library. It runs the same CUDA-core kernel with the same
launch configuration as a handle made with GLM_FLAG_NO_TENSOR_CORES, and the
cross-CTA sums are order-independent integer fixed-point, so its results must
equal the handle's bit for bit; both must also meet the oracle's tolerances.

This file runs last so that a failure here does not hide the results of the
other tests; it also passes when run on its own.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import Handle, assert_close, to_dev, torch

pytestmark = pytest.mark.gpu


def _noalloc(Xd, sc, yd, n, p, ld, xtype, B):
    t = torch()
    k = B.shape[0]
    bd = to_dev(B)
    f = t.full((k,), float("nan"), dtype=t.float64, device="cuda")
    g = t.full((k, p), float("nan"), dtype=t.float32, device="cuda")
    glm.glm_logpost_grad_noalloc(Xd, sc, yd, n, p, ld, xtype, 10.0, bd, k, f, g)
    t.cuda.synchronize()
    return f.cpu().numpy(), g.cpu().numpy()


def _bitwise(f, g, f_ref, g_ref, what):
    assert np.array_equal(f.view(np.uint64), f_ref.view(np.uint64)), what
    assert np.array_equal(g.view(np.uint32), g_ref.view(np.uint32)), what


@pytest.mark.parametrize("n,p,k", [(100_003, 100, 3), (5_000, 37, 11), (1, 1, 1)])
def test_noalloc_matches_handle_entry_point_twice(n, p, k):
    d = synth.make_glm(n, p, 4242 + n, dtype=np.float32)
    ld = synth.padded_ld(p, 4)
    Xs = synth.pad_columns(d.X, ld)
    rng = np.random.default_rng(p)
    B = (d.beta_star[None, :] + 0.2 * rng.standard_normal((k, p))).astype(np.float32)
    h = Handle(Xs, d.y, p, k_max=k, flags=glm.GLM_FLAG_NO_TENSOR_CORES)
    f_ref, g_ref = h.eval(B)
    f_o, g_o = oracle.logpost_grad(Xs.astype(np.float64), d.y, B.astype(np.float64), p=p)
    for _ in range(2):                      # two calls in a row share the scratch
        f, g = _noalloc(h.X, None, h.y, n, p, ld, glm.GLM_X_F32, B)
        _bitwise(f, g, f_ref, g_ref, "noalloc vs handle (FP32)")
        assert_close(f, g, f_o, g_o, what="noalloc vs oracle (FP32)")


def test_noalloc_bf16_matches_handle_entry_point():
    n, p, k = 30_000, 64, 2
    d = synth.make_glm(n, p, 77, dtype=np.float32)
    q = oracle.bf16_from_f32(d.X)
    B = np.stack([d.beta_star, -d.beta_star]).astype(np.float32)
    h = Handle(q, d.y, p, xtype=glm.GLM_X_BF16, k_max=k, flags=glm.GLM_FLAG_NO_TENSOR_CORES)
    f_ref, g_ref = h.eval(B)
    f_o, g_o = oracle.logpost_grad(oracle.bf16_to_f64(q), d.y, B.astype(np.float64), p=p)
    for _ in range(2):
        f, g = _noalloc(h.X, None, h.y, n, p, p, glm.GLM_X_BF16, B)
        _bitwise(f, g, f_ref, g_ref, "noalloc vs handle (BF16)")
        assert_close(f, g, f_o, g_o, f_rtol=1e-4, g_rtol=1e-4, what="noalloc vs oracle (BF16)")


def test_noalloc_fp8_with_scales_and_several_launches():
    """FP8 E4M3 storage: column scales applied in the last CTA, and K = 11
    vectors in launches of at most 4 (the FP8 chunk) through one scratch."""
    n, p, k = 40_001, 70, 11
    d = synth.make_glm(n, p, 91, dtype=np.float32)
    ld = synth.padded_ld(p, 1)
    Xq, sc = oracle.quantize_e4m3(d.X, p, ld)
    rng = np.random.default_rng(5)
    B = (d.beta_star[None, :] + 0.3 * rng.standard_normal((k, p))).astype(np.float32)
    h = Handle(Xq, d.y, p, xtype=glm.GLM_X_FP8E4M3, k_max=k, x_scale=sc,
               flags=glm.GLM_FLAG_NO_TENSOR_CORES)
    f_ref, g_ref = h.eval(B)
    f_o, g_o = oracle.logpost_grad(oracle.dequantize_e4m3(Xq, sc), d.y, B.astype(np.float64), p=p)
    for _ in range(2):
        f, g = _noalloc(h.X, h.x_scale, h.y, n, p, ld, glm.GLM_X_FP8E4M3, B)
        _bitwise(f, g, f_ref, g_ref, "noalloc vs handle (FP8)")
        assert_close(f, g, f_o, g_o, f_rtol=1e-4, g_rtol=1e-4, what="noalloc vs oracle (FP8)")


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_arguments():
    t = torch()
    x = t.zeros((4, 1028), dtype=t.float32, device="cuda")
    y = t.zeros(4, dtype=t.uint8, device="cuda")
    b = t.zeros((1, 1028), dtype=t.float32, device="cuda")
    f = t.full((1,), 7.0, dtype=t.float64, device="cuda")
    g = t.full((1, 1028), 7.0, dtype=t.float32, device="cuda")
    cases = [
        # P beyond the fixed scratch
        (dict(p=1025, ld=1028), glm.GLM_ERR_INVALID_ARG),
        # rows wider than 1 MiB (ld * 4 bytes), as glm_create refuses
        (dict(p=8, ld=(1 << 18) + 4), glm.GLM_ERR_UNSUPPORTED),
        # a non-finite prior scale
        (dict(p=8, ld=8, sigma=float("inf")), glm.GLM_ERR_INVALID_ARG),
        # a misaligned gradient pointer
        (dict(p=8, ld=8, g=g.data_ptr() + 2), glm.GLM_ERR_INVALID_ARG),
        # a misaligned coefficient pointer
        (dict(p=8, ld=8, b=b.data_ptr() + 1), glm.GLM_ERR_INVALID_ARG),
    ]
    for c, want in cases:
        with pytest.raises(glm.GLMError) as e:
            glm.glm_logpost_grad_noalloc(x, None, y, 4, c["p"], c["ld"], glm.GLM_X_F32,
                                         c.get("sigma", 10.0), c.get("b", b), 1, f,
                                         c.get("g", g))
        assert e.value.status == want, c
    t.cuda.synchronize()
    assert (f == 7.0).all() and (g == 7.0).all()     # nothing was launched
