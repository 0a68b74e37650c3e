"""The allocation-free entry point (glm_logpost_grad_noalloc) against the
handle entry point (glm_logpost_grad).

glm_logpost_grad_noalloc serves callers that cannot allocate device memory
while they evaluate (memory pools that own all device memory, real-time loops,
plugins whose host forbids allocation): it keeps its scratch in a fixed device
array inside the library. This file runs last so that a failure here does not
hide the results of the other tests; it also passes when run on its own.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("n,p,k", [(100_003, 100, 3), (5_000, 37, 11), (1, 1, 1)])
def test_noalloc_matches_handle_entry_point_twice(n, p, k):
    d = synth.make_glm(n, p, 4242 + n, dtype=np.float32)
    ld = synth.padded_ld(p, 4)
    Xs = synth.pad_columns(d.X, ld)
    rng = np.random.default_rng(p)
    B = (d.beta_star[None, :] + 0.2 * rng.standard_normal((k, p))).astype(np.float32)
    h = Handle(Xs, d.y, p, k_max=k)
    f_ref, g_ref = h.eval(B)
    for _ in range(2):                      # two calls in a row share the scratch
        f, g = _noalloc(h.X, None, h.y, n, p, ld, glm.GLM_X_F32, B)
        assert_close(f, g, f_ref, g_ref, what="noalloc vs handle")


def test_noalloc_bf16_matches_handle_entry_point():
    n, p, k = 30_000, 64, 2
    d = synth.make_glm(n, p, 77, dtype=np.float32)
    import oracle
    q = oracle.bf16_from_f32(d.X)
    B = np.stack([d.beta_star, -d.beta_star]).astype(np.float32)
    h = Handle(q, d.y, p, xtype=glm.GLM_X_BF16, k_max=k, flags=glm.GLM_FLAG_NO_TENSOR_CORES)
    f_ref, g_ref = h.eval(B)
    for _ in range(2):
        f, g = _noalloc(h.X, None, h.y, n, p, p, glm.GLM_X_BF16, B)
        assert_close(f, g, f_ref, g_ref, what="noalloc bf16")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    t = torch()
    x = t.zeros((4, 1028), dtype=t.float32, device="cuda")
    y = t.zeros(4, dtype=t.uint8, device="cuda")
    b = t.zeros((1, 1028), dtype=t.float32, device="cuda")
    f = t.zeros(1, dtype=t.float64, device="cuda")
    g = t.zeros((1, 1028), dtype=t.float32, device="cuda")
    with pytest.raises(glm.GLMError) as e:
        glm.glm_logpost_grad_noalloc(x, None, y, 4, 1025, 1028, glm.GLM_X_F32, 10.0, b, 1, f, g)
    assert e.value.status == glm.GLM_ERR_INVALID_ARG
