"""Row shards evaluated through the library on one GPU, one after another
(one handle per shard; rank 0's keeps the prior, the others are created with
GLM_FLAG_NO_PRIOR): their sum equals the whole-data evaluation and the
oracle, on the CUDA-core path (FP32) and the tensor-core path (BF16)."""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from paper_1310_1537_gb300 import sharding
from tests.glmgpu import assert_close, to_dev, torch

pytestmark = pytest.mark.gpu


def _eval(h, X, y, B, p):
    t = torch()
    k = B.shape[0]
    f = t.empty(k, dtype=t.float64, device="cuda")
    g = t.empty((k, p), dtype=t.float32, device="cuda")
    glm.glm_logpost_grad(h, X, None, y, to_dev(B), k, f, g)
    assert glm.glm_sync(h) == glm.GLM_OK
    return f.cpu().numpy(), g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("xtype,n,p,k,world", [
    (glm.GLM_X_F32, 100_003, 100, 3, 2),
    (glm.GLM_X_F32, 50_000, 37, 8, 3),
    (glm.GLM_X_BF16, 200_001, 256, 32, 4),
])
def test_shards_sum_to_the_whole(xtype, n, p, k, world):
    es = glm.ELEM_BYTES[xtype]
    d = synth.make_glm(n, p, 880 + n + p, dtype=np.float32)
    ld = synth.padded_ld(p, es)
    Xs = synth.pad_columns(d.X, ld)
    if xtype == glm.GLM_X_BF16:
        Xstore = oracle.bf16_from_f32(Xs)
        Xr = oracle.bf16_to_f64(Xstore)
    else:
        Xstore, Xr = Xs, Xs.astype(np.float64)
    rng = np.random.default_rng(n)
    B = (d.beta_star[None, :] + 0.1 * rng.standard_normal((k, p))).astype(np.float32)
    Xd, yd = to_dev(Xstore), to_dev(d.y)
    f_sum = np.zeros(k)
    g_sum = np.zeros((k, p))
    for rank in range(world):
        r0, r1 = sharding.shard_rows(n, world, rank)
        h = glm.glm_create(r1 - r0, p, ld, k, xtype, 10.0, 0, sharding.shard_flags(rank))
        try:
            if rank > 0:
                with pytest.raises(glm.GLMError):   # no Metropolis on a prior-less shard
                    glm.glm_rwm_run(h, Xd[r0:r1], None, yd[r0:r1], 1, 0, 0.0, None, None,
                                    to_dev(B[:1]), to_dev(np.zeros(1)), 1, None, None, None)
            f, g = _eval(h, Xd[r0:r1], yd[r0:r1], B, p)
        finally:
            glm.glm_destroy(h)
        f_sum += f
        g_sum += g
    h = glm.glm_create(n, p, ld, k, xtype, 10.0, 0, 0)
    try:
        f_w, g_w = _eval(h, Xd, yd, B, p)
    finally:
        glm.glm_destroy(h)
    f_o, g_o = oracle.logpost_grad(Xr, d.y, B.astype(np.float64), p=p)
    rt = 1e-5 if xtype == glm.GLM_X_F32 else 1e-4
    assert_close(f_sum, g_sum, f_o, g_o, f_rtol=rt, g_rtol=1e-4, what="shards vs oracle")
    assert_close(f_sum, g_sum, f_w, g_w, f_rtol=rt, g_rtol=1e-4, what="shards vs whole")
