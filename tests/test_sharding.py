"""Row sharding across ranks (CPU, gloo): each rank evaluates its row block
(the oracle stands in for the GPU here), rank 0 keeps the prior, and the
package's one sum all-reduce gives the whole-data posterior and gradient."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_1310_1537_gb300 import GLM_FLAG_NO_PRIOR, GLM_FLAG_NO_TENSOR_CORES
from paper_1310_1537_gb300 import sharding


def test_shard_rows_cover_every_row_once():
    for n in (0, 1, 5, 7, 1000, 2_000_001):
        for world in (1, 2, 3, 8):
            blocks = [sharding.shard_rows(n, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
                assert a1 == b0 and a0 <= a1
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.shard_rows(10, 2, 2)


def test_shard_flags_keep_the_prior_on_rank_zero_only():
    assert sharding.shard_flags(0) == 0
    assert sharding.shard_flags(1) == GLM_FLAG_NO_PRIOR
    assert sharding.shard_flags(3, GLM_FLAG_NO_TENSOR_CORES) == (GLM_FLAG_NO_TENSOR_CORES |
                                                                  GLM_FLAG_NO_PRIOR)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d = synth.make_glm(3001, 13, 777, dtype=np.float32)
        X = d.X.astype(np.float64)
        rng = np.random.default_rng(5)
        B = d.beta_star[None, :] + 0.2 * rng.standard_normal((3, 13))
        r0, r1 = sharding.shard_rows(X.shape[0], world, rank)
        if sharding.shard_flags(rank) & GLM_FLAG_NO_PRIOR:
            f, g = oracle.loglik_partial(X, d.y, B, r0, r1)
        else:
            f, g = oracle.logpost_grad(X[r0:r1], d.y[r0:r1], B)
        ft = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float64))
        gt = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float64))
        sharding.allreduce_sum_(ft, gt)
        if rank == 0:
            f_o, g_o = oracle.logpost_grad(X, d.y, B)
            np.save(os.path.join(out_dir, "f.npy"), ft.numpy())
            np.save(os.path.join(out_dir, "g.npy"), gt.numpy())
            np.save(os.path.join(out_dir, "f_o.npy"), f_o)
            np.save(os.path.join(out_dir, "g_o.npy"), g_o)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sum_equals_whole_on_gloo_ranks(world, tmp_path):
    import torch.multiprocessing as mp
    oracle.build()
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    f = np.load(tmp_path / "f.npy")
    g = np.load(tmp_path / "g.npy")
    f_o = np.load(tmp_path / "f_o.npy")
    g_o = np.load(tmp_path / "g_o.npy")
    np.testing.assert_allclose(f, f_o, rtol=1e-12)
    np.testing.assert_allclose(g, g_o, rtol=1e-10, atol=1e-9)
