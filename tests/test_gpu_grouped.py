"""GPU parity of the grouped (hierarchical-Bayes) pass against the FP64 oracle.

Per group: |f - f_o|/|f_o| <= 1e-5 and ||g - g_o||/||g_o|| <= 1e-4 (FP32 X),
1e-4 on both for BF16/FP8-stored X against the oracle on the same rounded X.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import assert_close, to_dev, torch

pytestmark = pytest.mark.gpu


def _run_grouped(Xs, y, off, beta, mu, tau, p, xtype=glm.GLM_X_F32, x_scale=None, repeat=1,
                 n_rows=None, shape=None):
    t = torch()
    n, ld = Xs.shape
    G = len(off) - 1
    h = glm.glm_create(n if n_rows is None else n_rows, p, ld, 1, xtype, 10.0, 0, 0, G)
    try:
        if shape is not None:
            glm.glm_grouped_set_shape(h, *shape)
            assert glm.glm_grouped_get_shape(h) == tuple(shape)
        Xd = to_dev(Xs) if n > 0 else t.empty(16, dtype=t.uint8, device="cuda")
        yd = to_dev(y) if n > 0 else t.empty(16, dtype=t.uint8, device="cuda")
        od = to_dev(np.asarray(off, dtype=np.int64))
        bd = to_dev(np.asarray(beta, dtype=np.float32))
        md = to_dev(np.asarray(mu, dtype=np.float32))
        sd = None if x_scale is None else to_dev(np.asarray(x_scale, dtype=np.float32))
        outs = []
        for _ in range(repeat):
            f = t.full((G,), 7.0, dtype=t.float64, device="cuda")
            g = t.full((G, p), 7.0, dtype=t.float32, device="cuda")
            glm.glm_logpost_grad_grouped(h, Xd, sd, yd, od, G, bd, md, tau, f, g)
            assert glm.glm_sync(h) == glm.GLM_OK
            outs.append((f.cpu().numpy(), g.cpu().numpy()))
        return outs
    finally:
        glm.glm_destroy(h)


def _oracle_grouped(Xr, y, off, beta, mu, tau, p):
    return oracle.logpost_grad_grouped(Xr[:, :p] if Xr.shape[1] != p else Xr, y, off,
                                       np.asarray(beta, np.float64), np.asarray(mu, np.float64),
                                       tau)


@pytest.mark.parametrize("sizes", [
    [20, 0, 1, 57, 3000, 33, 0, 0, 512, 31, 32, 64, 1, 2, 4000],
    [0, 0, 0, 5],
    [1] * 300,
    [12345],
])
def test_grouped_small_cases(sizes):
    gd = synth.make_grouped(len(sizes), 32, 31 + len(sizes), dtype=np.float32,
                            sizes=np.array(sizes))
    (f, g), = _run_grouped(gd.X, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau, 32)
    f_o, g_o = _oracle_grouped(gd.X.astype(np.float64), gd.y, gd.offsets,
                               gd.beta.astype(np.float32), gd.mu.astype(np.float32), gd.tau, 32)
    assert_close(f, g, f_o, g_o, what=f"grouped {len(sizes)}")


def test_grouped_hb_workload_full_size():
    """G=4,000 groups, sizes log-normal (median 400, [20, 50,000]), P=32, FP32 X."""
    gd = synth.make_grouped(4000, 32, synth.seed_for(3), dtype=np.float32)
    outs = _run_grouped(gd.X, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau, 32, repeat=2)
    (f, g), (f2, g2) = outs
    np.testing.assert_array_equal(f, f2)       # deterministic
    np.testing.assert_array_equal(g, g2)
    f_o, g_o = _oracle_grouped(gd.X.astype(np.float64), gd.y, gd.offsets,
                               gd.beta.astype(np.float32), gd.mu.astype(np.float32), gd.tau, 32)
    ef, eg = assert_close(f, g, f_o, g_o, what="hb workload")
    print(f"hb: rows {gd.offsets[-1]}, max rel err f {ef:.2e} g {eg:.2e}")


def test_grouped_offsets_not_starting_at_zero_and_padded_stride():
    sizes = np.array([40, 0, 333, 7])
    gd = synth.make_grouped(4, 20, 99, dtype=np.float32, sizes=sizes)
    lead = 50
    X = np.vstack([np.full((lead, 20), 9.0, np.float32), gd.X])
    y = np.concatenate([np.ones(lead, np.uint8), gd.y])
    Xs = synth.pad_columns(X, 24)
    off = gd.offsets + lead
    (f, g), = _run_grouped(Xs, y, off, gd.beta, gd.mu, gd.tau, 20)
    f_o, g_o = oracle.logpost_grad_grouped(Xs.astype(np.float64), y, off,
                                           gd.beta.astype(np.float32).astype(np.float64),
                                           gd.mu.astype(np.float32).astype(np.float64), gd.tau)
    assert_close(f, g, f_o, g_o, what="offset start")


@pytest.mark.parametrize("xtype", [glm.GLM_X_BF16, glm.GLM_X_FP8E4M3])
def test_grouped_lowp(xtype):
    sizes = np.array([20, 400, 1, 0, 2500, 64, 130])
    p = 64
    gd = synth.make_grouped(len(sizes), p, 7, dtype=np.float32, sizes=sizes)
    if xtype == glm.GLM_X_BF16:
        q = oracle.bf16_from_f32(gd.X)
        Xr = oracle.bf16_to_f64(q)
        sc = None
    else:
        q, sc = oracle.quantize_e4m3(gd.X, ld_q=p)
        Xr = oracle.dequantize_e4m3(q, sc)
    (f, g), = _run_grouped(q, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau, p, xtype=xtype, x_scale=sc)
    f_o, g_o = _oracle_grouped(Xr, gd.y, gd.offsets, gd.beta.astype(np.float32),
                               gd.mu.astype(np.float32), gd.tau, p)
    assert_close(f, g, f_o, g_o, f_rtol=1e-4, g_rtol=1e-4, what=f"grouped xtype {xtype}")


def test_grouped_malformed_offsets_give_nan_not_a_fault():
    gd = synth.make_grouped(3, 8, 5, dtype=np.float32, sizes=np.array([10, 10, 10]))
    bad = np.array([0, 20, 10, 30], dtype=np.int64)           # decreasing
    (f, g), = _run_grouped(gd.X, gd.y, bad, gd.beta, gd.mu, gd.tau, 8)
    assert np.isnan(f).all() and np.isnan(g).all()
    beyond = np.array([0, 10, 20, 31], dtype=np.int64)         # past N = 30
    (f, g), = _run_grouped(gd.X, gd.y, beyond, gd.beta, gd.mu, gd.tau, 8)
    assert np.isnan(f).all()


def test_grouped_rejects_too_many_groups():
    t = torch()
    h = glm.glm_create(100, 8, 8, 1, glm.GLM_X_F32, 10.0, 0, 0, 2)
    try:
        X = t.zeros((100, 8), device="cuda")
        y = t.zeros(100, dtype=t.uint8, device="cuda")
        off = t.tensor([0, 10, 20, 100], dtype=t.int64, device="cuda")
        b = t.zeros((3, 8), device="cuda")
        mu = t.zeros(8, device="cuda")
        f = t.zeros(3, dtype=t.float64, device="cuda")
        g = t.zeros((3, 8), device="cuda")
        with pytest.raises(glm.GLMError) as e:
            glm.glm_logpost_grad_grouped(h, X, None, y, off, 3, b, mu, 0.5, f, g)
        assert e.value.status == glm.GLM_ERR_INVALID_ARG
    finally:
        glm.glm_destroy(h)


def test_grouped_launch_is_graph_capturable():
    """The grouped call allocates nothing and does not synchronise: it can be
    captured in a CUDA graph and replayed with bitwise-identical results."""
    t = torch()
    gd = synth.make_grouped(200, 32, 17, dtype=np.float32)
    G = 200
    h = glm.glm_create(gd.X.shape[0], 32, 32, 1, glm.GLM_X_F32, 10.0, 0, 0, G)
    try:
        Xd, yd = to_dev(gd.X), to_dev(gd.y)
        od = to_dev(gd.offsets)
        bd = to_dev(gd.beta.astype(np.float32))
        md = to_dev(gd.mu.astype(np.float32))
        f = t.zeros(G, dtype=t.float64, device="cuda")
        g = t.zeros((G, 32), dtype=t.float32, device="cuda")
        s = t.cuda.Stream()
        with t.cuda.stream(s):
            glm.glm_logpost_grad_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g, s)
        s.synchronize()
        f_eager, g_eager = f.cpu().numpy(), g.cpu().numpy()
        graph = t.cuda.CUDAGraph()
        with t.cuda.graph(graph, stream=s):
            glm.glm_logpost_grad_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g, s)
        for _ in range(3):
            f.zero_()
            graph.replay()
        t.cuda.synchronize()
        np.testing.assert_array_equal(f.cpu().numpy(), f_eager)
        np.testing.assert_array_equal(g.cpu().numpy(), g_eager)
    finally:
        glm.glm_destroy(h)


def test_grouped_autotuner_keeps_results_correct():
    """The autotuner times launch shapes on the real inputs; whatever it picks
    must give results within tolerance and stay deterministic."""
    t = torch()
    gd = synth.make_grouped(600, 32, 23, dtype=np.float32)
    G = 600
    h = glm.glm_create(gd.X.shape[0], 32, 32, 1, glm.GLM_X_F32, 10.0, 0, 0, G)
    try:
        Xd, yd, od = to_dev(gd.X), to_dev(gd.y), to_dev(gd.offsets)
        bd = to_dev(gd.beta.astype(np.float32))
        md = to_dev(gd.mu.astype(np.float32))
        f = t.zeros(G, dtype=t.float64, device="cuda")
        g = t.zeros((G, 32), dtype=t.float32, device="cuda")
        glm.glm_autotune_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g, 2)
        f.zero_()
        glm.glm_logpost_grad_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g)
        assert glm.glm_sync(h) == glm.GLM_OK
        f1, g1 = f.cpu().numpy(), g.cpu().numpy()
        glm.glm_logpost_grad_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g)
        assert glm.glm_sync(h) == glm.GLM_OK
        np.testing.assert_array_equal(f.cpu().numpy(), f1)
        f_o, g_o = _oracle_grouped(gd.X.astype(np.float64), gd.y, gd.offsets,
                                   gd.beta.astype(np.float32), gd.mu.astype(np.float32), gd.tau, 32)
        assert_close(f1, g1, f_o, g_o, what="autotuned grouped")
    finally:
        glm.glm_destroy(h)


def _shape_smem(shape, p, ld, elem_bytes=4):
    """Dynamic shared memory of a grouped launch shape (the library's sizing:
    each warp's ring of slots, its barriers, and the coefficient slice or the
    narrow kernel's transpose buffer)."""
    variant, warps, units, stages, _ = shape
    epc = 16 // elem_bytes
    pcue = -(-p // epc) * epc
    ring = -(-(stages * units * 32 * ld * elem_bytes) // 128) * 128
    extra = 64 + warps * 32 * 17 * 4 if variant else warps * pcue * 4
    return warps * ring + warps * stages * 8 + extra + 64


def _shape_fits(shape, p, ld):
    ctas = shape[4]
    return _shape_smem(shape, p, ld) <= 232448 // ctas - (1024 if ctas > 1 else 0)


@pytest.mark.parametrize("shape", [(0, 4, 1, 2, 1), (0, 16, 1, 3, 1), (0, 8, 1, 3, 2),
                                   (1, 4, 1, 2, 1), (1, 12, 2, 2, 1), (1, 4, 4, 2, 1),
                                   (1, 4, 2, 2, 2)])
def test_grouped_both_kernel_variants(shape):
    """The warp-stream kernel (variant 0) and the narrow-row kernel (variant
    1), set explicitly through glm_grouped_set_shape, on ragged, empty and
    single-row groups and several row widths: P = 8 and 20 (rows of 2 and 5
    chunks), 32 (the 128-byte-row instance) and 100 (variant 1 does not apply
    and is refused; a shape whose rings do not fit in shared memory is
    refused as unsupported)."""
    sizes = np.array([20, 0, 1, 57, 3000, 33, 0, 512, 31, 32, 64, 1, 2, 4000, 777])
    for p in (8, 20, 32, 100):
        gd = synth.make_grouped(len(sizes), p, 3 + p, dtype=np.float32, sizes=sizes)
        ld = synth.padded_ld(p, 4)
        Xs = synth.pad_columns(gd.X, ld)
        if shape[0] == 1 and p > 32:
            with pytest.raises(glm.GLMError) as e:
                _run_grouped(Xs, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau, p, shape=shape)
            assert e.value.status == glm.GLM_ERR_INVALID_ARG
            continue
        if not _shape_fits(shape, p, ld):
            with pytest.raises(glm.GLMError) as e:
                _run_grouped(Xs, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau, p, shape=shape)
            assert e.value.status == glm.GLM_ERR_UNSUPPORTED
            continue
        outs = _run_grouped(Xs, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau, p, shape=shape,
                            repeat=2)
        np.testing.assert_array_equal(outs[0][0], outs[1][0])
        np.testing.assert_array_equal(outs[0][1], outs[1][1])
        f_o, g_o = _oracle_grouped(Xs.astype(np.float64), gd.y, gd.offsets,
                                   gd.beta.astype(np.float32), gd.mu.astype(np.float32), gd.tau, p)
        assert_close(outs[0][0], outs[0][1], f_o, g_o, what=f"shape {shape} P={p}")


def test_grouped_shape_setter_rejects_bad_shapes():
    gd = synth.make_grouped(3, 32, 5, dtype=np.float32, sizes=np.array([10, 10, 10]))
    h = glm.glm_create(gd.X.shape[0], 32, 32, 1, glm.GLM_X_F32, 10.0, 0, 0, 3)
    try:
        before = glm.glm_grouped_get_shape(h)
        for bad in [(2, 8, 1, 2, 1), (0, 5, 1, 2, 1), (0, 20, 1, 2, 1), (1, 16, 1, 2, 1),
                    (0, 8, 2, 2, 1), (0, 8, 1, 1, 1), (0, 8, 1, 5, 1), (0, 8, 1, 2, 3)]:
            with pytest.raises(glm.GLMError) as e:
                glm.glm_grouped_set_shape(h, *bad)
            assert e.value.status == glm.GLM_ERR_INVALID_ARG, bad
        # 16 warps x 4 slots of 4 KB per warp: more shared memory than one CTA has
        with pytest.raises(glm.GLMError) as e:
            glm.glm_grouped_set_shape(h, 0, 16, 1, 4, 1)
        assert e.value.status == glm.GLM_ERR_UNSUPPORTED
        assert glm.glm_grouped_get_shape(h) == before
    finally:
        glm.glm_destroy(h)


def test_grouped_many_tiny_groups_among_long_ones():
    """Hundreds of 0-3 row groups mixed with long groups (many group
    switches inside one 32-row slot), deterministic, at P=32 and P=100."""
    rng = np.random.default_rng(91)
    sizes = np.concatenate([rng.integers(0, 4, 700), [9000], rng.integers(0, 3, 500), [20000]])
    for p in (32, 100):
        gd = synth.make_grouped(len(sizes), p, 93 + p, dtype=np.float32, sizes=sizes)
        ld = synth.padded_ld(p, 4)
        Xs = synth.pad_columns(gd.X, ld)
        outs = _run_grouped(Xs, gd.y, gd.offsets, gd.beta, gd.mu, gd.tau, p, repeat=2)
        np.testing.assert_array_equal(outs[0][0], outs[1][0])
        np.testing.assert_array_equal(outs[0][1], outs[1][1])
        f_o, g_o = _oracle_grouped(Xs.astype(np.float64), gd.y, gd.offsets,
                                   gd.beta.astype(np.float32), gd.mu.astype(np.float32), gd.tau, p)
        assert_close(outs[0][0], outs[0][1], f_o, g_o, what=f"crowded P={p}")
