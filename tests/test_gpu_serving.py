"""GPU tests of the serving loop (glm_server_*): continuous batching over
device-resident BF16 datasets.

Every result is checked against the FP64 oracle on the same BF16-rounded X
(|f - f_o|/|f_o| <= 1e-4, ||g - g_o||/||g_o|| <= 1e-4), and each request's
result alone (an idle server, nothing to merge with) against the same
request inside a mix of concurrent requests merged into shared batches.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import assert_close, rel_errors, to_dev

pytestmark = pytest.mark.gpu

RTOL = 1e-4


class Datasets:
    """BF16 datasets on the device (quantised by the library), with their
    rounded copies for the oracle."""

    def __init__(self, shapes, seed):
        self.items = []
        for i, (n, p) in enumerate(shapes):
            d = synth.make_glm(n, p, seed + 7 * i, dtype=np.float32)
            ld = synth.padded_ld(p, 2)
            q = oracle.bf16_from_f32(synth.pad_columns(d.X, ld))
            self.items.append(dict(n=n, p=p, ld=ld, X=to_dev(q), y=to_dev(d.y), y_host=d.y,
                                   Xr=oracle.bf16_to_f64(q), beta_star=d.beta_star))

    def register(self, server):
        return [glm.glm_server_add_dataset(server, it["X"], None, it["y"], it["n"], it["p"],
                                           it["ld"], glm.GLM_X_BF16, 10.0)
                for it in self.items]


def make_requests(dsets, count, seed, k_max=32, k_fixed=None):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        i = int(rng.integers(len(dsets.items)))
        k = int(rng.integers(1, k_max + 1)) if k_fixed is None else k_fixed
        it = dsets.items[i]
        b = (it["beta_star"][None, :] + 0.05 * rng.standard_normal((k, it["p"]))).astype(np.float32)
        reqs.append((i, k, np.ascontiguousarray(b)))
    return reqs


def run_alone(server, ids, reqs):
    out = []
    for i, k, b in reqs:
        rid = glm.glm_server_submit(server, ids[i], b, k)
        f = np.empty(k, np.float64)
        g = np.empty((k, b.shape[1]), np.float32)
        info = glm.glm_server_wait(server, rid, f, g)
        assert info["batch_requests"] == 1 and info["batch_k"] == k
        out.append((f, g, info))
    return out


def run_mix(server, ids, reqs):
    rids = [glm.glm_server_submit(server, ids[i], b, k) for i, k, b in reqs]
    out = []
    for rid, (i, k, b) in zip(rids, reqs):
        f = np.empty(k, np.float64)
        g = np.empty((k, b.shape[1]), np.float32)
        info = glm.glm_server_wait(server, rid, f, g)
        out.append((f, g, info))
    return out


SHAPES = [(3000, 8), (20011, 37), (50000, 100), (7000, 300), (120000, 64), (1000, 512),
          (257, 256)]


def test_serving_mix_equals_alone_and_oracle():
    dsets = Datasets(SHAPES, 9100)
    server = glm.glm_server_create(0, streams=4, max_batch_k=64)
    try:
        ids = dsets.register(server)
        reqs = make_requests(dsets, 80, 9101)
        alone = run_alone(server, ids, reqs)
        mix = run_mix(server, ids, reqs)
        stats = glm.glm_server_stats(server)
    finally:
        glm.glm_server_destroy(server)
    merged = sum(1 for _, _, info in mix if info["batch_requests"] > 1)
    assert merged > 0, "no request was merged into a shared batch"
    assert stats["requests_done"] == 2 * len(reqs) and stats["requests_failed"] == 0
    assert stats["batches"] < 2 * len(reqs)
    bitwise = 0
    for (i, k, b), (fa, ga, _), (fm, gm, info) in zip(reqs, alone, mix):
        it = dsets.items[i]
        f_o, g_o = oracle.logpost_grad(it["Xr"], it["y_host"], b.astype(np.float64), p=it["p"])
        assert_close(fa, ga, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what=f"alone ds={i} K={k}")
        assert_close(fm, gm, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL,
                     what=f"mix ds={i} K={k} batch_k={info['batch_k']}")
        assert info["path"] == expected_path(it["p"], info["batch_k"]), info
        ef, eg = rel_errors(fm, gm, fa, ga)
        assert ef.max() <= RTOL and eg.max() <= RTOL, (i, k, ef.max(), eg.max())
        bitwise += int(np.array_equal(fa, fm) and np.array_equal(ga, gm))
    print(f"{len(reqs)} requests, {merged} merged in the mix, {stats['batches']} batches, "
          f"{bitwise} bitwise equal alone vs mix, max concurrent "
          f"{stats['max_concurrent_batches']}")


def _r256(b):
    return (b + 255) // 256 * 256


def batch_bytes(k, p):
    """Device bytes of a batch of k vectors: coefficients, f and g."""
    return 2 * _r256(k * p * 4) + _r256(k * 8)


def resident_bytes(dsets, streams, max_k):
    """What the registered datasets count for (data plus per-slot workspaces),
    read from a server with the default budget."""
    server = glm.glm_server_create(0, streams=streams, max_batch_k=max_k)
    try:
        dsets.register(server)
        return glm.glm_server_stats(server)["hbm_resident_bytes"]
    finally:
        glm.glm_server_destroy(server)


def expected_path(p, batch_k):
    return glm.GLM_PATH_TENSOR_CORES if batch_k >= 16 and p <= 256 else glm.GLM_PATH_CUDA_CORES


def check_against_oracle(dsets, reqs, results, what):
    for (i, k, b), (f, g, info) in zip(reqs, results):
        it = dsets.items[i]
        f_o, g_o = oracle.logpost_grad(it["Xr"], it["y_host"], b.astype(np.float64), p=it["p"])
        assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL,
                     what=f"{what} ds={i} K={k} batch_k={info['batch_k']}")
        assert info["path"] == expected_path(it["p"], info["batch_k"]), info


def test_serving_admission_defers_batches_for_device_memory():
    """The budget holds the datasets and one full batch: four stream slots,
    but never two batches in flight, later batches deferred until a
    completion gives memory back, and every result still right."""
    p, max_k = 64, 32
    dsets = Datasets([(400000, p), (9000, p), (60001, p)], 9200)
    res = resident_bytes(dsets, 4, max_k)
    assert res >= sum(it["n"] * it["ld"] * 2 + it["n"] for it in dsets.items)
    budget = res + batch_bytes(max_k, p) + batch_bytes(max_k, p) // 2
    server = glm.glm_server_create(0, streams=4, max_batch_k=max_k, hbm_budget_bytes=budget)
    try:
        ids = dsets.register(server)
        reqs = make_requests(dsets, 40, 9201, k_fixed=max_k)
        mix = run_mix(server, ids, reqs)
        stats = glm.glm_server_stats(server)
    finally:
        glm.glm_server_destroy(server)
    assert stats["hbm_resident_bytes"] == res and stats["hbm_budget_bytes"] == budget
    assert stats["max_concurrent_batches"] == 1, stats
    assert stats["deferrals"] >= 1 and sum(info["deferrals"] for _, _, info in mix) >= 1, stats
    assert stats["requests_done"] == len(reqs) and stats["requests_failed"] == 0
    assert stats["hbm_in_flight_bytes"] == 0
    check_against_oracle(dsets, reqs, mix, "deferred")
    print(f"budget {budget} B, resident {res} B: {stats['deferrals']} deferrals, "
          f"{stats['batches']} batches, max concurrent {stats['max_concurrent_batches']}")


def test_serving_admission_trims_merged_batches_to_the_budget():
    """Room for 24 vectors of one dataset: requests of 8 are merged up to what
    fits, never to max_batch_k = 64, and the rest wait their turn."""
    p = 100
    dsets = Datasets([(200000, p)], 9250)
    res = resident_bytes(dsets, 2, 64)
    budget = res + batch_bytes(24, p) + 512
    server = glm.glm_server_create(0, streams=2, max_batch_k=64, hbm_budget_bytes=budget)
    try:
        ids = dsets.register(server)
        reqs = make_requests(dsets, 48, 9251, k_fixed=8)
        mix = run_mix(server, ids, reqs)
        stats = glm.glm_server_stats(server)
    finally:
        glm.glm_server_destroy(server)
    assert max(info["batch_k"] for _, _, info in mix) <= 24
    assert max(info["batch_requests"] for _, _, info in mix) >= 2
    assert stats["trimmed_batches"] >= 1, stats
    check_against_oracle(dsets, reqs, mix, "trimmed")


def test_serving_refuses_what_cannot_fit_and_removal_returns_memory():
    p = 32
    dsets = Datasets([(50000, p), (30000, p)], 9270)
    one = Datasets([(50000, p)], 9270)
    res1 = resident_bytes(one, 2, 64)
    # room for the first dataset and a 16-vector batch, not for the second dataset
    budget = res1 + batch_bytes(16, p) + 1024
    server = glm.glm_server_create(0, streams=2, max_batch_k=64, hbm_budget_bytes=budget)
    try:
        it0, it1 = dsets.items
        ds0 = glm.glm_server_add_dataset(server, it0["X"], None, it0["y"], it0["n"], p, it0["ld"],
                                         glm.GLM_X_BF16, 10.0)
        with pytest.raises(glm.GLMError) as e:
            glm.glm_server_add_dataset(server, it1["X"], None, it1["y"], it1["n"], p, it1["ld"],
                                       glm.GLM_X_BF16, 10.0)
        assert e.value.status == glm.GLM_ERR_OOM
        stats = glm.glm_server_stats(server)
        assert stats["hbm_resident_bytes"] == res1
        # a 40-vector batch can never fit: refused at submit, nothing queued
        b = (it0["beta_star"][None, :] + np.zeros((40, p))).astype(np.float32)
        with pytest.raises(glm.GLMError) as e:
            glm.glm_server_submit(server, ds0, b, 40)
        assert e.value.status == glm.GLM_ERR_OOM
        assert glm.glm_server_stats(server)["refused_requests"] == 1
        # 16 fit, on the tensor cores
        rid = glm.glm_server_submit(server, ds0, b[:16], 16)
        f = np.empty(16, np.float64)
        g = np.empty((16, p), np.float32)
        info = glm.glm_server_wait(server, rid, f, g)
        assert info["path"] == glm.GLM_PATH_TENSOR_CORES
        f_o, g_o = oracle.logpost_grad(it0["Xr"], it0["y_host"], b[:16].astype(np.float64), p=p)
        assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what="refusal case")
        # removing the first dataset makes room for the second
        rid = glm.glm_server_submit(server, ds0, b[:1], 1)
        removed = glm.glm_server_remove_dataset(server, ds0)
        glm.glm_server_wait(server, rid)
        removed = removed or glm.glm_server_remove_dataset(server, ds0)
        assert removed
        assert glm.glm_server_stats(server)["hbm_resident_bytes"] == 0
        with pytest.raises(glm.GLMError) as e:
            glm.glm_server_submit(server, ds0, b[:1], 1)
        assert e.value.status == glm.GLM_ERR_INVALID_ARG
        with pytest.raises(glm.GLMError):
            glm.glm_server_remove_dataset(server, ds0)
        ds1 = glm.glm_server_add_dataset(server, it1["X"], None, it1["y"], it1["n"], p, it1["ld"],
                                         glm.GLM_X_BF16, 10.0)
        b1 = (it1["beta_star"][None, :] + np.zeros((3, p))).astype(np.float32)
        rid = glm.glm_server_submit(server, ds1, b1, 3)
        f = np.empty(3, np.float64)
        g = np.empty((3, p), np.float32)
        info = glm.glm_server_wait(server, rid, f, g)
        assert info["path"] == glm.GLM_PATH_CUDA_CORES
        f_o, g_o = oracle.logpost_grad(it1["Xr"], it1["y_host"], b1.astype(np.float64), p=p)
        assert_close(f, g, f_o, g_o, f_rtol=RTOL, g_rtol=RTOL, what="after removal")
    finally:
        glm.glm_server_destroy(server)


def test_serving_rejects_bad_requests_and_reports_unknown_ids():
    dsets = Datasets([(5000, 16)], 9300)
    server = glm.glm_server_create(0, streams=2, max_batch_k=8, max_pending=4)
    try:
        (ds,) = dsets.register(server)
        b = np.zeros((9, 16), np.float32)
        for bad_ds, k in [(1, 1), (-1, 1), (ds, 0), (ds, 9)]:
            with pytest.raises(glm.GLMError) as e:
                glm.glm_server_submit(server, bad_ds, b, k)
            assert e.value.status == glm.GLM_ERR_INVALID_ARG
        with pytest.raises(glm.GLMError) as e:
            glm.glm_server_wait(server, 12345, timeout_ms=10)
        assert e.value.status == glm.GLM_ERR_INVALID_ARG
        rid = glm.glm_server_submit(server, ds, b, 2)
        glm.glm_server_wait(server, rid)
        with pytest.raises(glm.GLMError):           # a finished request is forgotten
            glm.glm_server_poll(server, rid)
    finally:
        glm.glm_server_destroy(server)


def test_serving_poisson_stream_latency_and_accuracy():
    """A short Poisson stream (2,000 requests/s) from a submitting thread
    while another collects: all requests finish, latencies are recorded, and
    a sample of results matches the oracle."""
    dsets = Datasets(SHAPES, 9400)
    reqs = make_requests(dsets, 600, 9401)
    arrivals = synth.poisson_arrivals(2000.0, len(reqs), 9402)
    server = glm.glm_server_create(0, streams=4, max_batch_k=64)
    rids = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def submitter():
        t0 = time.perf_counter()
        for j, (i, k, b) in enumerate(reqs):
            while True:
                rem = arrivals[j] - (time.perf_counter() - t0)
                if rem <= 0:
                    break
                if rem > 4e-4:
                    time.sleep(rem - 3e-4)
            rids[j] = glm.glm_server_submit(server, ids[i], b, k)
            ready.release()

    try:
        ids = dsets.register(server)
        th = threading.Thread(target=submitter)
        th.start()
        results = []
        for j, (i, k, b) in enumerate(reqs):
            ready.acquire()
            f = np.empty(k, np.float64)
            g = np.empty((k, b.shape[1]), np.float32)
            info = glm.glm_server_wait(server, rids[j], f, g)
            results.append((f, g, info))
        th.join()
        stats = glm.glm_server_stats(server)
    finally:
        glm.glm_server_destroy(server)
    lat = np.array([(r[2]["done_ns"] - r[2]["submit_ns"]) * 1e-6 for r in results])
    assert (lat > 0).all()
    assert stats["requests_done"] == len(reqs)
    for j in range(0, len(reqs), 15):
        i, k, b = reqs[j]
        it = dsets.items[i]
        f_o, g_o = oracle.logpost_grad(it["Xr"], it["y_host"], b.astype(np.float64), p=it["p"])
        assert_close(results[j][0], results[j][1], f_o, g_o, f_rtol=RTOL, g_rtol=RTOL,
                     what=f"stream request {j}")
    print(f"latency ms p50 {np.percentile(lat, 50):.3f} p99 {np.percentile(lat, 99):.3f}; "
          f"batches {stats['batches']} for {len(reqs)} requests")
