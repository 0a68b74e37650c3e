"""Benchmark of the logistic-GLM log-posterior + gradient hot path on GB300.

Workload: N = 2,000,000 rows, P = 100 covariates, X FP32 row-major (800 MB,
larger than the 129 MB L2), y uint8, prior N(0, 10^2 I), one coefficient
vector (K = 1). One step = one device-resident random-walk Metropolis step:
propose beta' = beta + s z, evaluate f(beta') and g(beta') in one fused pass
over X, accept in FP64 — one kernel launch. The metric is log-posterior +
gradient evaluations per second (one per step), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload big|small|batched|batched-fp8|grouped|serving|slice]

``--impl reference`` times the FP64 CPU oracle on this machine's host cores
(the same workload, a bounded row sample per step when a full evaluation
would not fit the time budget). Rank 0 prints one JSON line.

The default workload is the one above. The others measure the remaining
parts of the path, each printing its own JSON line:

- ``small``: N = 10,000, P = 50 (FP64 data stored FP32, ld 52), K = 1: 100
  evaluation points, then Metropolis steps (one launch each). X fits in L2,
  so the line reports steps/s and µs per step (launch/latency-bound) with no
  HBM fraction.
- ``batched`` / ``batched-fp8``: N = 1,000,000, P = 256, K = 64 vectors per
  call, X BF16 (tensor-core pass) or FP8 E4M3 with column scales; one step is
  one call evaluating all 64 vectors. Also times the FP32 path on the same
  X run as a loop of 64 single-vector calls.
- ``grouped``: 4,000 hierarchical-Bayes groups (log-normal sizes, median
  400, about 2.5M rows), P = 32, X FP32; one step is one replay of a CUDA
  graph holding the autotuned grouped launch (all groups' f and g).
- ``slice``: Gibbs sweeps of univariate slice sampling with the
  differential update of X beta (column-major X, N = 2,000,000, P = 100,
  FP32, w = 4.5/sqrt(N), m = 4); one step is one sweep (P coordinate
  updates, each several evaluation passes over one column).
- ``serving``: Poisson arrivals at 2,000 requests/s (``--rate``; 0 submits all at once) against 16 resident BF16
  datasets (N log-uniform in [1e3, 4e6], P log-uniform in [8, 512]), K
  uniform in 1..32 per request; one step is one request. Reports latency
  percentiles from submission to results on the host, the pass that served
  each batch, the device memory account, and a second stream at 20,000
  requests/s (``--overlap-rate``) where arrivals overlap and batches merge.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ROWS = 2_000_000
P = 100
K = 1
PRIOR_SIGMA = 10.0
WORKLOAD = "big-data logistic GLM: N=2,000,000 rows, P=100, X FP32 row-major, K=1"
METRIC = "log-posterior+grad evals/s"
UNIT = "evals/s"
PROFILE_MD = os.path.join(ROOT, "profiles", "fused_f32_big.md")
KERNEL_SOURCES = ["paper_1310_1537_gb300/csrc/glm_fused.cuh",
                  "paper_1310_1537_gb300/csrc/glm_fused_f32.cu",
                  "paper_1310_1537_gb300/csrc/glm_internal.cuh"]
TC_SOURCES = ["paper_1310_1537_gb300/csrc/glm_tc.cu",
              "paper_1310_1537_gb300/csrc/glm_tc_common.cuh",
              "paper_1310_1537_gb300/csrc/glm_internal.cuh"]
TC8_SOURCES = ["paper_1310_1537_gb300/csrc/glm_tc8.cu",
               "paper_1310_1537_gb300/csrc/glm_tc_common.cuh",
               "paper_1310_1537_gb300/csrc/glm_internal.cuh"]
GROUPED_SOURCES = ["paper_1310_1537_gb300/csrc/glm_grouped.cu",
                   "paper_1310_1537_gb300/csrc/glm_internal.cuh"]
SLICE_SOURCES = ["paper_1310_1537_gb300/csrc/glm_slice.cu",
                 "paper_1310_1537_gb300/csrc/glm_internal.cuh"]
HESS_SOURCES = ["paper_1310_1537_gb300/csrc/glm_hess.cu",
                "paper_1310_1537_gb300/csrc/glm_tc_common.cuh",
                "paper_1310_1537_gb300/csrc/glm_internal.cuh"]
ISING_SOURCES = ["paper_1310_1537_gb300/csrc/glm_ising.cu",
                 "paper_1310_1537_gb300/csrc/glm_internal.cuh"]


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for rel in (sources or KERNEL_SOURCES):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def algorithmic_bytes_per_step(n=N_ROWS, p=P, ld=P, es=4) -> int:
    """Bytes one step must move: X and y once, chain state and proposal in,
    f, g, sample, accept flag and log-posterior out."""
    x = n * ld * es
    y = n
    ins = 2 * p * 4 + 8 + 8          # state, z, f_state, log u
    outs = 8 + p * 4 + p * 4 + 1 + 8 + 8  # f, g, sample, accept, logpost, f_state
    return x + y + ins + outs


def measured_bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic(md=PROFILE_MD, sources=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    try:
        text = open(md).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_(?:launch|update):\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != kernel_source_hash(sources):
        return None
    return float(m_tr.group(1))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.gpu_id], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_data():
    import synth
    d = synth.make_glm(N_ROWS, P, synth.seed_for(1), dtype=np.float32)
    return d


def run_reference(args, world, rank):
    """The FP64 CPU oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    d = make_data()
    beta0 = d.beta_star.astype(np.float64)
    X64 = d.X.astype(np.float64)
    import synth
    z, _ = synth.rwm_streams(max(args.steps + args.warmup, 1), 1, P, synth.seed_for(1) + 3)
    step = synth.rwm_step_size(N_ROWS, P)
    # size the per-step row sample so that all steps fit about two minutes
    t0 = time.perf_counter()
    oracle.loglik_partial(X64, d.y, beta0, 0, 100_000)
    t_100k = time.perf_counter() - t0
    est_full = t_100k * N_ROWS / 100_000
    budget = 120.0 / max(args.steps + args.warmup, 1)
    rows = N_ROWS if est_full <= budget else max(10_000, int(N_ROWS * budget / est_full))
    b = beta0.copy()
    times = []
    for i in range(args.warmup + args.steps):
        bp = (b + step * z[i, 0]).astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        if rows == N_ROWS:
            oracle.logpost_grad(X64, d.y, bp, prior_sigma=PRIOR_SIGMA)
        else:
            oracle.loglik_partial(X64, d.y, bp, 0, rows)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt * N_ROWS / rows)
    per_eval = float(np.mean(times))
    value = 1.0 / per_eval
    sample = (f"full N={N_ROWS} evaluations" if rows == N_ROWS else
              f"rows [0, {rows}) of N={N_ROWS} per step, time scaled by N/rows")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_eval * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n_rows": N_ROWS, "p": P, "k": K},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def host_info():
    """Host cores this process may use and the CPU model."""
    try:
        nproc = len(os.sched_getaffinity(0))
    except Exception:
        nproc = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"nproc": nproc, "cpu_model": model, "machine": platform.machine()}


def hls_rate(X64, y, beta, p, seconds, n_total, prior_sigma=PRIOR_SIGMA):
    """The multi-core FP64 CPU baseline (the paper's partial loop fusion,
    cache fusion and one combine per thread, OpenMP on all host cores) on a
    row prefix, repeated for about `seconds`, scaled to `n_total` rows.
    Returns (evaluations/s counting every vector in beta, threads, sample)."""
    import oracle
    oracle.build_hls()
    b = np.atleast_2d(np.asarray(beta, dtype=np.float64))
    k = b.shape[0]
    nt = oracle.hls_max_threads()
    n = X64.shape[0]
    rows = min(n, 50_000)
    t0 = time.perf_counter()
    oracle.hls_logpost_grad(X64[:rows], y[:rows], b, prior_sigma, p=p, threads=nt)
    t_rows = time.perf_counter() - t0
    rows = int(min(n, max(rows, rows * seconds / max(t_rows, 1e-6) / 4)))
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.hls_logpost_grad(X64[:rows], y[:rows], b, prior_sigma, p=p, threads=nt)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 50:
            break
    per_pass = el / reps * n_total / rows
    return k / per_pass, nt, (f"{reps} x rows [0, {rows}) of N={n_total}, {k} vector(s) per "
                              f"pass, time scaled by N/rows")


def multicore_baseline(X64, y, beta, p, seconds, n_total, unit=UNIT):
    v, nt, sample = hls_rate(X64, y, beta, p, seconds, n_total)
    return {"value": v, "unit": unit, "cores": nt, "kind": "hls-openmp",
            "what": "the paper's own CPU design (partial loop fusion, cache fusion, private "
                    "gradients with one combine per thread; FP64, OpenMP), oracle/cpu_hls.c",
            "sample": sample}


def cpu_baseline_sample(d, seconds=12.0):
    """The oracle as it stands, single-threaded, on full evaluations for about
    2/3 of `seconds`, and the multi-core baseline on all host cores for the rest."""
    import oracle
    oracle.build()
    X64 = d.X.astype(np.float64)
    b = d.beta_star.astype(np.float64)
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.logpost_grad(X64, d.y, b, prior_sigma=PRIOR_SIGMA)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds * 2 / 3 or n >= 50:
            break
    return {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full evaluations at N={N_ROWS}, P={P} (FP64, one thread), {el:.1f} s",
            "host": host_info(),
            "multicore": multicore_baseline(X64, d.y, b, P, seconds / 3, N_ROWS)}


def run_ours(args, world, rank, local):
    import torch
    import synth
    import paper_1310_1537_gb300 as glm

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for --impl ours")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    d = make_data()
    X = torch.from_numpy(d.X).cuda()
    y = torch.from_numpy(d.y).cuda()
    h = glm.glm_create(N_ROWS, P, P, 8, glm.GLM_X_F32, PRIOR_SIGMA, local, 0)
    info = glm.glm_get_info(h)
    steps, warmup = args.steps, args.warmup
    z, lu = synth.rwm_streams(steps + warmup, K, P, synth.seed_for(1) + 3 + rank)
    zd = torch.from_numpy(z).cuda()
    lud = torch.from_numpy(lu).cuda()
    step = synth.rwm_step_size(N_ROWS, P)
    state = torch.from_numpy(d.beta_star[None, :].astype(np.float32)).cuda()
    fst = torch.zeros(K, dtype=torch.float64, device="cuda")
    samples = torch.empty((steps + warmup, K, P), dtype=torch.float32, device="cuda")
    acc = torch.empty((steps + warmup, K), dtype=torch.uint8, device="cuda")
    lp = torch.empty((steps + warmup, K), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    kp = K * P

    # initial log-posterior, then warm-up steps
    glm.glm_rwm_run(h, X, None, y, K, warmup, step, zd, lud, state, fst, 1, samples, acc, lp,
                    stream)
    assert glm.glm_sync(h, stream) == glm.GLM_OK

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid or str(local))

    def chain(evs):
        # all K steps in one call: one kernel launch per step, back to back on
        # the stream, each launch programmatically dependent on the previous one
        evs[0].record(stream)
        glm.glm_rwm_run(h, X, None, y, K, steps, step, zd[warmup:], lud[warmup:], state, fst, 0,
                        samples[warmup:], acc[warmup:], lp[warmup:], stream)
        evs[1].record(stream)

    # the timed region repeats the K-step chain R times (each repeat timed on
    # its own) so that it lasts about two seconds and the clock record covers
    # the load; the line reports the median repeat
    probe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    chain(probe)
    torch.cuda.synchronize()
    est_ms = max(probe[0].elapsed_time(probe[1]), 1e-3)
    repeats = int(max(5, min(2000, math.ceil(2000.0 / est_ms))))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(repeats)]
    if rank == 0:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for r in range(repeats):
        chain(evs[r])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = glm.glm_sync(h, stream)
    assert st == glm.GLM_OK, glm.glm_status_str(st)
    clocks = sampler.stop() if rank == 0 else None
    rep_ms = np.array([e[0].elapsed_time(e[1]) for e in evs])
    t = torch.tensor(rep_ms, dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    rep_ms = t.cpu().numpy()
    total_ms = float(np.median(rep_ms))     # one repeat: exactly `steps` steps
    kern_ms = total_ms / steps              # average launch-to-launch time of the kernel
    value = world * steps / (total_ms / 1e3)

    # end to end through the host-buffer entry point: beta in, f and g out per step
    e2e_steps = max(50, min(steps, 1000))
    bh = torch.from_numpy(d.beta_star[None, :].astype(np.float32)).pin_memory()
    fh = torch.empty(K, dtype=torch.float64).pin_memory()
    gh = torch.empty((K, P), dtype=torch.float32).pin_memory()
    for i in range(5):
        glm.glm_logpost_grad_host(h, X, None, y, bh, K, fh, gh, stream)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        bh[0, 0] = float(d.beta_star[0]) + 1e-4 * (i % 7)
        glm.glm_logpost_grad_host(h, X, None, y, bh, K, fh, gh, stream)
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * e2e_steps / float(te.item())

    if rank == 0:
        cpu = cpu_baseline_sample(d, seconds=args.cpu_seconds + 2.0) if world == 1 else None
        peak, peak_kind = measured_hbm_peak()
        bytes_step = algorithmic_bytes_per_step()
        achieved = bytes_step / (kern_ms / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "repeats": {"count": repeats, "steps_each": steps, "reported": "median repeat",
                        "ms_min": float(rep_ms.min()), "ms_median": float(np.median(rep_ms)),
                        "ms_max": float(rep_ms.max())},
            "config": {"workload": WORKLOAD, "n_rows": N_ROWS, "p": P, "k": K, "xtype": "f32",
                       "step": "one device-resident Metropolis step: propose, fused f+g pass "
                               "over X, FP64 accept (1 kernel launch)",
                       "l2": "inputs larger than L2 (X 800 MB vs 129 MB L2), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "grid": info["grid"], "tile_rows": info["tile_rows"],
                       "stages": info["stages"]},
            "hbm_gbs": achieved,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profile_traffic(),
                         "traffic_source": "profiles/fused_f32_big.md (ncu dram bytes, one launch)",
                         "peak_kind": f"{peak_kind} hbm_gbs", "kernel":
                             "glm::fused_logpost_grad_kernel<F32Tag, 1, 1>",
                         "algorithmic_bytes_per_launch": bytes_step,
                         "kernel_ms": kern_ms,
                         "kernel_ms_def": "timed region / launches (launches overlap by "
                                          "programmatic dependent launch)"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": K * P * 4,
                    "d2h_bytes_per_step": K * 8 + K * P * 4,
                    "api": "glm_logpost_grad_host (X resident, beta in, f and g out, synced)"},
            "clocks": clocks,
            "gpu_launches": steps * repeats,
        }
    glm.glm_destroy(h)
    del X, y, samples
    if rank == 0 and world == 1 and not args.no_workloads:
        torch.cuda.empty_cache()
        line["workloads"] = run_workload_suite(args, local, d)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Further workloads (one JSON line each)
# ---------------------------------------------------------------------------

def _gpu_sampler(local):
    import torch
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    return ClockSampler(uuid or str(local))


def _oracle_rate(X64, y, beta, p, seconds, n_total, prior_sigma=PRIOR_SIGMA):
    """Oracle evaluations per second on a row prefix sized to take about
    `seconds`, scaled to the full row count (one thread)."""
    import oracle
    oracle.build()
    n = X64.shape[0]
    rows = min(n, 20_000)
    t0 = time.perf_counter()
    oracle.loglik_partial(X64, y, beta, 0, rows, p=p)
    t_rows = time.perf_counter() - t0
    rows = int(min(n, max(rows, rows * seconds / max(t_rows, 1e-6) / 3)))
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.loglik_partial(X64, y, beta, 0, rows, p=p)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 20:
            break
    per_eval = el / reps * n_total / rows
    return 1.0 / per_eval, f"{reps} x rows [0, {rows}) of N={n_total}, time scaled by N/rows"


def _emit(line):
    print(json.dumps(line), flush=True)


_DATA_CACHE = {}      # synthetic data shared by consecutive workloads of one run


def _compact(line, extra=()):
    """The parts of a workload's line that the default run's summary keeps."""
    out = {k: line[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup",
                                "dtype") if k in line}
    cfg = line.get("config") or {}
    out["workload"] = cfg.get("workload")
    roof = line.get("roofline")
    if roof:
        out["roofline"] = {k: v for k, v in roof.items()
                           if k in ("bound", "achieved", "peak", "unit", "frac", "traffic",
                                    "peak_kind", "kernel", "tensor_tflops_algorithmic",
                                    "tensor_frac", "kernel_ms", "algorithmic_bytes_per_launch",
                                    "algorithmic_bytes_per_update", "algorithmic_flops_per_eval")
                           and v is not None}
    else:
        out["roofline"] = None
    cpu = line.get("cpu_baseline")
    if cpu:
        out["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")
                               if k in cpu}
        if cpu.get("multicore"):
            out["cpu_baseline"]["multicore"] = {k: cpu["multicore"][k] for k in
                                                ("value", "unit", "cores", "kind", "sample")}
    else:
        out["cpu_baseline"] = None
    if line.get("e2e"):
        out["e2e"] = {k: line["e2e"][k] for k in ("value", "unit") if k in line["e2e"]}
    if line.get("clocks"):
        out["clocks"] = {k: line["clocks"].get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons",
                                                            "samples")}
    out["gpu_launches"] = line.get("gpu_launches")
    for k in extra:
        if k in line:
            out[k] = line[k]
        elif k in cfg:
            out[k] = cfg[k]
    return out


def run_workload_suite(args, local, d_big):
    """Every other configuration, shortened, for the default run's
    `workloads` key: each entry carries its own roofline, CPU baseline and
    clock record."""
    import torch

    def sub(steps, warmup, cpu_s, **extra):
        a = argparse.Namespace(**vars(args))
        a.steps, a.warmup, a.cpu_seconds = steps, warmup, cpu_s
        for k, v in extra.items():
            setattr(a, k, v)
        return a

    jobs = [
        ("small", lambda: run_small(sub(1000, 20, 3.0), local), ("acceptance_rate",)),
        ("batched_bf16", lambda: run_batched(sub(20, 5, 3.0), local), ("fp32_k64_loop", "path")),
        ("batched_fp8", lambda: run_batched(sub(20, 5, 3.0), local, fp8=True),
         ("fp32_k64_loop", "path")),
        ("grouped", lambda: run_grouped(sub(20, 5, 3.0), local), ()),
        ("serving", lambda: run_serving(sub(2000, 100, 2.5, rate=SERVING_RATE), local),
         ("latency_ms", "requests_per_s", "batching", "accuracy_vs_oracle", "admission",
          "overlap_stream")),
        ("slice", lambda: run_slice(sub(2, 1, 3.0, spec=0), local, d_big),
         ("passes_per_update", "us_per_pass")),
        ("ising", lambda: run_ising(sub(10, 3, 3.0), local), ()),
        ("hessian", lambda: run_hessian(sub(10, 3, 3.0), local), ()),
    ]
    out = {}
    for name, fn, extra in jobs:
        t0 = time.perf_counter()
        try:
            c = _compact(fn(), extra)
        except Exception as e:          # reported in the line, not hidden
            c = {"error": f"{type(e).__name__}: {e}"}
        c["wall_s"] = round(time.perf_counter() - t0, 1)
        out[name] = c
        if not name.startswith("batched"):
            _DATA_CACHE.clear()
        torch.cuda.empty_cache()
    _DATA_CACHE.clear()
    return out


def run_batched(args, local, fp8=False):
    import torch
    import synth
    import paper_1310_1537_gb300 as glm
    n, p, k = 1_000_000, 256, 64
    xtype = glm.GLM_X_FP8E4M3 if fp8 else glm.GLM_X_BF16
    es = 1 if fp8 else 2
    torch.cuda.set_device(local)
    key = ("batched", n, p)
    if key not in _DATA_CACHE:
        _DATA_CACHE.clear()
        _DATA_CACHE[key] = synth.make_glm(n, p, synth.seed_for(2), dtype=np.float32)
    d = _DATA_CACHE[key]
    rng = np.random.default_rng(synth.seed_for(2) + 1)
    B = (d.beta_star[None, :] + 0.05 * rng.standard_normal((k, p))).astype(np.float32)
    X32 = torch.from_numpy(d.X).cuda()
    y = torch.from_numpy(d.y).cuda()
    h = glm.glm_create(n, p, p, k, xtype, PRIOR_SIGMA, local, 0)
    Xq = torch.empty((n, p), dtype=torch.uint8 if fp8 else torch.bfloat16, device="cuda")
    xs = torch.empty(p, dtype=torch.float32, device="cuda") if fp8 else None
    glm.glm_quantize(h, X32, p, Xq, xs)
    Bd = torch.from_numpy(B).cuda()
    f = torch.empty(k, dtype=torch.float64, device="cuda")
    g = torch.empty((k, p), dtype=torch.float32, device="cuda")
    info = glm.glm_get_info(h)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        glm.glm_logpost_grad(h, Xq, xs, y, Bd, k, f, g, stream)
    assert glm.glm_sync(h, stream) == glm.GLM_OK
    sampler = _gpu_sampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        glm.glm_logpost_grad(h, Xq, xs, y, Bd, k, f, g, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    assert glm.glm_sync(h, stream) == glm.GLM_OK
    step_ms = ev0.elapsed_time(ev1) / args.steps
    tc = bool(info["tc_enabled"]) and k >= info["tc_min_k"]
    launches_per_step = 2 if tc else -(-k // (4 if fp8 else 8))

    # the FP32 path on the same (unrounded) X, as a loop of 64 single-vector calls
    h32 = glm.glm_create(n, p, p, 1, glm.GLM_X_F32, PRIOR_SIGMA, local, 0)
    f1 = torch.empty(1, dtype=torch.float64, device="cuda")
    g1 = torch.empty((1, p), dtype=torch.float32, device="cuda")
    for j in range(3):
        glm.glm_logpost_grad(h32, X32, None, y, Bd[j:j + 1], 1, f1, g1, stream)
    torch.cuda.synchronize()
    loops = 3
    ev0.record(stream)
    for _ in range(loops):
        for j in range(k):
            glm.glm_logpost_grad(h32, X32, None, y, Bd[j:j + 1], 1, f1, g1, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    assert glm.glm_sync(h32, stream) == glm.GLM_OK
    fp32_loop_ms = ev0.elapsed_time(ev1) / loops
    glm.glm_destroy(h32)

    # end to end: 64 host vectors in, f and g out, synchronised, per call
    bh = torch.from_numpy(B).pin_memory()
    fh = torch.empty(k, dtype=torch.float64).pin_memory()
    gh = torch.empty((k, p), dtype=torch.float32).pin_memory()
    for _ in range(3):
        glm.glm_logpost_grad_host(h, Xq, xs, y, bh, k, fh, gh, stream)
    e2e_n = max(20, min(args.steps, 200))
    t0 = time.perf_counter()
    for _ in range(e2e_n):
        glm.glm_logpost_grad_host(h, Xq, xs, y, bh, k, fh, gh, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_n

    import oracle
    Xr = (oracle.bf16_to_f64(oracle.bf16_from_f32(d.X[:200_000])) if not fp8 else
          d.X[:200_000].astype(np.float64))
    cpu_v, cpu_sample = _oracle_rate(Xr, d.y[:200_000], B[0].astype(np.float64), p,
                                     args.cpu_seconds, n)
    peak, peak_kind = measured_hbm_peak()
    bytes_step = n * p * es + n + k * p * 4 * 2 + k * 8 + (p * 4 if fp8 else 0)
    achieved = bytes_step / (step_ms / 1e3) / 1e9
    flops = 2 * 2 * n * p * k
    line = ({
        "metric": METRIC, "value": k / (step_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp8e4m3" if fp8 else "bf16", "data": "synthetic",
        "config": {"workload": f"batched chains: N={n}, P={p}, K={k} vectors per call, X "
                               f"{'FP8 E4M3 + column scales' if fp8 else 'BF16'}",
                   "path": ("tcgen05 kind::f8f6f4 pass on E4M3 operands + column reduce" if fp8
                            else "tcgen05 kind::f16 pass on BF16 operands + column reduce")
                           if tc else "CUDA-core fused pass, chunks of 8 vectors",
                   "l2": f"inputs larger than L2 (X {n * p * es / 1e6:.0f} MB), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profile_traffic(os.path.join(
                         ROOT, "profiles", "tc_fp8_batched.md" if fp8 else "tc_bf16_batched.md"),
                         TC8_SOURCES if fp8 else TC_SOURCES) if tc else None,
                     "traffic_source": "ncu dram bytes of the tensor-core kernel, one launch",
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": bytes_step, "kernel_ms": step_ms,
                     "kernel_ms_def": "whole call (all launches of one step)",
                     "tensor_tflops_algorithmic": flops / (step_ms / 1e3) / 1e12 if tc else None},
        "fp32_k64_loop": {"ms_per_64_evals": fp32_loop_ms,
                          "evals_per_s": k / (fp32_loop_ms / 1e3),
                          "speedup_of_this_path": fp32_loop_ms / step_ms},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": cpu_sample, "host": host_info(),
                         "multicore": multicore_baseline(Xr, d.y[:200_000], B.astype(np.float64), p,
                                                         args.cpu_seconds / 2, n)},
        "e2e": {"value": k / e2e_s, "unit": UNIT, "h2d_bytes_per_step": k * p * 4,
                "d2h_bytes_per_step": k * 8 + k * p * 4,
                "api": "glm_logpost_grad_host (X resident, 64 vectors in, f and g out, synced)"},
        "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
    })
    glm.glm_destroy(h)
    return line


def run_grouped(args, local):
    import torch
    import synth
    import paper_1310_1537_gb300 as glm
    G, p = 4000, 32
    torch.cuda.set_device(local)
    gd = synth.make_grouped(G, p, synth.seed_for(3), dtype=np.float32)
    n = gd.X.shape[0]
    Xd = torch.from_numpy(gd.X).cuda()
    yd = torch.from_numpy(gd.y).cuda()
    od = torch.from_numpy(gd.offsets).cuda()
    bd = torch.from_numpy(gd.beta.astype(np.float32)).cuda()
    md = torch.from_numpy(gd.mu.astype(np.float32)).cuda()
    f = torch.zeros(G, dtype=torch.float64, device="cuda")
    g = torch.zeros((G, p), dtype=torch.float32, device="cuda")
    h = glm.glm_create(n, p, p, 1, glm.GLM_X_F32, PRIOR_SIGMA, local, 0, G)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        glm.glm_autotune_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g, 5, s)
        glm.glm_logpost_grad_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g, s)
    s.synchronize()
    assert glm.glm_sync(h, s) == glm.GLM_OK
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        glm.glm_logpost_grad_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g, s)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            graph.replay()
    s.synchronize()
    sampler = _gpu_sampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        ev0.record(s)
        for _ in range(args.steps):
            graph.replay()
        ev1.record(s)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    assert glm.glm_sync(h, s) == glm.GLM_OK
    step_ms = ev0.elapsed_time(ev1) / args.steps

    # end to end: group coefficients in from pinned host memory, f and g out
    bh = torch.from_numpy(gd.beta.astype(np.float32)).pin_memory()
    fh = torch.empty(G, dtype=torch.float64).pin_memory()
    gh = torch.empty((G, p), dtype=torch.float32).pin_memory()
    e2e_n = max(20, min(args.steps, 200))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(s):
        for _ in range(e2e_n):
            bd.copy_(bh, non_blocking=True)
            glm.glm_logpost_grad_grouped(h, Xd, None, yd, od, G, bd, md, gd.tau, f, g, s)
            fh.copy_(f, non_blocking=True)
            gh.copy_(g, non_blocking=True)
            s.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_n

    import oracle
    oracle.build()
    X64 = gd.X.astype(np.float64)
    t0 = time.perf_counter()
    lim = 0
    while time.perf_counter() - t0 < args.cpu_seconds and lim < G:
        lim = min(G, lim + 200)
        oracle.logpost_grad_grouped(X64, gd.y, gd.offsets[:lim + 1], gd.beta[:lim], gd.mu, gd.tau)
    el = time.perf_counter() - t0
    rows_done = sum(int(gd.offsets[min(G, j + 200)]) for j in range(0, lim, 200))
    cpu_v = G / (el * n / rows_done)
    peak, peak_kind = measured_hbm_peak()
    bytes_step = n * p * 4 + n + (G + 1) * 8 + G * p * 4 * 2 + p * 4 + G * 8
    achieved = bytes_step / (step_ms / 1e3) / 1e9
    line = ({
        "metric": METRIC, "value": G / (step_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"hierarchical-Bayes groups: G={G}, P={p}, {n} rows, X FP32, "
                               "prior N(mu, 0.5^2 I)",
                   "step": "one CUDA-graph replay of the autotuned grouped launch",
                   "l2": f"X {n * p * 4 / 1e6:.0f} MB vs 129 MB L2, no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profile_traffic(os.path.join(ROOT, "profiles", "grouped_hb.md"),
                                                GROUPED_SOURCES),
                     "traffic_source": "ncu dram bytes of the grouped kernel, one launch",
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": bytes_step, "kernel_ms": step_ms},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"groups [0, {lim}) ({rows_done} rows) repeatedly, "
                                   f"scaled to {n} rows"},
        "e2e": {"value": G / e2e_s, "unit": UNIT, "h2d_bytes_per_step": G * p * 4,
                "d2h_bytes_per_step": G * 8 + G * p * 4,
                "api": "glm_logpost_grad_grouped with beta copied in and f, g copied out"},
        "clocks": clocks, "gpu_launches": args.steps,
    })
    glm.glm_destroy(h)
    return line


def run_small(args, local):
    import torch
    import synth
    import paper_1310_1537_gb300 as glm
    n, p = 10_000, 50
    torch.cuda.set_device(local)
    seed = synth.seed_for(0)
    d = synth.make_glm(n, p, seed, dtype=np.float64)
    ld = synth.padded_ld(p, 4)
    X32 = synth.pad_columns(d.X.astype(np.float32), ld)
    Xd = torch.from_numpy(X32).cuda()
    yd = torch.from_numpy(d.y).cuda()
    h = glm.glm_create(n, p, ld, 8, glm.GLM_X_F32, PRIOR_SIGMA, local, 0)
    # 100 evaluation points, 8 per call
    pts = synth.eval_points(d.beta_star, 100, 0.1, seed + 1).astype(np.float32)
    Pd = torch.from_numpy(pts).cuda()
    f = torch.empty(8, dtype=torch.float64, device="cuda")
    g = torch.empty((8, p), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for i in range(0, 100, 8):
        kk = min(8, 100 - i)
        glm.glm_logpost_grad(h, Xd, None, yd, Pd[i:i + kk], kk, f, g, stream)
    steps, warmup = args.steps, args.warmup
    z, lu = synth.rwm_streams(steps + warmup, 1, p, seed + 3)
    zd = torch.from_numpy(z).cuda()
    lud = torch.from_numpy(lu).cuda()
    step = synth.rwm_step_size(n, p)
    state = torch.from_numpy(d.beta_star[None, :].astype(np.float32)).cuda()
    fst = torch.zeros(1, dtype=torch.float64, device="cuda")
    samples = torch.empty((steps + warmup, 1, p), dtype=torch.float32, device="cuda")
    acc = torch.empty((steps + warmup, 1), dtype=torch.uint8, device="cuda")
    lp = torch.empty((steps + warmup, 1), dtype=torch.float64, device="cuda")
    glm.glm_rwm_run(h, Xd, None, yd, 1, warmup, step, zd, lud, state, fst, 1, samples, acc, lp,
                    stream)
    assert glm.glm_sync(h, stream) == glm.GLM_OK
    sampler = _gpu_sampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    glm.glm_rwm_run(h, Xd, None, yd, 1, steps, step, zd[warmup:], lud[warmup:], state, fst, 0,
                    samples[warmup:], acc[warmup:], lp[warmup:], stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    assert glm.glm_sync(h, stream) == glm.GLM_OK
    total_ms = ev0.elapsed_time(ev1)
    # end to end: host-buffer evaluations (beta in, f and g out, synchronised)
    bh = torch.from_numpy(d.beta_star[None, :].astype(np.float32)).pin_memory()
    fh = torch.empty(1, dtype=torch.float64).pin_memory()
    gh = torch.empty((1, p), dtype=torch.float32).pin_memory()
    for _ in range(5):
        glm.glm_logpost_grad_host(h, Xd, None, yd, bh, 1, fh, gh, stream)
    e2e_n = max(100, min(steps, 2000))
    t0 = time.perf_counter()
    for _ in range(e2e_n):
        glm.glm_logpost_grad_host(h, Xd, None, yd, bh, 1, fh, gh, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_n
    cpu_v, cpu_sample = _oracle_rate(d.X, d.y, d.beta_star, p, min(5.0, args.cpu_seconds), n)
    acc_rate = float(acc[warmup:].float().mean().item())
    line = ({
        "metric": "Metropolis steps/s (one log-posterior+grad eval each)",
        "value": steps / (total_ms / 1e3), "unit": "steps/s", "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"small: N={n}, P={p} (ld {ld}), X FP32 from FP64 data, K=1, "
                               "100 evaluation points then Metropolis steps",
                   "l2": "X 2.1 MB: L2-resident, no flush; latency/launch-bound",
                   "acceptance_rate": acc_rate},
        "roofline": None,
        "cpu_baseline": {"value": cpu_v, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": cpu_sample, "host": host_info(),
                         "multicore": multicore_baseline(d.X, d.y, d.beta_star, p,
                                                         min(3.0, args.cpu_seconds), n,
                                                         unit="evals/s")},
        "e2e": {"value": 1.0 / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": p * 4,
                "d2h_bytes_per_step": 8 + p * 4,
                "api": "glm_logpost_grad_host (beta in, f and g out, synchronised)"},
        "clocks": clocks, "gpu_launches": steps,
    })
    glm.glm_destroy(h)
    return line


def run_slice(args, local, d=None):
    import torch
    import synth
    import paper_1310_1537_gb300 as glm
    n, p = N_ROWS, P
    torch.cuda.set_device(local)
    seed = synth.seed_for(1)
    if d is None:
        d = make_data()
    ld = (n + 3) // 4 * 4
    Xt = torch.from_numpy(np.ascontiguousarray(d.X.T)).cuda()      # P x N column-major X
    y = torch.from_numpy(d.y).cuda()
    w, m, s_max = 4.5 / math.sqrt(n), 4, 30
    spec = args.spec if args.spec > 0 else 2
    sm = glm.glm_slice_create(n, p, ld, w=w, m=m, s_max=s_max, spec=spec)
    sweeps, warm = args.steps, args.warmup
    lu, uni = synth.slice_streams(warm + sweeps, p, s_max, seed + 9)
    lud, unid = torch.from_numpy(lu).cuda(), torch.from_numpy(uni).cuda()
    beta = torch.from_numpy(d.beta_star.astype(np.float32)).cuda()
    eta = torch.empty(n, dtype=torch.float32, device="cuda")
    fs = torch.zeros(1, dtype=torch.float64, device="cuda")
    xk = torch.empty((warm + sweeps, p), dtype=torch.float32, device="cuda")
    gk = torch.empty((warm + sweeps, p), dtype=torch.float64, device="cuda")
    ns = torch.empty((warm + sweeps, p), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    glm.glm_slice_eta(sm, Xt, beta, eta, stream)
    glm.glm_slice_run(sm, Xt, y, eta, beta, fs, 1, warm, lud, unid, xk, gk, ns, stream)
    assert glm.glm_slice_sync(sm, stream) == glm.GLM_OK
    sampler = _gpu_sampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    glm.glm_slice_run(sm, Xt, y, eta, beta, fs, 0, sweeps, lud[warm:], unid[warm:], xk[warm:],
                      gk[warm:], ns[warm:], stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    assert glm.glm_slice_sync(sm, stream) == glm.GLM_OK
    total_ms = ev0.elapsed_time(ev1)
    updates = sweeps * p
    nsh = ns[warm:].cpu().numpy()
    # evaluation passes: one stepping-out pass (when J + K > 0; m > 1 here) plus
    # the shrinkage passes, spec proposals each, up to the accepted proposal
    props = np.minimum(nsh + 1, s_max)
    passes = int(updates + ((props + spec - 1) // spec).sum())
    # end to end: each sweep's random numbers in from pinned host memory and its
    # per-update results out, one run per sweep
    luh = torch.from_numpy(lu[warm:]).pin_memory()
    unh = torch.from_numpy(uni[warm:]).pin_memory()
    xh = torch.empty((sweeps, p), dtype=torch.float32).pin_memory()
    gh = torch.empty((sweeps, p), dtype=torch.float64).pin_memory()
    lub = torch.empty((1, p), dtype=torch.float64, device="cuda")
    unb = torch.empty((1, p, 2 + s_max), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(sweeps):
        lub.copy_(luh[i:i + 1], non_blocking=True)
        unb.copy_(unh[i:i + 1], non_blocking=True)
        glm.glm_slice_run(sm, Xt, y, eta, beta, fs, 0, 1, lub, unb, xk[i:i + 1], gk[i:i + 1],
                          None, stream)
        xh[i].copy_(xk[i], non_blocking=True)
        gh[i].copy_(gk[i], non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    assert glm.glm_slice_sync(sm, stream) == glm.GLM_OK
    # the oracle: plain log-posterior evaluations (no differential update) on a
    # row prefix, scaled to N rows and to this run's evaluations per update
    import oracle
    oracle.build()
    rows = 200_000
    X64 = d.X[:rows].astype(np.float64)
    b64 = d.beta_star.astype(np.float64)
    reps, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < args.cpu_seconds or reps < 2:
        oracle.logpost_grad(X64, d.y[:rows], b64)
        reps += 1
    eval_s = (time.perf_counter() - t1) / reps * n / rows
    # the oracle evaluates each stepping-out point separately (J + K = m - 1)
    oracle_evals = (m - 1) + props.sum() / updates
    cpu_v = 1.0 / (oracle_evals * eval_s)
    peak, peak_kind = measured_hbm_peak()
    bytes_update = n * 4 + p * 4 * 2
    achieved = bytes_update * updates / (total_ms / 1e3) / 1e9
    line = ({
        "metric": "slice-sampler coordinate updates/s", "value": updates / (total_ms / 1e3),
        "unit": "updates/s", "n_gpus": 1, "steps": sweeps, "warmup": warm,
        "ms_per_step": total_ms / sweeps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"Gibbs slice sampling with differential update: N={n}, P={p}, "
                               f"X FP32 column-major, w={w:.3g}, m={m}, s_max={s_max}, "
                               f"spec={spec}",
                   "step": "one sweep: P coordinate updates in one cooperative launch",
                   "passes_per_update": passes / updates,
                   "us_per_pass": total_ms * 1e3 / passes,
                   "l2": "each update reads one 8 MB column from HBM; eta and y stay in "
                         "shared memory"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profile_traffic(os.path.join(ROOT, "profiles", "slice_run_big.md"),
                                                SLICE_SOURCES),
                     "traffic_unit": "DRAM bytes per coordinate update",
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_update": bytes_update,
                     "note": "each update is several evaluation passes joined by grid "
                             "barriers: latency-bound, not bandwidth-bound"},
        "cpu_baseline": {"value": cpu_v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{reps} plain evaluations on rows [0, {rows}), scaled to "
                                   f"N={n} and {oracle_evals:.2f} evaluations per update"},
        "e2e": {"value": updates / e2e_s, "unit": "updates/s",
                "h2d_bytes_per_step": p * (8 + 4 * (2 + s_max)), "d2h_bytes_per_step": p * 12,
                "api": "glm_slice_run per sweep with its random numbers copied in and "
                       "per-update results copied out"},
        "clocks": clocks, "gpu_launches": 1,
    })
    glm.glm_slice_destroy(sm)
    return line


def run_ising(args, local):
    """Checkerboard Gibbs sweeps of the square-lattice Ising model (§4.3.1):
    an 8192 x 8192 denoising lattice, colour planes resident in HBM, one batch
    of uniforms per sweep. Metric: site updates per second."""
    import torch
    import synth
    import paper_1310_1537_gb300 as glm
    torch.cuda.set_device(local)
    rows = cols = 8192
    w = 2.0
    sweeps, warm = args.steps, args.warmup
    seed = synth.seed_for(5)
    y, b, _ = synth.ising_lattice(rows, cols, seed, w=w)
    H = cols // 2
    plane = rows * H
    yd = torch.from_numpy(y).cuda()
    bd = torch.from_numpy(b).cuda()
    s0 = torch.empty((rows, H), dtype=torch.uint8, device="cuda")
    s1 = torch.empty_like(s0)
    b0 = torch.empty((rows, H), dtype=torch.float32, device="cuda")
    b1 = torch.empty_like(b0)
    glm.glm_ising_split(yd, 1, rows, cols, s0, s1)
    glm.glm_ising_split(bd, 4, rows, cols, b0, b1)
    # uniforms: drawn on the device by torch's generator (setup, not timed);
    # the same (n, 2, rows, cols / 2) batch layout the oracle reads
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 1)
    u = torch.rand((warm + sweeps, 2, rows, H), dtype=torch.float32, device="cuda", generator=gen)
    ones = torch.zeros(2 * (warm + sweeps), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    glm.glm_ising_sweeps(s0, s1, b0, b1, rows, cols, w, warm, u[:warm], ones[:2 * warm], stream)
    torch.cuda.synchronize()
    sampler = _gpu_sampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    glm.glm_ising_sweeps(s0, s1, b0, b1, rows, cols, w, sweeps, u[warm:], ones[2 * warm:], stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = ev0.elapsed_time(ev1)
    updates = rows * cols * sweeps
    # the denoised fraction agreeing with the clean image (a sanity figure)
    s_nat = torch.empty((rows, cols), dtype=torch.uint8, device="cuda")
    glm.glm_ising_merge(s0, s1, 1, rows, cols, s_nat)
    # end to end: each sweep's uniforms copied in from pinned host memory and
    # its two counts of ones copied out
    e2e_sweeps = min(sweeps, 4)
    uh = u[warm:warm + e2e_sweeps].cpu().pin_memory()
    ub = torch.empty((1, 2, rows, H), dtype=torch.float32, device="cuda")
    oh = torch.empty(2 * e2e_sweeps, dtype=torch.int64).pin_memory()
    ob = torch.empty(2, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_sweeps):
        ub.copy_(uh[i:i + 1], non_blocking=True)
        glm.glm_ising_sweeps(s0, s1, b0, b1, rows, cols, w, 1, ub, ob, stream)
        oh[2 * i:2 * i + 2].copy_(ob, non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    # the oracle: NumPy half-sweeps on a 2048 x 2048 corner of the lattice
    import oracle
    sr, sc = 2048, 2048
    ys, bs = y[:sr, :sc], b[:sr, :sc]
    us = synth.ising_uniforms(1, sr, sc, seed + 2)
    reps, t1 = 0, time.perf_counter()
    st = ys
    while time.perf_counter() - t1 < args.cpu_seconds or reps < 1:
        for c in (0, 1):
            st, _ = oracle.ising_half_sweep(st, bs, w, c, us[0, c])
        reps += 1
    cpu_rate = reps * sr * sc / (time.perf_counter() - t1)
    peak, peak_kind = measured_hbm_peak()
    bytes_update = 4 + 4 + 1 + 1       # bias, uniform, spin written, other colour read
    achieved = bytes_update * updates / (total_ms / 1e3) / 1e9
    return ({
        "metric": "Ising site updates/s", "value": updates / (total_ms / 1e3),
        "unit": "site updates/s", "n_gpus": 1, "steps": sweeps, "warmup": warm,
        "ms_per_step": total_ms / sweeps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"checkerboard Gibbs, square-lattice Ising denoising: "
                               f"{rows} x {cols} spins, w={w}, colour planes, batch uniforms",
                   "step": "one sweep (two half-sweep launches)",
                   "l2": "inputs larger than L2 (uniforms 268 MB per sweep), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profile_traffic(os.path.join(ROOT, "profiles", "ising_big.md"),
                                                ISING_SOURCES),
                     "traffic_unit": "DRAM bytes per site update",
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_update": bytes_update},
        "cpu_baseline": {"value": cpu_rate, "unit": "site updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{reps} NumPy sweeps of a {sr} x {sc} corner"},
        "e2e": {"value": rows * cols * e2e_sweeps / e2e_s, "unit": "site updates/s",
                "h2d_bytes_per_step": plane * 2 * 4, "d2h_bytes_per_step": 16,
                "api": "glm_ising_sweeps per sweep with its uniforms copied in and the counts out"},
        "clocks": clocks, "gpu_launches": 2 * sweeps,
    })


def run_hessian(args, local):
    """One pass returning f, g and the Hessian (N = 2,000,000, P = 64, FP32,
    one coefficient vector); X^T W X on the tensor cores."""
    import torch
    import synth
    import paper_1310_1537_gb300 as glm
    torch.cuda.set_device(local)
    n, p = 2_000_000, 64
    d = synth.make_glm(n, p, synth.seed_for(6), dtype=np.float32)
    Xd = torch.from_numpy(d.X).cuda()
    yd = torch.from_numpy(d.y).cuda()
    bd = torch.from_numpy(d.beta_star.astype(np.float32)).cuda()
    f = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(p, dtype=torch.float32, device="cuda")
    H = torch.empty((p, p), dtype=torch.float32, device="cuda")
    h = glm.glm_hess_create(n, p, p)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        glm.glm_hess_eval(h, Xd, yd, bd, f, g, H, stream)
    assert glm.glm_hess_sync(h, stream) == glm.GLM_OK
    sampler = _gpu_sampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        glm.glm_hess_eval(h, Xd, yd, bd, f, g, H, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    assert glm.glm_hess_sync(h, stream) == glm.GLM_OK
    ms = ev0.elapsed_time(ev1) / args.steps
    # end to end: beta in from pinned host memory, f, g and H out, synchronised
    bh = torch.from_numpy(d.beta_star.astype(np.float32)).pin_memory()
    fh = torch.empty(1, dtype=torch.float64).pin_memory()
    gh = torch.empty(p, dtype=torch.float32).pin_memory()
    Hh = torch.empty((p, p), dtype=torch.float32).pin_memory()
    reps = 50
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        bd.copy_(bh, non_blocking=True)
        glm.glm_hess_eval(h, Xd, yd, bd, f, g, H, stream)
        fh.copy_(f, non_blocking=True)
        gh.copy_(g, non_blocking=True)
        Hh.copy_(H, non_blocking=True)
        stream.synchronize()
    e2e = reps / (time.perf_counter() - t0)
    glm.glm_hess_destroy(h)
    # the oracle on a row sample, scaled to N
    import oracle
    rows = 200_000
    X64 = d.X[:rows].astype(np.float64)
    b64 = d.beta_star.astype(np.float64)
    k, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < args.cpu_seconds or k < 2:
        oracle.logpost_grad_hess(X64, d.y[:rows], b64)
        k += 1
    cpu = 1.0 / ((time.perf_counter() - t1) / k * n / rows)
    flops = 2 * n * p * p                          # X^T W X (the full P x P contraction)
    # issued tensor-core work: per 128-row tile one 128 x 128 x 128 product
    # (hi/lo terms of w x against hi/lo terms of x), BF16 operands
    mma_flops = 2 * 128 * 128 * 128 * (-(-n // 128))
    bf16_peak = measured_bf16_peak()
    bytes_eval = n * p * 4 + n + p * 4 + 8 + p * 4 + p * p * 4
    peak, peak_kind = measured_hbm_peak()
    achieved = bytes_eval / (ms / 1e3) / 1e9
    line = ({
        "metric": "log-posterior+grad+Hessian evals/s", "value": 1e3 / ms, "unit": "evals/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"one-pass f, g, Hessian: N={n}, P={p}, X FP32 row-major, K=1",
                   "path": "tcgen05 kind::f16: X^T W X from BF16 hi/lo terms, D in tensor memory",
                   "l2": "inputs larger than L2 (X 512 MB), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profile_traffic(os.path.join(ROOT, "profiles", "hess_big.md"),
                                                HESS_SOURCES),
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": bytes_eval,
                     "tensor_tflops_issued": mma_flops / (ms / 1e3) / 1e12,
                     "tensor_frac": mma_flops / (ms / 1e3) / 1e12 / bf16_peak[0],
                     "tensor_peak_kind": f"{bf16_peak[1]} bf16_tflops (dense, burst)",
                     "algorithmic_flops_per_eval": flops},
        "cpu_baseline": {"value": cpu, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": f"{k} NumPy evaluations on rows [0, {rows}), scaled to N={n}"},
        "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": p * 4,
                "d2h_bytes_per_step": 8 + p * 4 + p * p * 4,
                "api": "glm_hess_eval with beta in and f, g, H out, synced"},
        "clocks": clocks, "gpu_launches": 2 * args.steps,
    })
    return line


SERVING_RATE = 2000.0


def run_serving(args, local):
    import threading
    import torch
    import synth
    import paper_1310_1537_gb300 as glm
    torch.cuda.set_device(local)
    seed = synth.seed_for(4)
    shapes = synth.serving_datasets(16, seed)
    server = glm.glm_server_create(local, streams=4, max_batch_k=64)
    dsets = []
    for i, (n, p) in enumerate(shapes):
        d = synth.make_glm(n, p, seed + 1 + i, dtype=np.float32)
        ld = synth.padded_ld(p, 2)
        X32 = torch.from_numpy(synth.pad_columns(d.X, ld)).cuda()
        Xq = torch.empty((n, ld), dtype=torch.bfloat16, device="cuda")
        hq = glm.glm_create(n, p, ld, 1, glm.GLM_X_BF16, PRIOR_SIGMA, local, 0)
        glm.glm_quantize(hq, X32, ld, Xq, None)
        torch.cuda.synchronize()
        glm.glm_destroy(hq)
        del X32
        yd = torch.from_numpy(d.y).cuda()
        ds = glm.glm_server_add_dataset(server, Xq, None, yd, n, p, ld, glm.GLM_X_BF16,
                                        PRIOR_SIGMA)
        dsets.append(dict(n=n, p=p, ld=ld, Xq=Xq, y=yd, d=d, id=ds))
    def stream(rate, count, seed_off, keep_from, keep_every):
        """One request stream at `rate` requests/s (0: all at once); returns
        the request infos, kept results, failures, submit lags and requests."""
        rng = np.random.default_rng(seed + seed_off)
        reqs = []
        for _ in range(count):
            i = int(rng.integers(len(dsets)))
            k = int(rng.integers(1, 33))
            it = dsets[i]
            b = (it["d"].beta_star[None, :] + 0.05 * rng.standard_normal((k, it["p"])))
            reqs.append((i, k, np.ascontiguousarray(b, dtype=np.float32)))
        arrivals = (synth.poisson_arrivals(rate, count, seed + seed_off + 1) if rate > 0
                    else np.zeros(count))
        rids = [0] * count
        submit_lag = np.zeros(count)
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
                submit_lag[j] = time.perf_counter() - t0 - arrivals[j]
                rids[j] = glm.glm_server_submit(server, dsets[i]["id"], b, k)
                ready.release()

        th = threading.Thread(target=submitter)
        th.start()
        infos, outs, failures = [], {}, []
        keep = set(range(keep_from, count, keep_every))
        for j, (i, k, b) in enumerate(reqs):
            ready.acquire()
            fbuf = np.empty(k, np.float64)
            gbuf = np.empty((k, b.shape[1]), np.float32)
            try:
                infos.append(glm.glm_server_wait(server, rids[j], fbuf, gbuf, timeout_ms=120000))
            except glm.GLMError as e:
                failures.append({"request": j, "dataset": i, "n": dsets[i]["n"],
                                 "p": dsets[i]["p"], "k": k, "status": e.status})
                continue
            if j in keep:
                outs[j] = (fbuf, gbuf)
        th.join()
        return infos, outs, failures, submit_lag, reqs

    def batch_table(timed):
        batches = {}
        for r in timed:
            batches.setdefault((r["start_ns"], r["batch_k"]), (r["batch_requests"], r["path"]))
        return batches

    rate = SERVING_RATE if args.rate is None else args.rate
    count = args.warmup + args.steps
    sampler = _gpu_sampler(local)
    sampler.start()
    infos, outs, failures, submit_lag, reqs = stream(rate, count, 100, args.warmup,
                                                      max(1, args.steps // 400))
    clocks = sampler.stop()
    # a second stream at a rate where arrivals for one dataset overlap the
    # batches in flight, so that merging is exercised beyond the saturation case
    overlap = None
    if failures == [] and args.overlap_rate > 0 and rate > 0:
        o_infos, _, o_fail, _, _ = stream(args.overlap_rate, 2 * args.steps + args.warmup, 200,
                                          1 << 62, 1)
        failures += o_fail
        o_timed = o_infos[args.warmup:]
        o_lat = np.array([(r["done_ns"] - r["submit_ns"]) * 1e-6 for r in o_timed])
        o_span = (max(r["done_ns"] for r in o_timed) - min(r["submit_ns"] for r in o_timed)) * 1e-9
        o_batches = batch_table(o_timed)
        overlap = {"rate_per_s": args.overlap_rate, "requests": len(o_timed),
                   "value": sum(r["k"] for r in o_timed) / o_span, "unit": UNIT,
                   "requests_per_s": len(o_timed) / o_span,
                   "latency_ms": {"p50": float(np.percentile(o_lat, 50)),
                                  "p99": float(np.percentile(o_lat, 99))},
                   "mean_requests_per_batch": float(np.mean([v[0] for v in o_batches.values()])),
                   "mean_vectors_per_batch": float(np.mean([bk for _, bk in o_batches])),
                   "batches_tensor_cores": sum(1 for v in o_batches.values()
                                               if v[1] == glm.GLM_PATH_TENSOR_CORES)}
    stats = glm.glm_server_stats(server)
    glm.glm_server_destroy(server)
    if failures:
        raise RuntimeError(json.dumps({"failed_requests": len(failures),
                                       "first_failures": failures[:10], "server_stats": stats}))
    timed = infos[args.warmup:]
    lat_ms = np.array([(r["done_ns"] - r["submit_ns"]) * 1e-6 for r in timed])
    queue_ms = np.array([(r["start_ns"] - r["submit_ns"]) * 1e-6 for r in timed])
    span_s = (max(r["done_ns"] for r in timed) - min(r["submit_ns"] for r in timed)) * 1e-9
    vectors = sum(r["k"] for r in timed)
    batches = batch_table(timed)
    # accuracy: sampled requests against the FP64 oracle on the rounded X,
    # bounded to about 20 s of oracle time
    import oracle
    oracle.build()
    errs_f, errs_g, checked = [], [], 0
    t0 = time.perf_counter()
    rounded = {}
    for j in sorted(outs, key=lambda j: dsets[reqs[j][0]]["n"] * dsets[reqs[j][0]]["ld"]):
        if time.perf_counter() - t0 > 2 * args.cpu_seconds:
            break
        i, k, b = reqs[j]
        it = dsets[i]
        if i not in rounded:
            rounded.clear()
            rounded[i] = oracle.bf16_to_f64(oracle.bf16_from_f32(
                synth.pad_columns(it["d"].X, it["ld"])))
        f_o, g_o = oracle.logpost_grad(rounded[i], it["d"].y, b[:1].astype(np.float64),
                                       p=it["p"])
        fo, go = outs[j]
        errs_f.append(float(abs(fo[0] - f_o[0]) / abs(f_o[0])))
        errs_g.append(float(np.linalg.norm(go[0] - g_o[0]) / np.linalg.norm(g_o[0])))
        checked += 1
    bytes_total = sum(dsets[reqs[j][0]]["n"] * dsets[reqs[j][0]]["ld"] * 2 for j in
                      range(args.warmup, count))
    peak, peak_kind = measured_hbm_peak()
    value = vectors / span_s
    return ({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": span_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": (f"serving: Poisson {rate:.0f} requests/s" if rate > 0 else
                                "serving: all requests submitted at once (saturation)") +
                               ", 16 resident BF16 datasets (N log-uniform [1e3, 4e6], "
                               "P log-uniform [8, 512]), K uniform 1..32 per request",
                   "step": "one request", "streams": 4, "max_batch_k": 64,
                   "datasets": [[it["n"], it["p"]] for it in dsets],
                   "l2": "datasets 0.79 GB in total, mostly larger than L2; no flush"},
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                       "p90": float(np.percentile(lat_ms, 90)),
                       "p99": float(np.percentile(lat_ms, 99)),
                       "max": float(lat_ms.max()), "mean": float(lat_ms.mean()),
                       "queue_p50": float(np.percentile(queue_ms, 50)),
                       "queue_p99": float(np.percentile(queue_ms, 99)),
                       "def": "host steady clock, request submitted -> results on the host"},
        "submit_lag_ms_p99": float(np.percentile(submit_lag[args.warmup:], 99) * 1e3),
        "overlap_stream": overlap,
        "requests_per_s": args.steps / span_s,
        "batching": {"batches": len(batches),
                     "mean_requests_per_batch": float(np.mean([v[0] for v in batches.values()])),
                     "mean_vectors_per_batch": float(np.mean([bk for _, bk in batches])),
                     "batches_tensor_cores": sum(1 for v in batches.values()
                                                 if v[1] == glm.GLM_PATH_TENSOR_CORES),
                     "batches_cuda_cores": sum(1 for v in batches.values()
                                               if v[1] == glm.GLM_PATH_CUDA_CORES),
                     "path_rule": "tensor cores for batches of >= 16 vectors on datasets "
                                  "with P <= 256, else CUDA cores",
                     "max_concurrent_batches": stats["max_concurrent_batches"],
                     "failed": stats["requests_failed"]},
        "admission": {"budget_bytes": stats["hbm_budget_bytes"],
                      "resident_bytes": stats["hbm_resident_bytes"],
                      "deferrals": stats["deferrals"],
                      "trimmed_batches": stats["trimmed_batches"],
                      "refused_requests": stats["refused_requests"],
                      "rule": "datasets + per-slot workspaces + batches in flight within "
                              "the budget (default: free device memory at start less 1/16)"},
        "accuracy_vs_oracle": {"requests_checked": checked,
                               "max_rel_err_f": max(errs_f) if errs_f else None,
                               "max_rel_err_g": max(errs_g) if errs_g else None,
                               "x": "oracle on the same BF16-rounded X, first vector"},
        "roofline": {"bound": "hbm", "achieved": bytes_total / span_s / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": bytes_total / span_s / 1e9 / peak,
                     "traffic": None, "peak_kind": f"{peak_kind} hbm_gbs",
                     "note": "offered load: X bytes of every request over the run; the "
                             "stream is latency-bound at this arrival rate"},
        "cpu_baseline": None,
        "e2e": {"value": value, "unit": UNIT,
                "h2d_bytes_per_step": int(np.mean([k * dsets[i]["p"] * 4 for i, k, _ in reqs])),
                "d2h_bytes_per_step": int(np.mean([k * (8 + dsets[i]["p"] * 4)
                                                   for i, k, _ in reqs])),
                "api": "glm_server_submit / glm_server_wait (host buffers)"},
        "clocks": clocks, "gpu_launches": None,
    })


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rate", type=float, default=None,
                    help="serving arrival rate in requests/s (0: all at once); default 2000")
    ap.add_argument("--overlap-rate", type=float, default=20000.0,
                    help="serving: rate of a second stream where arrivals overlap (0: none)")
    ap.add_argument("--spec", type=int, default=0,
                    help="slice workload: shrinkage proposals per evaluation pass (0: 2)")
    ap.add_argument("--workload", default="big",
                    choices=["big", "small", "batched", "batched-fp8", "grouped", "serving",
                             "slice", "ising", "hessian"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="host time per CPU-baseline measurement")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default run: leave out the summary of the other workloads")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.workload != "big":
        if rank != 0:
            return
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle arm is timed for the default workload only; the "
                              "other workload lines carry their own cpu_baseline"}))
            return
        _emit({"small": lambda: run_small(args, local),
         "slice": lambda: run_slice(args, local),
         "ising": lambda: run_ising(args, local),
         "hessian": lambda: run_hessian(args, local),
         "batched": lambda: run_batched(args, local),
         "batched-fp8": lambda: run_batched(args, local, fp8=True),
         "grouped": lambda: run_grouped(args, local),
         "serving": lambda: run_serving(args, local)}[args.workload]())
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
