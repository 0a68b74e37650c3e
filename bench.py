"""Benchmark of the logistic-GLM log-posterior + gradient hot path on GB300.

Workload: N = 2,000,000 rows, P = 100 covariates, X FP32 row-major (800 MB,
larger than the 129 MB L2), y uint8, prior N(0, 10^2 I), one coefficient
vector (K = 1). One step = one device-resident random-walk Metropolis step:
propose beta' = beta + s z, evaluate f(beta') and g(beta') in one fused pass
over X, accept in FP64 — one kernel launch. The metric is log-posterior +
gradient evaluations per second (one per step), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on this machine's host cores
(the same workload, a bounded row sample per step when a full evaluation
would not fit the time budget). Rank 0 prints one JSON line.
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


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
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


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    try:
        text = open(PROFILE_MD).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != kernel_source_hash():
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


def cpu_baseline_sample(d, seconds=12.0):
    """The oracle as it stands, single-threaded, on full evaluations for ~seconds."""
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
        if el >= seconds or n >= 50:
            break
    return {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full evaluations at N={N_ROWS}, P={P} (FP64, one thread), {el:.1f} s"}


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
    if rank == 0:
        sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # all K steps in one call: one kernel launch per step, back to back on the
    # stream, each launch programmatically dependent on the previous one
    ev0.record(stream)
    glm.glm_rwm_run(h, X, None, y, K, steps, step, zd[warmup:], lud[warmup:], state, fst, 0,
                    samples[warmup:], acc[warmup:], lp[warmup:], stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = glm.glm_sync(h, stream)
    assert st == glm.GLM_OK, glm.glm_status_str(st)
    clocks = sampler.stop() if rank == 0 else None
    total_ms = ev0.elapsed_time(ev1)
    kern_ms = total_ms / steps          # average launch-to-launch time of the kernel
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
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
        cpu = cpu_baseline_sample(d) if world == 1 else None
        peak, peak_kind = measured_hbm_peak()
        bytes_step = algorithmic_bytes_per_step()
        achieved = bytes_step / (kern_ms / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
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
            "gpu_launches": steps,
        }
        print(json.dumps(line), flush=True)
    glm.glm_destroy(h)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
