"""Benchmark: HER-accelerated BCD (HER-HALS) iterations/s and MTTKRP HBM GB/s on
one GB300, BF16 vs FP32 tensor storage, on a synthetic 500x500x500 rank-20
nonnegative tensor (factors U[0,1], 1% relative Gaussian noise clipped at 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

A step is one outer HER iteration (N MTTKRPs, N HALS block updates with
extrapolation, the F-hat restart test and the accept/restart copies).  The
tensor (500 MB FP32 / 250 MB BF16) is larger than L2, so no flush is needed.
Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica of the same workload ("replicas only": the method has no
data-parallel exchange at this size) and value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HER-BCD iterations/s and MTTKRP HBM GB/s (% of roofline), BF16 vs FP32, at equal rel. error"
WORKLOAD = "cube500_r20"
WORKLOAD_DESC = ("3-way 500x500x500 rank 20; factors U[0,1]; T = max(0, CP + N(0, sigma^2)), sigma = 1e-2 "
                 "||T_clean||_F / sqrt(numel); init U[0,1]; HER-HALS (one HALS sweep per block update, "
                 "beta0 .5, gamma 1.05, gamma_bar 1.01, eta 1.5)")
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
TIMING_EVERY = 10
KERNEL_SOURCES = ["paper_2001_04321_gb300/csrc/mttkrp_kernels.cuh", "paper_2001_04321_gb300/csrc/mttkrp_host.cu",
                  "paper_2001_04321_gb300/csrc/mttkrp_tc.cuh", "paper_2001_04321_gb300/csrc/mttkrp_tc.cu",
                  "paper_2001_04321_gb300/csrc/ntf_common.cuh", "paper_2001_04321_gb300/csrc/fused.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------
# distributed plumbing
# ----------------------------------------------------------------------------
def dist_setup(n_gpus: int):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ms_local: float, ws: int):
    """Replicas: every rank processes ``units_per_rank``; the job's time is the
    slowest rank's, so the rate is ``units_per_rank * ws / max_rank(ms)``."""
    ms = max_over_ranks(ms_local, ws)
    return units_per_rank * ws / (ms * 1e-3), ms


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ntf_clocks_{os.getpid()}_{gpu_index}.csv")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop_rows(self):
        if not self.proc:
            return []
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return rows


def summarize_clocks(rows):
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# inputs
# ----------------------------------------------------------------------------
def make_inputs():
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    T, _ = synth.make_tensor(w["dims"], w["rank"], w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    init = synth.make_init(w["dims"], w["rank"], seed=42)
    return T, init, w


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_form(ntf, torch, Td, init_d, dtype: str, steps: int, warmup: int, ws: int, stream, sample_clocks: bool,
             gpu_index: int):
    """Time `steps` HER iterations of one storage form; returns a dict."""
    F = [A.clone() for A in init_d]
    with torch.cuda.stream(stream):
        s = ntf.Solver(Td, F, ntf.Opts(compute_dtype=dtype, use_graph=True))
        s.run(warmup)
        # the timed steps replay one CUDA graph of `steps` iterations, captured here
        # (outside the timed region) with CUDA events around the MTTKRP streams of
        # every TIMING_EVERY-th iteration (the other iterations keep programmatic
        # dependent launch on every kernel boundary)
        s.set_timing(TIMING_EVERY)
        s.prepare_graph(steps)
        stream.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        sampler = ClockSampler(gpu_index) if sample_clocks else None
        L0 = ntf.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.run(steps)
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier(ws)
        L1 = ntf.launch_count()
        clocks = sampler.stop_rows() if sampler else []
        ms = e0.elapsed_time(e1)
        k_ms, k_n, k_bytes = s.mttkrp_time()
        s.set_timing(False)
        rep = s.report()
        s.close()
    return {"ms": ms, "launches": L1 - L0, "mttkrp_ms": k_ms, "mttkrp_launches": k_n, "mttkrp_bytes": k_bytes,
            "rel_error_after": rep.rel_error, "iters": rep.iters, "clock_rows": clocks}


def converge_form(ntf, torch, Td, init_d, dtype: str, iters: int, stream):
    F = [A.clone() for A in init_d]
    with torch.cuda.stream(stream):
        s = ntf.Solver(Td, F, ntf.Opts(compute_dtype=dtype, use_graph=True))
        s.run(iters)
        rep = s.report()
        s.close()
    return rep


def cpu_baseline(T, init, budget_s: float = 20.0):
    """The FP64 oracle (single thread, as it stands) on a bounded sample: HER
    iterations on the leading s x 500 x 500 slab, scaled by 500/s."""
    import numpy as np
    import oracle
    s = 25
    Ts = np.ascontiguousarray(T[:s], dtype=np.float64)
    init_s = [init[0][:s], init[1], init[2]]
    # the oracle's one-time F-hat_0 evaluation is excluded: time(iters = k) - time(iters = 0)
    t0 = time.perf_counter()
    oracle.solve(Ts, init_s, 0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.solve(Ts, init_s, 1)
    t1 = max(time.perf_counter() - t0 - t_setup, 1e-6)
    k = int(max(1, min(6, (budget_s - 2 * t_setup - t1) // t1)))
    t0 = time.perf_counter()
    oracle.solve(Ts, init_s, k)
    t_iter = time.perf_counter() - t0 - t_setup
    per_iter_full = max(t_iter, 1e-9) / k * (T.shape[0] / s)
    return {"value": 1.0 / per_iter_full, "unit": "iterations/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} HER-HALS iterations of the FP64 C oracle on the leading {s}x500x500 slab of the same "
                      f"tensor (one thread), time scaled by {T.shape[0] // s} to the full 500^3 iteration"}


def e2e_run(ntf, torch, T, init, dtype: str, steps: int, warmup: int):
    """ntf_solve_host: host T and factors (pinned) -> device -> K iterations -> factors back."""
    Th = torch.from_numpy(T).pin_memory()
    Fh = [torch.from_numpy(A.copy()).pin_memory() for A in init]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ntf.solve_host(Th, [A.clone().pin_memory() for A in Fh],
                       ntf.Opts(max_iters=max(1, warmup), compute_dtype=dtype, use_graph=True))
        st.synchronize()
        walls = []
        for _ in range(3):     # the median of three calls: one call's host copies vary from run to run
            F_call = [A.clone().pin_memory() for A in Fh]
            st.synchronize()
            t0 = time.perf_counter()
            rep = ntf.solve_host(Th, F_call, ntf.Opts(max_iters=steps, compute_dtype=dtype, use_graph=True))
            st.synchronize()
            walls.append(time.perf_counter() - t0)
    wall = sorted(walls)[1]
    h2d = T.nbytes + sum(A.nbytes for A in init)
    d2h = sum(A.nbytes for A in init)
    return {"value": steps / wall, "unit": "iterations/s", "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps,
            "calls_it_per_s": [round(steps / w, 1) for w in walls],
            "note": f"median of three ntf_solve_host calls of {steps} iterations each from pinned host memory; the "
                    f"tensor and factors are copied in once and the factors out once per call (bytes per step = per "
                    f"call / {steps}); includes solver set-up (bf16 cast, ||T||^2, F-hat_0) and the graph capture",
            "rel_error": rep.rel_error}


def read_traffic(workload: str, dtype: str):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    ent = d.get(f"{workload}:{dtype}")
    if not ent or ent.get("kernel_hash") != kernel_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def gpu_arm(args):
    import numpy as np
    import torch
    import paper_2001_04321_gb300 as ntf

    ws, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ntf.load()
    T, init, w = make_inputs()
    Td = torch.from_numpy(T).to(dev)
    init_d = [torch.from_numpy(A).to(dev) for A in init]
    stream = torch.cuda.Stream(device=dev)
    stream.wait_stream(torch.cuda.current_stream())

    forms = {}
    for dtype in ("bf16", "f32"):
        forms[dtype] = run_form(ntf, torch, Td, init_d, dtype, args.steps, args.warmup, ws, stream, rank == 0, local)
    clocks = summarize_clocks(forms["bf16"]["clock_rows"] + forms["f32"]["clock_rows"])
    rate, ms = {}, {}
    for d in forms:
        rate[d], ms[d] = whole_job_rate(args.steps, forms[d]["ms"], ws)

    # quality at matched iteration counts (untimed): both forms from the same init
    quality = {}
    for dtype in ("bf16", "f32"):
        rep = converge_form(ntf, torch, Td, init_d, dtype, args.quality_iters, stream)
        quality[dtype] = rep.rel_error
    ntf.device_status(stream)

    peaks, peak_kind = measured_peaks()
    head = "bf16"
    f = forms[head]
    per_launch_ms = f["mttkrp_ms"] / max(1, f["mttkrp_launches"])
    achieved = f["mttkrp_bytes"] / (per_launch_ms * 1e-3) / 1e9
    traffic = read_traffic(WORKLOAD, head)
    out = {
        "metric": METRIC,
        "value": rate[head],
        "unit": "iterations/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms[head] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "dims": list(w["dims"]), "rank": w["rank"],
                   "storage": "bf16 tensor (cast once, RNE), fp32 factors and accumulation, fp64 objective/restart",
                   "l2": "inputs larger than L2 (250 MB bf16 / 500 MB fp32 tensor): no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "kernel": "MTTKRP tensor-core streams k_tc_rows / k_tc_last (tcgen05, TMA)",
                     "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs (copy)",
                     "algorithmic_bytes_per_launch": f["mttkrp_bytes"],
                     "avg_launch_us": per_launch_ms * 1e3, "launches_timed": f["mttkrp_launches"],
                     "timing": f"CUDA events on the solver's stream around each MTTKRP stream launch of every "
                               f"{TIMING_EVERY}th timed iteration"},
        "forms": {},
        "gpu_launches": f["launches"],
        "clocks": clocks,
        "quality": {"iters": args.quality_iters, "rel_error_bf16": quality["bf16"], "rel_error_f32": quality["f32"],
                    "abs_diff": abs(quality["bf16"] - quality["f32"])},
    }
    for d in forms:
        g = forms[d]
        pl = g["mttkrp_ms"] / max(1, g["mttkrp_launches"])
        ach = g["mttkrp_bytes"] / (pl * 1e-3) / 1e9
        out["forms"][d] = {"iterations_per_s": rate[d], "ms_per_step": ms[d] / args.steps,
                           "mttkrp_gbs": ach, "mttkrp_frac_of_measured_hbm": ach / peaks["hbm_gbs"],
                           "mttkrp_frac_of_8tbs_nominal": ach / 8000.0, "mttkrp_avg_us": pl * 1e3,
                           "gpu_launches": g["launches"]}
    if rank == 0:
        out["e2e"] = e2e_run(ntf, torch, T, init, head, args.steps, args.warmup)
        if not args.skip_cpu:
            out["cpu_baseline"] = cpu_baseline(T, init)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------
def reference_arm(args):
    import numpy as np
    import oracle
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    T, init, w = make_inputs()
    s = 5
    Ts = np.ascontiguousarray(T[:s], dtype=np.float64)
    init_s = [init[0][:s], init[1], init[2]]
    scale = T.shape[0] / s
    st = oracle.solve(Ts, init_s, 0)  # warm the library
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.solve(Ts, init_s, 1)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    t0 = time.perf_counter()
    oracle.solve(Ts, init_s, 0)
    t_setup = time.perf_counter() - t0
    per_iter = max(statistics.mean(times) - t_setup, 1e-9) * scale
    value = 1.0 / per_iter
    sample = (f"each step: one HER-HALS iteration of the FP64 C oracle (one thread) on the leading {s}x500x500 "
              f"slab of the same tensor, minus the oracle's one-time F-hat_0 evaluation, scaled by {int(scale)}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "dims": list(w["dims"]), "rank": w["rank"]},
        "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quality-iters", type=int, default=300)
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not args.skip_cpu:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
