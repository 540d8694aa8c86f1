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
# CUDA events bracket the three MTTKRP streams of every TIMING_EVERY-th iteration of a timed
# region; those launches (and the kernels right after them) run without programmatic dependent
# launch, so the instrumentation itself costs throughput (measured at 500^3 BF16: 6999 it/s with no
# events, 6914 with every 20th iteration timed, 6824 with every 10th).  One timed iteration per
# 20 keeps that cost near 1% and still times every mode's stream in every region.
TIMING_EVERY = 20
MIN_TIMED_S = 0.5           # every form's timed regions cover at least this much GPU time ...
MIN_TIMED_LAUNCHES = 90     # ... and at least this many event-timed MTTKRP launches
MAX_REPEATS = 400
# the files that define the timed tensor-core stream kernels (the traffic record goes null when
# any of them changes)
KERNEL_SOURCES = ["paper_2001_04321_gb300/csrc/mttkrp_tc.cu", "paper_2001_04321_gb300/csrc/mttkrp_tc.cuh",
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
    """Time `steps` HER iterations of one storage form.  Every timed region is exactly `steps`
    iterations (one replay of a CUDA graph of `steps` iterations, bracketed by a barrier and
    synchronisation); the region is repeated until at least MIN_TIMED_S seconds and
    MIN_TIMED_LAUNCHES event-timed MTTKRP launches are covered, and the median is reported."""
    F = [A.clone() for A in init_d]
    with torch.cuda.stream(stream):
        s = ntf.Solver(Td, F, ntf.Opts(compute_dtype=dtype, use_graph=True))
        s.run(warmup)
        # the graph is captured here (outside the timed regions) with CUDA events around the
        # MTTKRP streams of every TIMING_EVERY-th iteration (the other iterations keep
        # programmatic dependent launch on every kernel boundary)
        s.set_timing(TIMING_EVERY)
        s.prepare_graph(steps)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # one untimed replay sizes the repeats
        e0.record(stream)
        s.run(steps)
        e1.record(stream)
        stream.synchronize()
        est_ms = max(e0.elapsed_time(e1), 1e-3)
        _, n_timed, _ = s.mttkrp_time()
        reps = max(1, -(-int(MIN_TIMED_S * 1e3) // int(max(1, est_ms))),
                   -(-MIN_TIMED_LAUNCHES // max(1, n_timed)))
        reps = int(max_over_ranks(float(min(reps, MAX_REPEATS)), ws))
        sampler = ClockSampler(gpu_index) if sample_clocks else None
        times, k_ms, k_n, k_bytes, launches = [], 0.0, 0, 0.0, 0
        for _ in range(reps):
            barrier(ws)
            torch.cuda.synchronize()
            L0 = ntf.launch_count()
            e0.record(stream)
            s.run(steps)
            e1.record(stream)
            stream.synchronize()
            torch.cuda.synchronize()
            barrier(ws)
            launches = ntf.launch_count() - L0
            times.append(e0.elapsed_time(e1))
            a, b, c = s.mttkrp_time()
            k_ms, k_n, k_bytes = k_ms + a, k_n + b, c
        clocks = sampler.stop_rows() if sampler else []
        s.set_timing(False)
        rep = s.report()
        s.close()
    return {"ms": statistics.median(times), "repeats": reps, "timed_s": sum(times) * 1e-3, "launches": launches,
            "mttkrp_ms": k_ms, "mttkrp_launches": k_n, "mttkrp_bytes": k_bytes, "rel_error_after": rep.rel_error,
            "iters": rep.iters, "clock_rows": clocks}


def time_to_target(ntf, torch, Td, init_d, dtype: str, target: float, stream, chunk: int = 10,
                   max_iters: int = 1200):
    """Iterations and GPU seconds for one storage form to reach a relative error (explicit,
    against the FP32 tensor) of `target`: chunks of `chunk` iterations replayed as a graph and
    timed with CUDA events; the error is evaluated between chunks, outside the timing."""
    F = [A.clone() for A in init_d]
    with torch.cuda.stream(stream):
        s = ntf.Solver(Td, F, ntf.Opts(compute_dtype=dtype, use_graph=True))
        s.prepare_graph(chunk)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms, it, err = 0.0, 0, float("inf")
        while it < max_iters:
            e0.record(stream)
            s.run(chunk)
            e1.record(stream)
            stream.synchronize()
            ms += e0.elapsed_time(e1)
            it += chunk
            err = s.report().rel_error
            if err <= target:
                break
        s.close()
    return {"iterations": it, "seconds": ms * 1e-3, "rel_error": err, "reached": err <= target}


def converge_form(ntf, torch, Td, init_d, dtype: str, iters: int, stream):
    F = [A.clone() for A in init_d]
    with torch.cuda.stream(stream):
        s = ntf.Solver(Td, F, ntf.Opts(compute_dtype=dtype, use_graph=True))
        s.run(iters)
        rep = s.report()
        s.close()
    return rep


def _oracle_slab_iterations(Ts, init_s, k):
    """Seconds for k HER-HALS iterations of the oracle on one slab, without its one-time
    F-hat_0 evaluation (time(k) - time(0)).  Module level: runs in spawned worker processes."""
    import numpy as np
    import oracle
    Ts = np.ascontiguousarray(Ts, dtype=np.float64)
    t0 = time.perf_counter()
    oracle.solve(Ts, init_s, 0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.solve(Ts, init_s, k)
    return max(time.perf_counter() - t0 - t_setup, 1e-9)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(T, init, budget_s: float = 20.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: HER-HALS
    iterations on 25 x 500 x 500 slabs (the leading slab on one thread; one slab per host core
    in spawned processes for the all-cores figure), each slab iteration scaled by 500/25."""
    import multiprocessing as mp
    import numpy as np
    s = 25
    scale = T.shape[0] // s
    slab = lambda i: np.ascontiguousarray(T[i * s:(i + 1) * s])
    init_slab = lambda i: [init[0][i * s:(i + 1) * s], init[1], init[2]]
    t1 = _oracle_slab_iterations(slab(0), init_slab(0), 1)
    k = int(max(1, min(6, budget_s // 2 // t1)))
    t_k = _oracle_slab_iterations(slab(0), init_slab(0), k)
    single = k / (t_k * scale)
    P = host_cores()
    P_used = min(P, scale)
    with mp.get_context("spawn").Pool(P_used) as pool:
        secs = pool.starmap(_oracle_slab_iterations, [(slab(i), init_slab(i), k) for i in range(P_used)])
    allc = P_used * k / (max(secs) * scale)
    return {"value": single, "unit": "iterations/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} HER-HALS iterations of the FP64 C oracle on the leading {s}x500x500 slab of the same "
                      f"tensor (one thread), without its one-time F-hat_0, time scaled by {scale} to the full "
                      f"500^3 iteration (an extrapolation: no full 500^3 oracle iteration is timed)",
            "all_cores": {"value": allc, "unit": "iterations/s", "cores": P_used, "host_cores": P,
                          "sample": f"{P_used} oracle processes at once, each {k} iterations on its own {s}x500x500 "
                                    f"slab; full-iteration rate = slab iterations done / slowest process time / "
                                    f"{scale}"}}


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


# ----------------------------------------------------------------------------
# further workloads of the method (each its own key in the JSON line)
# ----------------------------------------------------------------------------
def _free(torch):
    import gc
    gc.collect()
    torch.cuda.empty_cache()


def _timed(torch, stream, fn, reps=1):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) / reps


def wl_illcond(ntf, torch, dev, stream, peaks):
    """100^3 rank 10, ill-conditioned factors, 0.1% noise: HALS vs HER-HALS, 500 iterations."""
    import numpy as np
    import synth
    w = synth.WORKLOADS["cube100_r10_illcond"]
    T, A_true = synth.make_tensor(w["dims"], w["rank"], w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    init = synth.make_init(w["dims"], w["rank"], seed=42)
    Td = torch.from_numpy(T).to(dev)
    iters = 500
    out = {"dims": list(w["dims"]), "rank": w["rank"], "dtype": "f32", "iterations": iters,
           "gram_condition_numbers": [float(np.linalg.cond(A.T @ A)) for A in A_true]}
    for name, her in (("hals", False), ("her_hals", True)):
        F = [torch.from_numpy(A).to(dev) for A in init]
        with torch.cuda.stream(stream):
            s = ntf.Solver(Td, F, ntf.Opts(her=her, use_graph=True))
            s.prepare_graph(iters)
        ms = _timed(torch, stream, lambda: s.run(iters))
        rep = s.report(stream)
        s.close()
        out[name] = {"iterations_per_s": iters / (ms * 1e-3), "ms": ms, "rel_error": rep.rel_error,
                     "restarts": rep.restarts}
    del Td
    _free(torch)
    return out


def wl_form_rates(ntf, torch, dev, stream, peaks, key, steps=100):
    """HER-HALS iterations/s and MTTKRP GB/s per storage form on a named workload."""
    import synth
    w = synth.WORKLOADS[key]
    T, _ = synth.make_tensor(w["dims"], w["rank"], w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    init = synth.make_init(w["dims"], w["rank"], seed=42)
    Td = torch.from_numpy(T).to(dev)
    init_d = [torch.from_numpy(A).to(dev) for A in init]
    out = {"dims": list(w["dims"]), "rank": w["rank"], "recipe": w["recipe"], "steps_per_region": steps}
    for dtype in ("bf16", "f32"):
        f = run_form(ntf, torch, Td, init_d, dtype, steps, 5, 1, stream, False, 0)
        pl = f["mttkrp_ms"] / max(1, f["mttkrp_launches"])
        ach = f["mttkrp_bytes"] / (pl * 1e-3) / 1e9
        out[dtype] = {"iterations_per_s": steps / (f["ms"] * 1e-3), "rel_error_after": f["rel_error_after"],
                      "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": ach / peaks["hbm_gbs"], "avg_launch_us": pl * 1e3,
                                   "launches_timed": f["mttkrp_launches"],
                                   "algorithmic_bytes_per_launch": f["mttkrp_bytes"]},
                      "gpu_launches_per_step": f["launches"] / steps}
    del Td, init_d
    _free(torch)
    return out


def wl_autograd(ntf, torch, dev, stream, peaks):
    """300^3 rank 32 FP32: CP-loss forward + hand-written backward (autograd), and 200
    iterations of projected gradient blocks with HER."""
    import synth
    w = synth.WORKLOADS["cube300_r32"]
    T, _ = synth.make_tensor(w["dims"], w["rank"], w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    init = synth.make_init(w["dims"], w["rank"], seed=42)
    Td = torch.from_numpy(T).to(dev)
    leaves = [torch.from_numpy(A).to(dev).requires_grad_(True) for A in init]
    N = len(w["dims"])
    with torch.cuda.stream(stream):
        tn = ntf.tensor_norm_sq(Td)       # a property of the data, computed once

    def step():
        for A in leaves:
            A.grad = None
        loss = ntf.cp_loss(Td, leaves, tnorm_sq=tn)
        loss.backward()

    with torch.cuda.stream(stream):
        for _ in range(3):
            step()
    reps = 20
    eager_ms = _timed(torch, stream, step, reps)
    nbytes = N * T.size * 4          # N MTTKRP passes: 1 in the forward, N-1 in the backward
    # the same forward + backward captured once as a CUDA graph and replayed (how a training
    # loop runs it): the eager figure above is bound by Python and launch overhead
    graph_ms, graph_note = None, None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
            step()
        graph_ms = _timed(torch, stream, g.replay, reps)
    except Exception as exc:          # capture not possible: report the eager figure only
        graph_note = f"graph capture failed: {type(exc).__name__}: {exc}"[:200]
    best = graph_ms if graph_ms is not None else eager_ms
    ach = nbytes / (best * 1e-3) / 1e9
    out = {"dims": list(w["dims"]), "rank": w["rank"], "dtype": "f32",
           "cp_loss_fwd_bwd": {"ms_eager": eager_ms, "ms_graph": graph_ms, "repeats": reps, "note": graph_note,
                               "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                                            "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                                            "algorithmic_bytes": nbytes,
                                            "timing": "graph replay" if graph_ms is not None else "eager",
                                            "note": "N MTTKRP passes over the 108 MB tensor (1 forward, N-1 "
                                                    "backward; ||T||^2 passed in); Grams, V and the block "
                                                    "gradients are O(I r^2)"}}}
    iters = 200
    F = [torch.from_numpy(A).to(dev) for A in init]
    with torch.cuda.stream(stream):
        s = ntf.Solver(Td, F, ntf.Opts(method="pgd", inner_max=1, her=True, use_graph=True))
        s.prepare_graph(iters)
    ms = _timed(torch, stream, lambda: s.run(iters))
    rep = s.report(stream)
    s.close()
    out["pgd_her"] = {"iterations": iters, "iterations_per_s": iters / (ms * 1e-3), "rel_error": rep.rel_error,
                      "restarts": rep.restarts}
    del Td, leaves, tn
    _free(torch)
    return out


def wl_tucker(ntf, torch, dev, stream, peaks):
    """Tucker-format data (Appendix A) of the surveillance video's shape 153 x 238 x 14000:
    core 30^3 (the Tucker form of a noisy rank-20 CP tensor), CP rank 20, HER-HALS on F_t."""
    import synth
    dims, cdims, r = (153, 238, 14000), (30, 30, 30), 20
    G, U = synth.make_tucker(dims, cdims, seed=1300, rank=20, noise=0.05)
    X = ntf.Tucker(torch.from_numpy(G).to(dev), [torch.from_numpy(u).to(dev) for u in U])
    init = synth.make_init(dims, r, seed=42)
    init_d = [torch.from_numpy(A).to(dev) for A in init]
    out = {"dims": list(dims), "core": list(cdims), "rank": r, "dtype": "f32",
           "note": "expanded tensor (510M entries, 2 GB FP32) is never formed"}
    with torch.cuda.stream(stream):
        for n in range(3):
            ntf.tucker_mttkrp(X, init_d, n)
    out["mttkrp_us"] = [1e3 * _timed(torch, stream, lambda n=n: ntf.tucker_mttkrp(X, init_d, n), 20)
                        for n in range(3)]
    iters = 100
    F = [A.clone() for A in init_d]
    with torch.cuda.stream(stream):
        s = ntf.Solver.tucker(X, F, ntf.Opts(use_graph=True))
        s.run(5)
        s.prepare_graph(iters)
    ms = _timed(torch, stream, lambda: s.run(iters))
    rep = s.report(stream)
    s.close()
    out["her_hals"] = {"iterations_per_s": iters / (ms * 1e-3), "rel_error": rep.rel_error,
                       "bound": "latency (r_p x rank products and a 27k-entry core per MTTKRP)"}
    del X, init_d
    _free(torch)
    return out


def wl_streamed(ntf, torch, dev, stream, peaks, T, init):
    """The 500^3 FP32 tensor left in pinned host memory and streamed by slabs for every pass."""
    Th = torch.from_numpy(T).pin_memory()
    init_d = [torch.from_numpy(A).to(dev) for A in init]
    # the host-to-device copy rate of this machine, measured here on the same 500 MB (denominator)
    buf = torch.empty(T.shape, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        buf.copy_(Th, non_blocking=True)
    h2d_ms = _timed(torch, stream, lambda: buf.copy_(Th, non_blocking=True), 3)
    del buf
    _free(torch)
    h2d = T.nbytes / (h2d_ms * 1e-3) / 1e9
    with torch.cuda.stream(stream):
        for n in range(3):
            ntf.mttkrp_streamed(Th, init_d, n)
    # median of 5 single calls per mode: the host link's rate varies from call to call
    mt = [statistics.median(_timed(torch, stream, lambda n=n: ntf.mttkrp_streamed(Th, init_d, n), 1)
                            for _ in range(5)) for n in range(3)]
    mean_ms = sum(mt) / 3
    ach = T.nbytes / (mean_ms * 1e-3) / 1e9
    out = {"dims": list(T.shape), "dtype": "f32", "slab_rows": "default (64 MB slabs)",
           "mttkrp_ms": mt,
           "roofline": {"bound": "host-to-device link", "achieved": ach, "peak": h2d, "unit": "GB/s",
                        "frac": ach / h2d,
                        "peak_source": "measured in this run: one 500 MB pinned host-to-device copy (torch)",
                        "algorithmic_bytes_per_launch": T.nbytes}}
    iters = 5
    F = [A.clone() for A in init_d]
    with torch.cuda.stream(stream):
        s = ntf.Solver.streamed(Th, F, ntf.Opts())
        s.run(1)
    ms = _timed(torch, stream, lambda: s.run(iters))
    rep = s.report(stream)
    s.close()
    out["her_hals"] = {"iterations": iters, "iterations_per_s": iters / (ms * 1e-3), "rel_error": rep.rel_error}
    del Th, init_d
    _free(torch)
    return out


def wl_nesterov(ntf, torch, dev, stream, peaks):
    """The paper's gradient-method shape 150 x 1000 x 50, rank 10, 1% noise: AO-Nesterov50
    and HER-Nesterov50 (50 inner steps, stop rule 1e-2), 50 iterations each."""
    import synth
    import numpy as np
    dims, r = (150, 1000, 50), 10
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=1240)
    init = synth.make_init(dims, r, seed=42)
    # the library reads 16-byte rows: the 50-entry last mode is stored with pitch 52
    ld = -(-dims[-1] // 4) * 4
    host = np.zeros((dims[0] * dims[1], ld), dtype=np.float32)
    host[:, :dims[-1]] = T.reshape(-1, dims[-1])
    Td = torch.from_numpy(host).to(dev)
    iters = 50
    out = {"dims": list(dims), "rank": r, "dtype": "f32", "iterations": iters}
    for name, her in (("ao_nesterov50", False), ("her_nesterov50", True)):
        F = [torch.from_numpy(A).to(dev) for A in init]
        with torch.cuda.stream(stream):
            s = ntf.Solver(Td, F, ntf.Opts(her=her, method="nesterov", inner_max=50, inner_tol=1e-2,
                                           use_graph=True), dims=list(dims), ld=ld)
            s.prepare_graph(iters)
        ms = _timed(torch, stream, lambda: s.run(iters))
        rep = s.report(stream)
        s.close()
        out[name] = {"iterations_per_s": iters / (ms * 1e-3), "rel_error": rep.rel_error, "restarts": rep.restarts}
    del Td
    _free(torch)
    return out


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
    # at equal relative error: iterations and GPU seconds for each form to reach the same target
    target = 1.02 * quality["f32"]
    equal = {d: time_to_target(ntf, torch, Td, init_d, d, target, stream) for d in ("bf16", "f32")}
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
                    "abs_diff": abs(quality["bf16"] - quality["f32"]),
                    "rel_diff": abs(quality["bf16"] - quality["f32"]) / quality["f32"]},
        "equal_error": {"target_rel_error": target,
                        "target_rule": f"1.02 x the FP32 form's relative error after {args.quality_iters} iterations",
                        "bf16": equal["bf16"], "f32": equal["f32"],
                        "speedup_bf16_over_f32": (equal["f32"]["seconds"] / equal["bf16"]["seconds"]
                                                  if equal["bf16"]["reached"] and equal["f32"]["reached"] else None),
                        "timing": "chunks of 10 iterations replayed as a graph, CUDA events; the explicit error "
                                  "between chunks is not timed"},
    }
    for d in forms:
        g = forms[d]
        pl = g["mttkrp_ms"] / max(1, g["mttkrp_launches"])
        ach = g["mttkrp_bytes"] / (pl * 1e-3) / 1e9
        out["forms"][d] = {"iterations_per_s": rate[d], "ms_per_step": ms[d] / args.steps,
                           "mttkrp_gbs": ach, "mttkrp_frac_of_measured_hbm": ach / peaks["hbm_gbs"],
                           "mttkrp_frac_of_8tbs_nominal": ach / 8000.0, "mttkrp_avg_us": pl * 1e3,
                           "mttkrp_launches_timed": g["mttkrp_launches"], "timed_regions": g["repeats"],
                           "timed_s": g["timed_s"], "gpu_launches": g["launches"]}
    if rank == 0 and not args.no_extra:
        wl = {}
        wl["cube100_r10_illcond"] = wl_illcond(ntf, torch, dev, stream, peaks)
        wl["hyper80_r16_sparse30"] = wl_form_rates(ntf, torch, dev, stream, peaks, "hyper80_r16_sparse30")
        wl["cube300_r32"] = wl_autograd(ntf, torch, dev, stream, peaks)
        wl["nesterov_150x1000x50_r10"] = wl_nesterov(ntf, torch, dev, stream, peaks)
        wl["tucker_video153x238x14000_core30_r20"] = wl_tucker(ntf, torch, dev, stream, peaks)
        wl["streamed_cube500_r20_f32"] = wl_streamed(ntf, torch, dev, stream, peaks, T, init)
        ntf.device_status(stream)
        out["workloads"] = wl
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
    t0 = time.perf_counter()
    oracle.solve(Ts, init_s, 0)
    t_setup = time.perf_counter() - t0
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.solve(Ts, init_s, 1)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    step_s = statistics.mean(times)
    per_iter_full = max(step_s - t_setup, 1e-9) * scale
    value = 1.0 / per_iter_full
    sample = (f"each step: one HER-HALS iteration of the FP64 C oracle (one thread) on the leading {s}x500x500 "
              f"slab of the same tensor; value = that iteration's time without the oracle's one-time F-hat_0 "
              f"evaluation, scaled by {int(scale)} to the full 500^3 iteration (an extrapolation)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "dims": list(w["dims"]), "rank": w["rank"],
                   "timed_sample": f"{s}x500x500 slab per step (ms_per_step is the sample's measured wall time)",
                   "value_basis": f"extrapolated: sample iteration time x {int(scale)}"},
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
    ap.add_argument("--no-extra", action="store_true", help="only the 500^3 headline workload (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not args.skip_cpu:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
