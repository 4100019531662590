#!/usr/bin/env python
"""Benchmark of the DID sweep on one GB300 (or N independent replicas).

A step is one sweep: for k = 1..K the b_k update (grid reduction of R c_k^T),
the c_k update fused with the residual write-back, the objective of the
sweep, and -- at the workload's cadence -- the dense refresh R = X - B C.

Prints one JSON line (rank 0).  `value` is sweeps/s summed over ranks, timed
with CUDA events on the library's stream between barriers; `roofline` is the
sweep kernel's algorithmic HBM bytes over its own CUDA-event time against the
measured copy bandwidth; `e2e` is the same metric through the public API from
pinned host memory (X uploaded, factors read back, inside the timed region);
`cpu_baseline` is the FP64 oracle on one host core over a column slice of the
same workload, scaled linearly in N (sweep cost is O(MNK)).

`--impl reference` times the oracle itself as the reference arm.
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DID sweeps/s + HBM GB/s (BF16-R vs FP32 plain); serve solves/s, p50/p99 ms"

# Workloads (synthetic, seeded; shapes of the paper's experiments).
WORKLOADS = {
    "planted_exp_5000x200000_k50": dict(M=5000, N=200000, K=50, gen="planted", coords=1, zero_frac=0.3,
                                        sigma=0.05, salt_frac=0.0, refresh_every=10, init_scale=False),
    "image_like_784x70000_k16": dict(M=784, N=70000, K=16, gen="image", refresh_every=0, init_scale=True),
    "salt_10000x500000_k100": dict(M=10000, N=500000, K=100, gen="planted", coords=0, zero_frac=0.0,
                                   sigma=0.0, salt_frac=0.01, refresh_every=5, init_scale=False),
    "planted_uniform_200x1000_k10": dict(M=200, N=1000, K=10, gen="planted", coords=0, zero_frac=0.0,
                                         sigma=0.01, salt_frac=0.0, refresh_every=0, init_scale=False),
}
DEFAULT_WORKLOAD = "planted_exp_5000x200000_k50"
# Block orders (did_options.order): per-k interleaved, per-k C-first, batched Algorithm 3.
ORDERS = {"interleaved": 0, "did": 1, "did_batched": 2}
# float32 FMA peak of the SIMT pipes: 152 SMs x 128 lanes x 2 flops x 2070 MHz (maximum SM clock)
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Column slice of each workload for the oracle timing (about 10-20 s of CPU work).
CPU_SAMPLE_COLS = {"planted_exp_5000x200000_k50": 1000, "image_like_784x70000_k16": 4000,
                   "salt_10000x500000_k100": 250, "planted_uniform_200x1000_k10": 1000}
CPU_SAMPLE_SWEEPS = 3

SWEEP_SOURCES = ["paper_1802_08938_gb300/csrc/did_sweep.cu", "paper_1802_08938_gb300/csrc/did_sweep_kernel.cuh",
                 "paper_1802_08938_gb300/csrc/did_internal.cuh"]


def sweep_source_hash():
    h = hashlib.sha256()
    for p in SWEEP_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(workload, precision):
    """DRAM bytes per sweep-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "sweep_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get("%s/%s" % (workload, precision))
    if not e or e.get("source_hash") != sweep_source_hash():
        return None
    return e.get("bytes_per_sweep")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------- CPU oracle
def cpu_sample(workload, cols, sweeps, threads=1):
    """Time `sweeps` oracle sweeps on the first `cols` columns (runs in a child
    process with `threads` BLAS threads).  Returns seconds per sweep of the slice."""
    t = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._cpu_sample_child(%r, %d, %d)))" % (ROOT, workload, cols, sweeps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("cpu sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_sample_child(workload, cols, sweeps):
    from oracle import did_oracle as O
    from synth import workloads as SW
    w = WORKLOADS[workload]
    M, K = w["M"], w["K"]
    if w["gen"] == "image":
        X = SW.image_like(M, cols, 0)
    else:
        X, _, _ = SW.planted(M, cols, K, 0, coords="exp" if w["coords"] == 1 else "uniform",
                             zero_frac=w["zero_frac"], sigma=w["sigma"], salt_frac=w["salt_frac"])
    B, C = SW.init_factors(M, cols, K, 0)
    if w["init_scale"]:
        B, C = O.init_scale(X, B, C)
    R = O.residual(X, B, C)
    times = []
    for _ in range(sweeps):
        t = time.perf_counter()
        B, C, R, _ = O.sweep_hals(X, B, C, R)
        times.append(time.perf_counter() - t)
    return {"sec_per_sweep": sum(times) / len(times), "times": times}


def cpu_baseline(workload):
    """The FP64 oracle as it stands on the host cores: one thread (the
    baseline), and all cores (BLAS threads; the oracle's elementwise NumPy
    steps stay single-threaded)."""
    w = WORKLOADS[workload]
    cols = min(CPU_SAMPLE_COLS[workload], w["N"])
    r = cpu_sample(workload, cols, CPU_SAMPLE_SWEEPS)
    sweeps_per_s = (1.0 / r["sec_per_sweep"]) * cols / w["N"]
    out = {"value": sweeps_per_s, "unit": "sweeps/s", "cores": 1, "kind": "oracle",
           "sample": "%d FP64 oracle sweeps (NumPy, 1 thread) on the first %d of %d columns (M=%d, K=%d), "
                     "scaled linearly in N" % (CPU_SAMPLE_SWEEPS, cols, w["N"], w["M"], w["K"])}
    ncpu = os.cpu_count() or 1
    if ncpu > 1:
        rm = cpu_sample(workload, cols, CPU_SAMPLE_SWEEPS, threads=ncpu)
        out["all_cores"] = {"value": (1.0 / rm["sec_per_sweep"]) * cols / w["N"], "unit": "sweeps/s",
                            "cores": ncpu, "sample": "same slice, %d BLAS threads" % ncpu}
    return out


# ------------------------------------------------------------------ main
def serve_bench(did, n_req, rate, precision, budget_gb=120.0, max_slots=64, round_sweeps=4):
    """Submit the first n_req requests of the serving stream at their Poisson
    arrival times; return throughput and latency percentiles."""
    from synth import workloads as SW
    shapes = [SW.request_shape(0, r) for r in range(n_req)]
    arrivals = SW.arrival_times(0, n_req, rate)
    srv = did.Server(int(budget_gb * (1 << 30)), precision=precision, max_slots=max_slots,
                     round_sweeps=round_sweeps)
    tickets = []
    t0 = time.perf_counter()
    for r, (m, n, k) in enumerate(shapes):
        d = t0 + arrivals[r] - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets.append(srv.submit(m, n, k, SW.request_seed(0, r), max_iter=300, tol=1e-4))
    results = [srv.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    iters = [r["iters"] for r in results]
    work = sum(2.0 * m * n * k * (4 if precision == did.DID_FP32 else 2) * it
               for (m, n, k), it in zip(shapes, iters))
    return {"requests": n_req, "rate_req_per_s": rate, "precision": "fp32" if precision == did.DID_FP32 else "bf16r",
            "completed": st["completed"], "failed": st["failed"], "solves_per_s": st["solves_per_s"],
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "wall_s": wall, "peak_active": st["peak_active"],
            "peak_gb": st["peak_bytes"] / 1e9, "rounds": st["rounds"], "busy_s": st["busy_s"],
            "mean_sweeps": float(sum(iters)) / len(iters), "sweep_GBps": work / st["busy_s"] / 1e9 if st["busy_s"] else None,
            "note": "saturated: offered work exceeds one GPU at this rate" if rate >= 50 else ""}


def workload_run(did, name, precision, sweeps, warmup, stream, tol=0.0, max_sweeps=None):
    """One context on a named workload (device-generated X, seed 0): warm-up
    sweeps, then `sweeps` timed sweeps (or, with tol > 0, did_factor up to
    max_sweeps under the relative-change rule).  Returns sweeps/s over the
    timed region (CUDA events on the library's stream), the sweep kernel's
    roofline on the bytes it moves, the refreshes, and f(B, C)."""
    import torch
    w = WORKLOADS[name]
    M, N, K = w["M"], w["N"], w["K"]
    prec = did.DID_BF16R if precision == "bf16r" else did.DID_FP32
    s_bytes = 2 if prec == did.DID_BF16R else 4
    X = torch.empty((N, M), dtype=torch.float32, device="cuda")
    if w["gen"] == "image":
        did.did_generate_image(X, M, N, 0, 0.8, stream=stream)
    else:
        did.did_generate_planted(X, M, N, K, 0, coords=w["coords"], zero_frac=w["zero_frac"], sigma=w["sigma"],
                                 salt_frac=w["salt_frac"], salt_value=5.0, stream=stream)
    c = did.Context(X, M, N, K, seed=0, precision=prec, refresh_every=w["refresh_every"],
                    init_scale=w["init_scale"], stream=stream)
    del X
    for _ in range(warmup):
        c.sweep(1)
    i0 = c.info()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if tol > 0:
        done, _ = c.factor(max_sweeps, tol)
    else:
        c.sweep(sweeps)
        done = sweeps
    e1.record(stream)
    torch.cuda.synchronize()
    i1 = c.info()
    ms = e0.elapsed_time(e1)
    kms = i1["sweep_kernel_ms"] - i0["sweep_kernel_ms"]
    passes = sweep_passes(K, i1["lazy_writeback"])
    alg = done * float(passes) * M * N * s_bytes + (i1["prologue_launches"] - i0["prologue_launches"]) * M * N * s_bytes
    peak, _ = measured_peaks()
    f = c.objective()
    trace = c.trace()
    c.close()
    return {"workload": name, "precision": precision, "sweeps": int(done), "warmup": warmup,
            "value": done / (ms / 1000.0), "unit": "sweeps/s", "ms_per_sweep": ms / max(1, done),
            "roofline_frac": alg / (kms / 1e3) / 1e9 / peak if kms > 0 else None,
            "alg_bytes_per_sweep": float(passes) * M * N * s_bytes, "writeback": "deferred" if i1["lazy_writeback"] else "eager",
            "refreshes": int(i1["refreshes"] - i0["refreshes"]),
            "refresh_kind": ("tcgen05" if i1["tc_refreshes"] > i0["tc_refreshes"] else "SIMT") if i1["refreshes"] > i0["refreshes"] else None,
            "objective_fBC": f, "trace_last": float(trace[-1]),
            "gpu_launches": int((i1["sweep_launches"] - i0["sweep_launches"]) + (i1["dense_launches"] - i0["dense_launches"])
                                + 3 * (i1["tc_refreshes"] - i0["tc_refreshes"]))}


def precision_pair(did, name, sweeps, warmup, stream, tol=0.0, max_sweeps=None):
    """FP32 and BF16-R on the same workload and seed: both throughputs, their
    ratio, and how far apart the factorisations' objectives f(B, C) end."""
    f32 = workload_run(did, name, "fp32", sweeps, warmup, stream, tol, max_sweeps)
    # With a stopping rule the BF16-R arm runs the sweeps the float32 arm took:
    # its monitored objective carries the residual's rounding (about 1e-5
    # relative change per sweep), so the same rule would run it to max_sweeps.
    b16 = workload_run(did, name, "bf16r", f32["sweeps"] if tol > 0 else sweeps, warmup, stream)
    note = "same seed and start; the float32 line is the library's default for this shape (%s write-back)" % (
        f32["writeback"])
    if tol > 0:
        note += "; float32 stops at relative change < %g (max %d sweeps), BF16-R runs the same sweep count" % (
            tol, max_sweeps)
    return {"workload": name, "fp32": f32, "bf16r": b16, "ratio_bf16r_vs_fp32": b16["value"] / f32["value"],
            "objective_rel_diff": abs(b16["objective_fBC"] - f32["objective_fBC"]) / f32["objective_fBC"],
            "note": note}


def batched_flops(M, N, K):
    """Algorithmic float32 flops of one batched sweep of Algorithm 3 with a
    pending correction: g = B^T R (2KMN), R -= [D B][C_old; dl] (4KMN),
    W = R C^T (2KMN), the K x K products and the per-column / per-row solves."""
    return 8.0 * K * M * N + 2.0 * K * K * N * 2 + 2.0 * (2 * K) ** 2 * M + 2.0 * K * K * (N + M)


def order_bench(did, X, M, N, K, w, seed, stream, order, steps, warmup, flags=0, inner=(1, 1)):
    """Sweeps/s of one block order on the same workload, seed and start."""
    import torch
    c = did.Context(X, M, N, K, seed=seed, precision=did.DID_FP32, order=ORDERS[order],
                    refresh_every=w["refresh_every"], init_scale=w["init_scale"], stream=stream, flags=flags,
                    inner_c=inner[0], inner_b=inner[1])
    for _ in range(warmup):
        c.sweep(1)
    i0 = c.info()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        c.sweep(1)
    e1.record(stream)
    torch.cuda.synchronize()
    i1 = c.info()
    ms = e0.elapsed_time(e1)
    f = c.objective()
    trace = c.trace()
    c.close()
    out = {"order": order, "writeback": "eager" if flags & did.DID_FLAG_EAGER_WRITEBACK else "deferred",
           "inner": list(inner), "trace": [float(v) for v in trace],
           "value": steps / (ms / 1000.0), "unit": "sweeps/s", "ms_per_sweep": ms / steps,
           "objective_after": f, "sweeps": warmup + steps,
           "sweep_ms": (i1["sweep_kernel_ms"] - i0["sweep_kernel_ms"]) / steps}
    if order == "did_batched":
        out["roofline"] = batched_roofline(M, N, K, out["sweep_ms"])
    return out


def batched_roofline(M, N, K, ms_per_sweep):
    """Whole-sweep roofline of the batched order: its three passes of R (the g
    pass reads R, the update pass reads and writes it) against the measured
    copy bandwidth, with the tensor-core work beside it (six bfloat16 products
    per float32 product, against the measured sustained bfloat16 peak)."""
    peak, kind = measured_peaks()
    alg = 3.0 * M * N * 4
    gbs = alg / (ms_per_sweep / 1e3) / 1e9
    fl = batched_flops(M, N, K)
    tpeak = 1700.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            tpeak = float(json.load(f)["bf16_tflops_sustained"])
    tf6 = 6 * fl / (ms_per_sweep / 1e3) / 1e12
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_kind": peak_kind_note(kind), "alg_bytes_per_sweep": alg,
            "passes_of_R": 3, "tensor_tflops_bf16x6": tf6, "tensor_frac_of_sustained_bf16": tf6 / tpeak,
            "flops_per_sweep_f32": fl,
            "note": "whole sweep: g pass (reads R), update pass (reads and writes R), solves and the B step"}


def peak_kind_note(kind):
    return kind


def sweep_passes(K, lazy):
    """Passes over R per sweep of the interleaved kernel: a read and a write per
    k, less one write for each deferred k (pairs (k, k+1) share a write)."""
    return 2 * K - (K // 2 if lazy else 0)


def max_over_ranks(x, ws):
    """The largest value of x over the job's ranks (x itself with one rank).
    The reduction tensor lives where the process group's backend wants it:
    on the rank's GPU for NCCL, in host memory for gloo."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, steps, max_ms):
    """Whole-job throughput: units every rank processed over the slowest rank's time."""
    return ws * steps / (max_ms / 1000.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    cols = min(CPU_SAMPLE_COLS[args.workload], w["N"])
    r = cpu_sample(args.workload, cols, args.warmup + args.steps)
    times = r["times"][args.warmup:]
    sec = sum(times) / len(times)
    value = (1.0 / sec) * cols / w["N"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "ms_per_step_kind": "extrapolated: measured on a %d-column slice, scaled linearly in N to %d columns"
                                % (cols, w["N"]),
            "ms_per_step_measured_slice": 1000.0 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "M": w["M"], "N": w["N"], "K": w["K"],
                                            "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: one FP64 oracle sweep (NumPy, 1 thread) on the first %d of %d "
                                       "columns, scaled linearly in N" % (cols, w["N"])},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16r"])
    ap.add_argument("--shape", default=None,
                    help="M,N,K override of the workload's sizes (same generator); for profiling small cases")
    ap.add_argument("--order", default="interleaved", choices=sorted(ORDERS),
                    help="block order of the main line: per-k interleaved (Section 4.1), per-k C-first "
                         "(Algorithm 2), or the batched form of Algorithm 3")
    ap.add_argument("--eager", action="store_true",
                    help="interleaved order: write R after every k (no deferred write-back)")
    ap.add_argument("--no-orders", action="store_true",
                    help="skip the C-first and batched Algorithm 3 measurements on the same workload")
    ap.add_argument("--phases", action="store_true",
                    help="also report the per-k phase split of the last timed sweep (globaltimer stamps)")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-R measurement on the same workload")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the precision workload (10000x500000, K=100: FP32 vs BF16-R, 50 sweeps each) and "
                         "the image-like workload (784x70000, K=16) lines")
    ap.add_argument("--precision-sweeps", type=int, default=50,
                    help="timed sweeps of each arm on the precision workload")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=128,
                    help="requests of the serving stream to run (4096 in the full stream)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving measurement")
    ap.add_argument("--serve-sustain-rate", type=float, default=1.5,
                    help="arrival rate (req/s) of the second, sustainable serving measurement (FP32); 0 = skip")
    ap.add_argument("--serve-sustain-requests", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did

    if args.serve_only:
        out = [serve_bench(did, args.serve_requests, args.serve_rate, p)
               for p in ((did.DID_BF16R,) if args.precision == "bf16r" else (did.DID_FP32,))]
        if rank == 0:
            print(json.dumps({"metric": METRIC, "serving": out}), flush=True)
        return 0

    w = dict(WORKLOADS[args.workload])
    if args.shape:
        w["M"], w["N"], w["K"] = (int(v) for v in args.shape.split(","))
    M, N, K = w["M"], w["N"], w["K"]
    prec = did.DID_BF16R if args.precision == "bf16r" else did.DID_FP32
    s_bytes = 2 if prec == did.DID_BF16R else 4
    seed = rank
    stream = torch.cuda.current_stream()

    X = torch.empty((N, M), dtype=torch.float32, device="cuda")   # M x N column-major
    if w["gen"] == "image":
        did.did_generate_image(X, M, N, seed, 0.8, stream=stream)
    else:
        did.did_generate_planted(X, M, N, K, seed, coords=w["coords"], zero_frac=w["zero_frac"],
                                 sigma=w["sigma"], salt_frac=w["salt_frac"], salt_value=5.0, stream=stream)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    if args.order == "did_batched" and prec != did.DID_FP32:
        ap.error("the batched order runs in float32 only")
    flags = did.DID_FLAG_PHASE_TIMES if args.phases else 0
    if args.eager:
        flags |= did.DID_FLAG_EAGER_WRITEBACK
    ctx = did.Context(X, M, N, K, seed=seed, precision=prec, order=ORDERS[args.order],
                      refresh_every=w["refresh_every"], init_scale=w["init_scale"], stream=stream, flags=flags)
    for _ in range(args.warmup):
        ctx.sweep(1)
    info0 = ctx.info()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    step_ms = []
    last = info0["sweep_kernel_ms"] + info0["dense_kernel_ms"] + info0["tc_refresh_ms"]
    for _ in range(args.steps):
        ctx.sweep(1)
        cur = ctx.info()
        now = cur["sweep_kernel_ms"] + cur["dense_kernel_ms"] + cur["tc_refresh_ms"]
        step_ms.append(round(now - last, 3))
        last = now
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    info1 = ctx.info()
    phases = None
    if args.phases:
        t = ctx.phase_times().astype("int64")
        if len(t):
            d = lambda a, b: float(((t[:, b] - t[:, a]) / 1e3).mean())
            phases = {"us_per_k": {"b_reduce+wait1": d(0, 1), "c_pass": d(1, 2), "wait2": d(2, 3),
                                   "gap_to_next_k": float((t[1:, 0] - t[:-1, 3]).mean() / 1e3) if len(t) > 1 else 0.0},
                      "k_steps": int(len(t))}
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws)
    value = job_value(ws, args.steps, ms)

    # Roofline of the sweep kernel: algorithmic bytes / its own event time.
    launches = info1["sweep_launches"] - info0["sweep_launches"]
    prologues = info1["prologue_launches"] - info0["prologue_launches"]
    kms = info1["sweep_kernel_ms"] - info0["sweep_kernel_ms"]
    passes = sweep_passes(K, info1["lazy_writeback"]) if args.order == "interleaved" else 2 * K
    alg_bytes = args.steps * float(passes) * M * N * s_bytes + prologues * 1.0 * M * N * s_bytes
    achieved = alg_bytes / (kms / 1000.0) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic(args.workload, args.precision)
    dense_launches = info1["dense_launches"] - info0["dense_launches"]
    tc_launches = info1["tc_refreshes"] - info0["tc_refreshes"]
    # each tensor-core refresh is three launches: two operand splits and the GEMM
    gpu_launches = launches + dense_launches + 3 * tc_launches   # the timed region of the line
    other_launches = 0                                            # the other measurements' timed regions
    refresh = None
    nref = dense_launches + tc_launches
    if nref:
        rms = (info1["dense_kernel_ms"] - info0["dense_kernel_ms"] + info1["tc_refresh_ms"] - info0["tc_refresh_ms"]) / nref
        rbytes = M * N * (4 + s_bytes)
        kind = ("tcgen05 BF16x3" if prec == did.DID_BF16R else "tcgen05 BF16x6") if tc_launches else "SIMT FP32"
        refresh = {"kind": kind, "launches": int(nref),
                   "ms_per_refresh": rms, "alg_bytes": rbytes, "GBps": rbytes / (rms / 1e3) / 1e9,
                   "tflops": 2.0 * M * N * K * (3 if tc_launches else 1) / (rms / 1e3) / 1e12}
    ctx.close()
    del ctx

    bf16 = None
    if not args.no_bf16 and prec == did.DID_FP32:
        c16 = did.Context(X, M, N, K, seed=seed, precision=did.DID_BF16R, refresh_every=w["refresh_every"],
                          init_scale=w["init_scale"], stream=stream)
        for _ in range(args.warmup):
            c16.sweep(1)
        i0 = c16.info()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            c16.sweep(1)
        e1.record(stream)
        torch.cuda.synchronize()
        i1 = c16.info()
        ms16 = e0.elapsed_time(e1)
        kms16 = i1["sweep_kernel_ms"] - i0["sweep_kernel_ms"]
        ab16 = (args.steps * float(sweep_passes(K, i1["lazy_writeback"])) * M * N * 2
                + (i1["prologue_launches"] - i0["prologue_launches"]) * M * N * 2.0)
        f16 = c16.objective()
        c16.close()
        v16 = ws * args.steps / (ms16 / 1000.0)
        bf16 = {"value": v16, "unit": "sweeps/s", "ratio_vs_fp32": v16 / value, "lazy": int(i1["lazy_writeback"]),
                "roofline_frac": ab16 / (kms16 / 1e3) / 1e9 / peak,
                "tc_refreshes": int(i1["tc_refreshes"] - i0["tc_refreshes"]),
                "objective_after": f16,
                "note": "same workload and seed, R stored in bfloat16, tensor-core BF16x3 refresh"}
        other_launches += args.steps + 3 * int(i1["tc_refreshes"] - i0["tc_refreshes"])

    orders = None
    if not args.no_orders and prec == did.DID_FP32 and args.order == "interleaved":
        batched_ok = K <= 64
        runs = [("interleaved", did.DID_FLAG_EAGER_WRITEBACK, (1, 1)), ("did", 0, (1, 1))]
        if batched_ok:
            runs += [("did_batched", 0, (1, 1)), ("did_batched", 0, (2, 2)), ("did_batched", 0, (4, 4))]
        orders = [order_bench(did, X, M, N, K, w, seed, stream, o, args.steps, args.warmup, f, r)
                  for o, f, r in runs]
        # inner repeats: sweeps (and time) to reach the objective that plain batched sweeps reach
        target = orders[2]["trace"][-1] if batched_ok else orders[1]["trace"][-1]
        for o in orders:
            o["ratio_vs_main"] = o["value"] / value
            hit = [i for i, v in enumerate(o.pop("trace")) if v <= target]
            o["sweeps_to_plain_final"] = hit[0] if hit else None
            o["ms_to_plain_final"] = hit[0] * o["ms_per_sweep"] if hit else None
        # the per-k orders launch one sweep kernel per sweep; the batched order 8 kernels per sweep
        other_launches += 2 * args.steps + (3 * 8 * args.steps if batched_ok else 0)

    e2e = None
    if not args.no_e2e:
        Xh = torch.empty((N, M), dtype=torch.float32, pin_memory=True)
        Xh.copy_(X)
        del X
        torch.cuda.empty_cache()
        Bh = torch.empty((K, M), dtype=torch.float32, pin_memory=True)
        Ch = torch.empty((K, N), dtype=torch.float32, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = did.Context(Xh, M, N, K, seed=seed, precision=prec, refresh_every=w["refresh_every"],
                         init_scale=w["init_scale"], stream=stream)
        c2.sweep(args.steps)
        did.did_get_factors(c2.h, Bh, Ch)
        t1 = time.perf_counter()
        c2.close()
        e_sec = max_over_ranks(t1 - t0, ws)
        e2e = {"value": ws * args.steps / e_sec, "unit": "sweeps/s",
               "h2d_bytes_per_step": int(M * N * 4 / args.steps),
               "d2h_bytes_per_step": int((M * K + K * N) * 4 / args.steps),
               "note": "one job per run: did_create from pinned host X, %d sweeps, factors read back" % args.steps}
    else:
        del X

    workloads = None
    if not args.no_workloads and not args.shape and args.order == "interleaved" and ws == 1:
        # the configuration the BF16-R target is quoted on, and the MNIST-shaped one
        workloads = {
            "salt_10000x500000_k100": precision_pair(did, "salt_10000x500000_k100", args.precision_sweeps, 3,
                                                     stream),
            "image_like_784x70000_k16": precision_pair(did, "image_like_784x70000_k16", 0, 3, stream,
                                                       tol=1e-5, max_sweeps=200),
        }
        other_launches += sum(v[a]["gpu_launches"] for v in workloads.values() for a in ("fp32", "bf16r"))
        if bf16 is not None:
            # the BF16-R ratio on the configuration its target is quoted on,
            # beside the same-workload ratio above
            pw = workloads["salt_10000x500000_k100"]
            bf16["precision_workload"] = {
                "workload": pw["workload"], "sweeps": pw["fp32"]["sweeps"],
                "fp32_sweeps_per_s": pw["fp32"]["value"], "bf16r_sweeps_per_s": pw["bf16r"]["value"],
                "ratio_vs_fp32": pw["ratio_bf16r_vs_fp32"], "objective_rel_diff": pw["objective_rel_diff"],
                "note": "same seed and start; the float32 line is the library's default for this shape"}

    serving = None
    if not args.no_serve and not args.shape:
        serving = [serve_bench(did, args.serve_requests, args.serve_rate, did.DID_FP32),
                   serve_bench(did, args.serve_requests, args.serve_rate, did.DID_BF16R)]
        if args.serve_sustain_rate > 0:
            # below the measured capacity (~2.7 solves/s of 300-sweep requests):
            # latencies are then service times plus a short queue
            serving.append(serve_bench(did, args.serve_sustain_requests, args.serve_sustain_rate, did.DID_FP32))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.shape:
        cpu = cpu_baseline(args.workload)

    if args.order == "did_batched":
        roofline = batched_roofline(M, N, K, kms / max(1, args.steps))
        roofline.update({"traffic": None, "kernel": "batched sweep", "kernel_ms_per_sweep": kms / max(1, args.steps)})
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic if args.order == "interleaved" else None,
                    "kernel": "sweep_kernel", "peak_kind": peak_kind,
                    "alg_bytes_per_sweep": float(passes) * M * N * s_bytes,
                    # the survey's per-sweep figure, one read and one write of R per k; the
                    # deferred write-back moves fewer bytes, and frac above uses the bytes it moves
                    "alg_bytes_per_sweep_2KMNs": 2.0 * K * M * N * s_bytes,
                    "frac_on_2KMNs": (2.0 * K * M * N * s_bytes * args.steps / (kms / 1000.0) / 1e9) / peak,
                    "bytes_note": ("frac counts the %d passes of R a sweep moves (%s write-back); on 2K = %d "
                                   "passes the same kernel time gives frac_on_2KMNs"
                                   % (passes, "deferred" if info1["lazy_writeback"] else "eager", 2 * K)),
                    "lazy_writeback": int(info1["lazy_writeback"]), "ring_stages": int(info1["ring_stages"]),
                    "kernel_ms_per_sweep": kms / max(1, args.steps)}

    if bf16 is not None and orders:
        eager32 = [o for o in orders if o["order"] == "interleaved" and o["writeback"] == "eager"]
        if eager32:
            bf16["ratio_vs_fp32_eager"] = bf16["value"] / eager32[0]["value"]
        bf16["writeback"] = "deferred" if bf16.pop("lazy", 0) else "eager"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == did.DID_FP32 else "bf16-storage/f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "M": M, "N": N, "K": K, "precision": args.precision,
                       "order": args.order,
                       "refresh_every": w["refresh_every"], "init_scale": w["init_scale"],
                       "l2": "inputs larger than L2 (R is %.1f GB)" % (M * N * s_bytes / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": int(gpu_launches),
            "gpu_launches_other_measurements": int(other_launches),
            "step_kernel_ms": step_ms,
            "refresh": refresh,
            "bf16r": bf16,
            "workloads": workloads,
            "orders": orders,
            "serving": serving,
            "phases": phases,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
