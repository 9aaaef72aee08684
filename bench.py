#!/usr/bin/env python
"""Throughput of the TLR quasi-Monte Carlo integrand, in QMC sample-dimensions per second.

Workload (one "step" = one full solve): Student-t nu = 7 probability in
n = 65,536 dimensions; exponential covariance (beta = 0.1) on a 256 x 256
jittered grid of the unit square; a = -inf, b_i ~ N(1, 0.5^2); tile m = 512,
ACA tolerance 1e-4, ranks <= 64; 20 random shifts x 5,000 Richtmyer points.
The factor is built once on the GPU (float64) before timing; the timed step
is tlrmvn_prob_device with the limits already resident in HBM.

Output: one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
METRIC = "MVN/MVT QMC sample-dims/sec at n=65,536 vs FP64 path; p50/p99 solve latency"
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel from one
# ncu capture, divided by the sample-dimensions the captured launch processed,
# with the digest of the sources the kernel is built from (build.source_digest
# of `files`).  A figure is reported, scaled to this run's launches, only while
# those sources are unchanged (otherwise null); the summaries with the capture
# commands are under profiles/.
TRAFFIC = {
    "k_sweep_tc": {"bytes_per_sample_dim": 20.7063,
                   "capture": "profiles/k_sweep_tc_n16384.md",
                   "files": ["paper_2003_11183_gb300/csrc/sweep_tc.cuh",
                             "paper_2003_11183_gb300/csrc/sweep.cuh",
                             "paper_2003_11183_gb300/csrc/sov_device.cuh",
                             "paper_2003_11183_gb300/csrc/tcgen05.cuh",
                             "paper_2003_11183_gb300/csrc/common.cuh",
                             "include/tlrmvn.h"],
                   "sources": "2091dce6350b70d328d34a085ab1b5bd34780cc9845b0990a2bf7b7e42bc9294"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=list(PRECISIONS),
                    help="bf16: float32 sweep with bf16 tensor-core shifts (the workload's precision)")
    ap.add_argument("--workload", type=int, default=3)
    ap.add_argument("--points", type=int, default=0, help="override points per shift (0 = workload's)")
    ap.add_argument("--shifts", type=int, default=0, help="override the number of shifts (0 = workload's)")
    ap.add_argument("--tile", type=int, default=0, help="override the workload's tile size (experiments only)")
    ap.add_argument("--n-side", type=int, default=0,
                    help="grid side of a smaller problem of the same family (profiling captures only)")
    ap.add_argument("--reorder", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="override the workload's preconditioner (-1 = workload's; 0 none, 1 Algorithm 4, 2 Algorithm 5)")
    ap.add_argument("--schur", default="exact", choices=["exact", "tlr"],
                    help="factor arithmetic: exact Schur complement or TLR arithmetic with truncated updates")
    ap.add_argument("--no-baselines", action="store_true", help="skip FP64-path and CPU-oracle legs")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default launch choices (profiling captures: fewer launches)")
    ap.add_argument("--sample-chunk", type=int, default=0,
                    help="samples per chunk of the solve (0 = the library's choice: all that fit)")
    ap.add_argument("--count", type=int, default=256, help="problems of the batched workload (--workload 4)")
    ap.add_argument("--requests", type=int, default=0,
                    help="requests of the serving leg (0: 160 in the default run, 400 with --workload 5)")
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals per second (--workload 5; 0 = measured)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


ORACLE_WORKER = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import synth
from oracle import sov
from tests.helpers import to_oracle_factor
from paper_2003_11183_gb300.api import parse_export
w = synth.workload({wl})
F = to_oracle_factor(parse_export(open({path!r}, 'rb').read()))
print("ready", flush=True)
for r, first in enumerate({firsts!r}):
    go = {go!r} + "." + str(r)
    while not os.path.exists(go):
        time.sleep(0.005)
    sel = np.arange(first, first + {count}, dtype=np.int64)
    t0 = time.time()
    out = sov.solve(F, w.a, w.b, w.nu, w.shifts, w.n_points, samples=sel, chunk={count})
    t1 = time.time()
    print(json.dumps({{"t0": t0, "t1": t1, "per_sample": out["per_sample"].tolist()}}), flush=True)
"""


class OraclePool:
    """The CPU oracle (oracle/, plain float64 NumPy, as it stands) run by `procs`
    single-threaded worker processes, each evaluating its own `count` lattice points
    of the workload per round on the same factor; a round is timed from the first
    worker's start to the last one's end (workers are loaded before the first round)."""

    def __init__(self, buf_path: str, wl: int, procs: int, count: int, rounds_firsts):
        self.procs, self.count = procs, count
        self.go = os.path.join(tempfile.gettempdir(), f"tlrmvn_oracle_go_{os.getpid()}_{id(self)}")
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        self.ps = []
        for p in range(procs):
            firsts = [f + p * count for f in rounds_firsts]
            code = ORACLE_WORKER.format(root=ROOT, wl=wl, path=buf_path, firsts=firsts, go=self.go, count=count)
            self.ps.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, text=True, env=env))
        for p in self.ps:
            line = p.stdout.readline().strip()
            if line != "ready":
                raise RuntimeError("oracle worker failed to start")
        self.round = 0

    def run_round(self) -> dict:
        """One round: seconds (wall, all workers), samples, per-sample values (worker order)."""
        open(f"{self.go}.{self.round}", "w").close()
        res = [json.loads(p.stdout.readline()) for p in self.ps]
        os.unlink(f"{self.go}.{self.round}")
        self.round += 1
        return {"seconds": max(r["t1"] for r in res) - min(r["t0"] for r in res), "samples": self.procs * self.count,
                "per_sample": [v for r in res for v in r["per_sample"]]}

    def close(self):
        for p in self.ps:
            try:
                p.wait(timeout=60)
            except Exception:
                p.kill()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def build_factor(tl, w):
    t0 = time.perf_counter()
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, w.max_rank, w.reorder,
                                schur=getattr(w, "schur", 0))
    return F, time.perf_counter() - t0


ORACLE_POINTS = 32  # lattice points per worker and round of the CPU oracle


def run_reference(args):
    ws, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    w = load_workload(args)
    torch.cuda.set_device(0)
    F, fs = build_factor(tl, w)
    path = os.path.join(tempfile.gettempdir(), f"tlrmvn_factor_{os.getpid()}.bin")
    with open(path, "wb") as fh:
        fh.write(tl.tlrmvn_factor_export(F))
    cores = host_cores()
    rounds = args.warmup + args.steps
    # round r takes the points of shift (r mod M): sample indices s*N + k - 1
    firsts = [(r % w.n_shifts) * w.n_points for r in range(rounds)]
    pool = OraclePool(path, args.workload, cores, ORACLE_POINTS, firsts)
    times = []
    for r in range(rounds):
        res = pool.run_round()
        if r >= args.warmup:
            times.append(res["seconds"])
    pool.close()
    os.unlink(path)
    per = statistics.mean(times)
    value = w.n * cores * ORACLE_POINTS / per
    sample = (f"{cores} worker processes x {ORACLE_POINTS} lattice points of one shift of the same workload per "
              f"step ({cores * ORACLE_POINTS} samples, all {w.n} dimensions), same factor")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sample-dims/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(bench_config(tl, F, w, args.precision), sample_chunk=args.sample_chunk or "all"),
            "cpu_baseline": {"value": value, "unit": "sample-dims/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "sample-dims/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "notes": "factor built once by the library's GPU factorisation (setup, untimed); timed step is the "
                     "oracle's TLR integrand alone, single-threaded BLAS in each worker"}
    print(json.dumps(line), flush=True)
    return 0


def load_workload(args):
    """The synthetic workload of --workload, with --n-side / --points / --shifts applied."""
    import synth
    w = synth.workload(args.workload, n_side=args.n_side or None)
    if args.tile:
        w.m = args.tile
    if args.points:
        w.n_points = args.points
    if args.shifts:
        if args.shifts > len(w.shifts):  # more shifts than the workload draws: append fresh ones
            extra = synth.lattice_shifts(args.shifts - len(w.shifts), w.shifts.shape[1], 3100 + args.workload)
            w.shifts = np.concatenate([w.shifts, extra])
        w.n_shifts = args.shifts
        w.shifts = w.shifts[:args.shifts]
    if args.reorder >= 0:
        w.reorder = args.reorder
    w.schur = 1 if args.schur == "tlr" else 0
    return w


def bench_config(tl, F, w, precision):
    """The workload a line is quoted on (shared by both arms)."""
    info = tl.tlrmvn_factor_info(F)
    return {"workload": w.name, "n": w.n, "tile": w.m, "tol": w.tol, "max_rank": w.max_rank, "nu": w.nu,
            "shifts": w.n_shifts, "points": w.n_points, "reorder": w.reorder,
            "schur": "tlr" if getattr(w, "schur", 0) else "exact", "precision": precision,
            "k_total": info["k_total"], "tiles": info["r"], "ranks": rank_summary(tl, F),
            "l2": "inputs larger than L2 (factor and W buffer)"}


def rank_summary(tl, F):
    """Mean, quartiles and maximum of the off-diagonal tile ranks of a factor."""
    rk = tl.tlrmvn_factor_ranks(F)
    low = rk[np.tril_indices(rk.shape[0], -1)]
    if low.size == 0:
        return {"mean": 0.0}
    q = np.percentile(low, [25, 50, 75]).tolist()
    return {"mean": float(low.mean()), "q25": q[0], "median": q[1], "q75": q[2], "max": int(low.max()),
            "zero_tiles": int((low == 0).sum()), "tiles": int(low.size)}


def device_solve_ms(tl, F, a, b, out, kw, reps, warm=1):
    """Device milliseconds per solve (CUDA events on the solve's stream, after `warm` untimed solves)."""
    import torch
    stream = kw["stream"]
    for _ in range(warm):
        tl.tlrmvn_prob_device(F, a, b, out, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(reps):
        e0.record(stream)
        tl.tlrmvn_prob_device(F, a, b, out, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def sweep_work(info, sizes, m, ktot, n):
    """Algorithmic work per sample-dimension of one solve, by where it runs.

    sweep   the diagonal-tile recursion of eq. 2: (mt - 1) flops per variable of a
            tile of mt variables (m - 1 = 511 for tiles of 512), whether the sums
            over earlier variables run in the per-sample chain or, regrouped, as
            the in-tile coupling products
    tensor  the low-rank shifts and projections, 4 m K_total / n flops, plus the
            coupling between 64-variable sub-tiles as the kernel issues it: three
            products (hi hi, hi lo, lo hi) of 2 mq q0 flops per sub-tile and sample
    """
    sweep = sum(mt * (mt - 1) for mt in sizes) / n
    couple = 0.0
    for mt in sizes:
        for q0 in range(64, mt, 64):
            couple += 3 * 2.0 * min(64, mt - q0) * q0
    return {"sweep": sweep, "tensor": 4.0 * m * ktot / n + couple / n, "shift_proj": 4.0 * m * ktot / n}


def serving_leg(tl, n_requests: int, rate: float = 0.0, seed: int = 7000) -> dict:
    """The serving workload: 8 resident factors (n = 1,024 ... 16,384 on jittered grids,
    Matern 1/2 and 3/2 kernels), a Poisson stream of requests with fresh b_i ~ U(0,1),
    nu in {3, 7, inf}, FP32 and BF16-shift classes, 10 shifts x 1,000 points each;
    4 lanes, 16 GiB scratch budget.  The arrival rate is `rate` requests/s, or (0) the
    rate a single lane sustains alone, measured from the first requests."""
    import threading
    import synth
    sides = [32, 45, 64, 64, 90, 90, 128, 128]          # n = 1,024 ... 16,384
    kernels = [(tl.KERNEL_EXP, (0.1,)), (tl.KERNEL_MATERN15, (0.05,))] * 4
    factors, sizes = [], []
    t0 = time.perf_counter()
    for f, g in enumerate(sides):
        xy = synth.jittered_grid(g, 5000 + f)
        n = g * g
        a, b = synth.limits_uniform(n, 6000 + f)
        kern, prm = kernels[f]
        factors.append(tl.tlrmvn_factor_kernel(xy, kern, prm, 1e-6, a, b, 128 if n <= 4096 else 256, 1e-5, 0,
                                               tl.REORDER_BLOCK))
        sizes.append(n)
    factor_s = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n_requests):
        f = int(rng.integers(0, len(factors)))
        reqs.append((f, np.full(sizes[f], -np.inf), rng.uniform(0.0, 1.0, sizes[f]), [3.0, 7.0, math.inf][q % 3],
                     tl.FP32 if q % 2 == 0 else tl.BF16_SHIFT))
    kw = dict(n_shifts=10, n_points=1000)
    srv = tl.Server(factors, lanes=4, memory_budget=16 << 30)
    alone = []
    for q, (f, a, b, nu, prec) in enumerate(reqs[:16]):  # warm-up and the alone service time
        rid = srv.submit(f, a, b, nu, prec, seed=q, **kw)
        alone.append(srv.wait(rid)[2])
    service = statistics.mean(alone[4:])
    rate = rate if rate > 0 else 1e3 / service
    srv.close()
    srv = tl.Server(factors, lanes=4, memory_budget=16 << 30)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    ids = [None] * n_requests
    t_start = time.perf_counter()

    def submitter():
        t = time.perf_counter()
        for q, (f, a, b, nu, prec) in enumerate(reqs):
            t += gaps[q]
            dt = t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids[q] = srv.submit(f, a, b, nu, prec, seed=q, **kw)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat = [srv.wait(i)[2] for i in ids]
    makespan = time.perf_counter() - t_start
    st = srv.stats()
    srv.close()
    sd = sum(sizes[f] for f, *_ in reqs) * kw["n_shifts"] * kw["n_points"]
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "rate_per_s": rate, "requests": n_requests, "throughput": sd / makespan, "unit": "sample-dims/s",
            "service_ms_alone_mean": service, "lanes": 4, "memory_budget_gib": 16,
            "load": "Poisson arrivals at the rate one lane sustains alone (1 / mean service time of a request "
                    "run alone)" if rate == 1e3 / service else f"Poisson arrivals at {rate} requests/s",
            "workload": "8 resident factors n=1,024..16,384 (exp / Matern-3/2, Algorithm 4), b~U(0,1) fresh per "
                        "request, nu in {3,7,inf}, FP32 and BF16-shift classes, 10 x 1,000 points each",
            "overlapped": st["overlapped"], "peak_in_flight": st["peak_in_flight"], "factor_seconds": factor_s}


def run_ours(args):
    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    import synth
    w = load_workload(args)
    if ws > 1:
        # disjoint shift batches per rank: same problem, independent replicas
        w.shifts = synth.lattice_shifts(w.n_shifts, w.n + 1, 3000 + args.workload + 7919 * rank)
    prec = PRECISIONS[args.precision]
    F, factor_s = build_factor(tl, w)
    info = tl.tlrmvn_factor_info(F)
    stream = torch.cuda.current_stream()
    a = torch.tensor(w.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(w.b, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    per_shift = torch.zeros(w.n_shifts, dtype=torch.float64, device="cuda")
    # launch choices for this problem: the library's autotuner (untimed setup; cached per box)
    cache = os.path.join(tempfile.gettempdir(), "tlrmvn_tune_cache.txt")
    if args.no_tune:
        tuned = dict(tl.tlrmvn_get_tuning(F, prec), note="library defaults (--no-tune)")
    else:
        tuned = tl.tlrmvn_autotune(F, w.a, w.b, w.nu, prec, n_shifts=w.n_shifts, n_points=w.n_points,
                                   shifts=w.shifts, cache_path=cache, stream=stream)
    kw = dict(nu=w.nu, precision=prec, n_shifts=w.n_shifts, n_points=w.n_points, shifts=w.shifts, stream=stream,
              per_shift=per_shift, sample_chunk=args.sample_chunk)

    for _ in range(args.warmup):
        tl.tlrmvn_prob_device(F, a, b, out, **kw)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler capture exactly the timed launches
    ev0.record(stream)
    for _ in range(args.steps):
        tl.tlrmvn_prob_device(F, a, b, out, **kw)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = allmax(ws, ms)
    # per-kernel-class times (events around every launch) from as many extra,
    # untimed steps: the events' own overhead stays out of the timed region
    tl.tlrmvn_profile_reset()
    tl.tlrmvn_profile_enable(True)
    for _ in range(args.steps):
        tl.tlrmvn_prob_device(F, a, b, out, **kw)
    torch.cuda.synchronize()
    tl.tlrmvn_profile_enable(False)
    logp, err = out.tolist()
    if ws > 1:
        # replicas: pool the per-shift log means of all ranks (one gather of M doubles per rank)
        import torch.distributed as dist
        from paper_2003_11183_gb300 import replicas
        logp, err = replicas.gather_and_combine(per_shift.cpu().numpy(), group=dist.new_group(backend="gloo"))
    kern = {tl.KC_NAMES[c]: tl.tlrmvn_profile_get(c) for c in range(len(tl.KC_NAMES))}
    launches = sum(v[1] for v in kern.values())
    C = w.n_shifts * w.n_points
    sd = w.n * C
    value = ws * sd / (ms / 1e3)

    # end to end through the public host-array entry point
    h2d = 2 * w.n * 8 + w.shifts.nbytes
    t_e2e = []
    for _ in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tl.tlrmvn_prob(F, w.a, w.b, **{k: v for k, v in kw.items() if k != "per_shift"})
        t_e2e.append(time.perf_counter() - t0)
    e2e = ws * sd / statistics.mean(t_e2e)

    # roofline of the dominant kernel class.  Algorithmic work per sample-dimension
    # (the accounting stated in sweep_work): the sweep's (mt - 1) flops per
    # variable against the FP32 peak derived from this device's SM count and the SM
    # clock sampled during the timed region (128 FP32 lanes x 2 flops per FMA per SM
    # and cycle); the tensor-core products beside it against the bf16 peak.
    pk, pk_kind = peaks()
    m, n = w.m, w.n
    sizes = [min(m, n - t * m) for t in range(info["r"])]
    work = sweep_work(info, sizes, m, info["k_total"], n)
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or pk.get("sm_max_mhz", 2070.0)
    fp32_peak = sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    fp32_src = (f"derived: {sm_count} SMs (device attribute) x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz "
                "(median SM clock sampled during the timed region)")
    bf16_peak = pk.get("bf16_tflops_sustained", 1700.0)
    # beside the derived peak, the library's own float32 FMA-throughput probe on this GPU
    fp32_meas = tl.tlrmvn_measure_fp32_peak(stream)
    classes = {}
    for cls, (t_ms, n_launch) in kern.items():
        if t_ms <= 0 or n_launch == 0:
            continue
        d = {"ms_per_step": t_ms / args.steps, "launches_per_step": n_launch / args.steps,
             "avg_launch_ms": t_ms / n_launch}
        if cls == "diag":
            units = float(n) * C * args.steps / n_launch  # sample-dims per launch
            ach = work["sweep"] * units / (d["avg_launch_ms"] / 1e3) / 1e12
            d.update(bound="alu", unit="TFLOP/s", achieved=ach, peak=fp32_peak, frac=ach / fp32_peak,
                     peak_source=fp32_src, peak_measured=fp32_meas, frac_of_measured=ach / fp32_meas,
                     peak_measured_source="tlrmvn_measure_fp32_peak: 8 independent FMA chains per thread, "
                                          "8 x 256 threads per SM, CUDA events",
                     flops_per_sample_dim=work["sweep"], sample_dims_per_launch=units,
                     kernel={0: "k_diag<double>", 1: "k_diag_f32"}.get(prec, "k_sweep_tc"))
            if prec >= 2:
                tach = work["tensor"] * units / (d["avg_launch_ms"] / 1e3) / 1e12
                d["tensor_share"] = {"bound": "tensor", "unit": "TFLOP/s", "achieved": tach, "peak": bf16_peak,
                                     "frac": tach / bf16_peak, "flops_per_sample_dim": work["tensor"],
                                     "peak_source": f"bf16 sustained, {pk_kind} (MEASURED_PEAKS.json)",
                                     "note": "low-rank shifts and projections 4 m K_total / n plus the split "
                                             "in-tile coupling (3 bf16 products), issued inside the same kernel"}
        classes[cls] = d
    from paper_2003_11183_gb300 import build as _build
    for cls, d in classes.items():
        t = TRAFFIC.get(d.get("kernel", ""))
        if t and t["bytes_per_sample_dim"] and t["sources"] == _build.source_digest(t["files"]):
            d["traffic"] = t["bytes_per_sample_dim"] * d["sample_dims_per_launch"]
            d["traffic_source"] = (f"ncu capture constant ({t['capture']}): DRAM bytes per sample-dimension of one "
                                   "captured launch, scaled to this run's launches by sample-dimensions")
        else:
            d["traffic"] = None
    dom = max(classes, key=lambda c: classes[c]["ms_per_step"])
    roof = {k: v for k, v in classes[dom].items() if k in ("bound", "achieved", "peak", "unit", "frac", "traffic",
                                                            "traffic_source", "peak_source", "kernel",
                                                            "peak_measured", "frac_of_measured",
                                                            "peak_measured_source",
                                                            "flops_per_sample_dim", "sample_dims_per_launch",
                                                            "tensor_share")}

    extra = {}
    cpu = None
    if rank == 0 and not args.no_baselines:
        # the same library's FP64 and FP32 paths on a sample count that fills the GPU
        # (20 x 2,500 = 50,000 samples: one wave of the FP64 sweep's blocks on every SM)
        pts_b = min(2500, w.n_points)
        kw_b = dict(kw, n_points=pts_b, per_shift=None)
        for name, p in (("fp64_path", 0), ("fp32_path", 1)):
            kw_p = dict(kw_b, precision=p)
            t_p = device_solve_ms(tl, F, a, b, out, kw_p, reps=2)
            v_p = w.n * w.n_shifts * pts_b / (t_p / 1e3)
            extra[name] = {"value": v_p, "unit": "sample-dims/s", "ms_per_solve": t_p,
                           "sample": f"{w.n_shifts} shifts x {pts_b} points (same factor and lattice), CUDA events",
                           "tuning": tl.tlrmvn_get_tuning(F, p), "speedup_of_this_line": (value / ws) / v_p}
        # the CPU oracle on bounded samples of the same workload and factor: all host cores, and one
        path = os.path.join(tempfile.gettempdir(), f"tlrmvn_factor_{os.getpid()}.bin")
        with open(path, "wb") as fh:
            fh.write(tl.tlrmvn_factor_export(F))
        cores = host_cores()
        pool = OraclePool(path, args.workload, cores, ORACLE_POINTS, [0])
        res_all = pool.run_round()
        pool.close()
        pool = OraclePool(path, args.workload, 1, ORACLE_POINTS, [0])
        res_one = pool.run_round()
        pool.close()
        os.unlink(path)
        v_all = w.n * res_all["samples"] / res_all["seconds"]
        v_one = w.n * res_one["samples"] / res_one["seconds"]
        cpu = {"value": v_all, "unit": "sample-dims/s", "cores": cores, "kind": "oracle",
               "sample": (f"{cores} single-threaded worker processes x {ORACLE_POINTS} lattice points of shift 0 "
                          f"of the same workload and factor ({res_all['samples']} samples x {w.n} dimensions)"),
               "one_core": {"value": v_one, "unit": "sample-dims/s",
                            "sample": f"1 process x {ORACLE_POINTS} points of shift 0"},
               "nproc": os.cpu_count()}
        # served latency at a stated load (the metric's second half)
        extra["serving"] = serving_leg(tl, args.requests if args.requests else 160, args.rate)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "sample-dims/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {0: "f64", 1: "f32", 2: "f32+bf16", 3: "f32+fp16"}[prec], "data": "synthetic",
                "config": dict(bench_config(tl, F, w, args.precision), sample_chunk=args.sample_chunk or "all",
                               tuning=tuned),
                "clocks": clk,
                "e2e": {"value": e2e, "unit": "sample-dims/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16},
                "gpu_launches": launches, "roofline": roof, "kernel_classes": classes, "cpu_baseline": cpu,
                "factor_seconds": factor_s, "logp": logp, "err": err,
                "accuracy": {"rel_err_qmc": err,
                             "note": "err is the QMC standard error of the estimate divided by it (the paper's "
                                     "relative error); at this sample count three of them span ~2.4 in log p, so "
                                     "the full-size accuracy claim is the per-shift comparison with the FP64 path "
                                     "in the GPU tests (1e-4 FP32, 1e-2 BF16-shift)"},
                "precision_note": {
                    0: "f64: every step in float64",
                    1: "f32: float32 sweep of eq. 2 (per-sample chains within 64-variable sub-tiles); low-rank "
                       "shifts, projections and the in-tile coupling between sub-tiles as float32 SIMT products",
                    2: "f32+bf16: float32 sweep of eq. 2 (per-sample chains within 64-variable sub-tiles); low-rank "
                       "shifts and projections bf16 x bf16 -> fp32 on tcgen05; the in-tile coupling between "
                       "sub-tiles as split-bf16 products (hi hi + hi lo + lo hi, ~1e-5 relative) -> fp32",
                    3: "f32+fp16: as f32+bf16 with fp16 operands, U and V scaled per tile by powers of two"}[prec]}
        if "serving" in extra:
            line["p50_ms"] = extra["serving"]["p50_ms"]
            line["p99_ms"] = extra["serving"]["p99_ms"]
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Batched workload: 256 MVN problems (n log-uniform in [256, 4096], own covariances,
    m = 128, tol 1e-5, iterative block reordering), 10 shifts x 2,000 points each, solved by
    one persistent launch (a replayed CUDA graph) per step."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    import synth
    probs = synth.batched_problems(args.count)
    t0 = time.perf_counter()
    factors = [tl.tlrmvn_factor_kernel(p["xy"], tl.KERNEL_EXP, (p["beta"],), 1e-8, p["a"], p["b"], 128, 1e-5, 0,
                                       tl.REORDER_ITERATIVE) for p in probs]
    factor_s = time.perf_counter() - t0
    M, N = 10, args.points or 2000
    a = [p["a"] for p in probs]
    b = [p["b"] for p in probs]
    sd = sum(len(p["a"]) for p in probs) * M * N
    cache = os.path.join(tempfile.gettempdir(), "tlrmvn_tune_cache.txt")
    # the line's precision (BF16-shift: the tensor-core persistent kernel; FP32: the SIMT
    # one), and the other one timed beside it on the same problems and shifts
    main = tl.BF16_SHIFT if args.precision in ("bf16", "fp16") else tl.FP32
    other = tl.FP32 if main == tl.BF16_SHIFT else tl.BF16_SHIFT
    name = {tl.BF16_SHIFT: "f32+bf16", tl.FP32: "f32"}

    def timed(prec, steps, clocks=None):
        plan = tl.BatchPlan(factors, math.inf, M, N, seed=4242, precision=prec)
        tuned = plan.tune(a, b, cache_path=cache)
        for _ in range(args.warmup):
            plan.run(a, b)
        if clocks:
            clocks.start()
        times = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            lp, err = plan.run(a, b)
            times.append(time.perf_counter() - t1)
        clk = clocks.stop() if clocks else None
        plan.close()
        return times, tuned, lp, err, clk

    times, tuned, lp, err, clk = timed(main, args.steps, Clocks(0))
    ms = statistics.mean(times) * 1e3
    t_o, tuned_o, lp_o, err_o, _ = timed(other, max(1, args.steps))
    ms_o = statistics.mean(t_o) * 1e3
    line = {"metric": "batched QMC sample-dims/sec", "value": sd / (ms / 1e3), "unit": "sample-dims/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "p50_ms": statistics.median(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": name[main],
            "data": "synthetic",
            "config": {"workload": f"batched_{len(probs)}_mvn_n256_4096_m128", "problems": len(probs),
                       "sum_n": sum(len(p["a"]) for p in probs), "shifts": M, "points": N, "tol": 1e-5,
                       "precision": name[main], "tuning": tuned,
                       "timing": "host clock around each plan replay (limits upload, one graph, results read back)"},
            "clocks": clk, "factor_seconds": factor_s,
            "e2e": {"value": sd / (ms / 1e3), "unit": "sample-dims/s",
                    "h2d_bytes_per_step": 2 * 8 * sum(len(p["a"]) for p in probs),
                    "d2h_bytes_per_step": 16 * len(probs)},
            "logp_mean": float(np.mean(lp)), "err_median": float(np.median(err)),
            "other_precision": {"dtype": name[other], "value": sd / (ms_o / 1e3), "unit": "sample-dims/s",
                                "ms_per_step": ms_o, "tuning": tuned_o,
                                "max_logp_gap_in_se": float(np.max(np.abs(lp - lp_o) / np.hypot(err, err_o)))}}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Serving workload (see serving_leg), as a line of its own."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    clocks = Clocks(0)
    clocks.start()
    r = serving_leg(tl, args.requests or 400, args.rate)
    clk = clocks.stop()
    line = {"metric": "served QMC sample-dims/sec and p50/p99 latency", "value": r["throughput"],
            "unit": "sample-dims/s", "n_gpus": 1, "steps": r["requests"], "warmup": 16,
            "ms_per_step": 1e3 / r["rate_per_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 | f32+bf16", "data": "synthetic",
            "config": {"workload": "serving_8_factors_n1024_16384", "requests": r["requests"],
                       "rate_per_s": r["rate_per_s"], "lanes": r["lanes"], "memory_budget_gib": r["memory_budget_gib"],
                       "shifts": 10, "points": 1000, "service_ms_alone_mean": r["service_ms_alone_mean"]},
            "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "serving": r, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_study(args):
    """Convergence study (the shape of Section 4, Table 3): for an MVN problem on a
    perturbed grid with an exponential kernel and a = -inf, b_i ~ N(5.5, 1.25^2)
    (the paper's simulated limits), tile m = sqrt(n), the same problem is solved
    with the geometric order alone, with Algorithm 4 and with Algorithm 5, at
    N = 1,000 and 10,000 lattice points per shift (20 shifts), and the line
    reports each estimate, its relative error (the QMC standard error over the
    estimate) and the device time.  The paper's claim under test: the block
    reorderings lower the error at equal N (Section 4)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    import synth
    g = args.n_side or 128
    n = g * g
    m = int(round(math.sqrt(n)))
    prec = PRECISIONS[args.precision if args.precision != "bf16" else "fp64"]
    rows = []
    for beta, tol in ((0.3, 1e-4), (0.1, 1e-3)):
        xy = synth.jittered_grid(g, 8000)
        a, b = synth.limits_normal(n, 8001, 5.5, 1.25)
        for reorder, schur, name in ((tl.REORDER_NONE, 0, "tlrmvn (geometric order)"),
                                     (tl.REORDER_BLOCK, 0, "rtlrmvn (Algorithm 4)"),
                                     (tl.REORDER_ITERATIVE, 0, "rrtlrmvn (Algorithm 5)"),
                                     (tl.REORDER_ITERATIVE, 1, "rrtlrmvn (Algorithm 5, TLR arithmetic)")):
            t0 = time.perf_counter()
            F = tl.tlrmvn_factor_kernel(xy, tl.KERNEL_EXP, (beta,), 1e-8, a, b, m, tol, 0, reorder, schur=schur)
            fs = time.perf_counter() - t0
            info = tl.tlrmvn_factor_info(F)
            for pts in (1000, 10000):
                shifts = synth.lattice_shifts(20, n + 1, 8100 + pts)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lp, err, _, _ = tl.tlrmvn_prob(F, a, b, math.inf, prec, 20, pts, shifts=shifts)
                t = time.perf_counter() - t0
                rows.append({"beta": beta, "tol": tol, "method": name, "reorder": reorder,
                             "schur": "tlr" if schur else "exact", "points": pts,
                             "shifts": 20, "logp": lp, "rel_err": err, "seconds": t, "factor_seconds": fs,
                             "k_total": info["k_total"]})
    # agreement of the three orderings (the same probability): largest pairwise gap in
    # log p over the combined standard errors, per beta and N
    agree = {}
    for beta in (0.3, 0.1):
        for pts in (1000, 10000):
            sel = [r for r in rows if r["beta"] == beta and r["points"] == pts]
            gap = max(abs(x["logp"] - y["logp"]) / math.hypot(x["rel_err"], y["rel_err"]) for x in sel for y in sel
                      if x is not y)
            agree[f"beta{beta}_N{pts}"] = gap
    line = {"metric": "QMC relative error at equal N: geometric order vs Algorithm 4 vs Algorithm 5",
            "value": min(r["rel_err"] for r in rows), "unit": "relative error", "n_gpus": 1, "steps": len(rows),
            "warmup": 0, "higher_is_better": False, "data": "synthetic",
            "dtype": {0: "f64", 1: "f32", 2: "f32+bf16", 3: "f32+fp16"}[prec],
            "config": {"workload": f"study_mvn_n{n}_exp", "n": n, "tile": m, "limits": "a=-inf, b~N(5.5,1.25^2)",
                       "kernel": "exponential", "betas": [0.3, 0.1], "tols": [1e-4, 1e-3], "shifts": 20},
            "rows": rows, "max_gap_in_combined_se": agree}
    print(json.dumps(line), flush=True)
    return 0


def run_skewnormal(args):
    """Skew-normal likelihood (Section 5.1, eq. 6; the shape of Table 4's MLE-TLR
    column): for n = 4^r, r = 4..7, locations on a 2^r x 2^r grid of spacing 1/15
    perturbed by U(0, 0.8/15), theta = (xi, sigma1, beta1, sigma2, beta2) =
    (0, 1, 0.3, 1, 0.3), one draw z of the model (eq. 5); each line reports the time
    of one log-likelihood evaluation and of its MVN factor (TLR factor of
    (I + C^T C)^-1 and the float32 integrand, tile sqrt(n), tolerance 1e-5,
    10 x 1,000 lattice points), after one untimed evaluation."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2003_11183_gb300 import skewnormal as sn
    theta = (0.0, 1.0, 0.3, 1.0, 0.3)
    rows = []
    for r in (4, 5, 6, 7):
        g = 2 ** r
        n = g * g
        xy = synth.expanding_grid(g, 1.0 / 15.0, 9000 + r)
        z = sn.simulate(xy, theta, 9100 + r)
        kw = dict(tile=int(math.isqrt(n)), tol=1e-5, n_shifts=10, n_points=1000, seed=9200 + r)
        sn.loglik(z, xy, theta, **kw)
        tm = {}
        t0 = time.perf_counter()
        lf, err = sn.loglik(z, xy, theta, timings=tm, **kw)
        rows.append({"n": n, "seconds": time.perf_counter() - t0, "mvn_seconds": tm["mvn"],
                     "dense_seconds": tm["dense"], "loglik": lf, "rel_err_mvn": err})
    line = {"metric": "skew-normal log-likelihood evaluation time (eq. 6); MVN factor time", "value": rows[-1]["seconds"],
            "unit": "s", "n_gpus": 1, "steps": len(rows), "warmup": 1, "higher_is_better": False,
            "dtype": "f64 dense algebra + f32 TLR-QMC", "data": "synthetic",
            "config": {"workload": "skewnormal_table4_shape", "theta": theta, "grid_spacing": 1 / 15,
                       "tol": 1e-5, "shifts": 10, "points": 1000, "tile": "sqrt(n)"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == 4:
        return run_batched(args)
    if args.workload == 5:
        return run_serving(args)
    if args.workload == 6:
        return run_study(args)
    if args.workload == 7:
        return run_skewnormal(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
