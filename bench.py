"""Benchmark: RHS-solves/s and preconditioner applies/s for the recursive
moving-PML sweeping preconditioner with GMRES, on the 64-source workload.

Workload (the configuration the headline metric is quoted on): n = 127
interior points per axis, b = 6 PML layers on every face (139^3 unknowns),
d = 1, omega = 2 pi 127 / 8 (8 points per wavelength), smooth random velocity
in [1, 2] (seed 0), 64 Gaussian sources on an 8 x 8 grid of the z = 0.1 plane,
GMRES(30) to a true relative residual of 1e-6.  Synthetic inputs, seeded.

The handle is set up once (helm_setup: coefficients, the quasi-1D
factorisations and, in the dense form, the restricted operators; its time is
reported as setup_s).  A step is one helm_solve of the 64 right-hand sides on
that handle (GMRES with the recursive sweep, stencil and FP64 residuals), so
value = 64 x steps / time: RHS-solves/s with the setup excluded.  Inputs are
resident in HBM for `value`; `e2e` repeats the user's whole path from pinned
host buffers (velocity and sources in, setup, solve, solutions out).  The
stored operators (about 150 GB) exceed L2, so no flush is needed between
steps.  The line also times the plain complex-FP32 form of the same method
(`plain_fp32`), which the split-precision form is compared against.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: the method has no data-parallel exchange here, so N GPUs run N
independent replicas (weak scaling, one process per GPU under torchrun).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RHS-solves/s and precond applies/s at n=127, 64 RHS, vs plain FP32; rel err"
TOL = 1e-6
# GMRES iterations per right-hand side on this workload (the GPU's measured
# count: 23-25 with two fronts and b_aux = 2, 21-22 with one front and b_aux = 6);
# the oracle applies the same preconditioner M, so its timed sample is scaled to
# RHS-solves/s with it when no GPU count is at hand.
NOMINAL_ITERS = {"two_front": 25, "one_front": 22}

# The headline configuration: the paper's own schedule of Section 5 (two fronts
# in both loops, an auxiliary PML thinner than the boundary PML) on the
# workload's grid (b = 6, d = 1).
DEFAULT_SCHEDULE = "two_front"
DEFAULT_B_AUX = 2


def _workload(n: int, per_side: int):
    from paper_1502_07266_gb300 import workloads as W
    return W.random_64_sources(n=n, b=6, d=1, seed=0, per_side=per_side)


ENTRY_BYTES = {"fp32": 8, "fp16": 4, "split_fp16": 8}   # stored bytes per complex factor entry
DENSE_TEXT = {
    "fp32": "dense restricted operators in complex FP32, FP32 SIMT products; FP64 residual, Arnoldi, "
            "Givens and solution",
    "split_fp16": "dense restricted operators as FP16 hi+lo (power-of-two row scales), inputs split hi+lo, "
                  "three tcgen05 FP16 products with FP32 accumulation; FP64 residual, Arnoldi, Givens and solution",
    "fp16": "dense restricted operators as FP16 hi (row scales), inputs split hi+lo, two tcgen05 FP16 products "
            "with FP32 accumulation; FP64 residual, Arnoldi, Givens and solution",
}
PRECISION_TEXT = {
    "fp32": "complex FP32 factors and products; FP64 residual, Arnoldi, Givens and solution",
    "fp16": "FP16 factors (power-of-two scale per block), FP32 products; FP64 residual, Arnoldi, "
            "Givens and solution",
    "split_fp16": "FP16 hi+lo factors (scale per block, ~22 bits), FP32 products; FP64 residual, "
                  "Arnoldi, Givens and solution",
}


def _blocks_and_bytes(n: int, b: int, d: int, precision: str = "fp32"):
    """Swept-axis block count and the algorithmic factor bytes of one apply.

    Every quasi-1D problem (M, M') is solved once per use: slab M is visited
    twice by Algorithm 6 (once if M is the last block) and line block M' twice
    by Algorithm 4 (once if last); a solve reads each of its N factor blocks
    (k x k entries of the stored precision) once when the forward and backward
    passes share L2.
    """
    esz = ENTRY_BYTES[precision]
    N = n + 2 * b
    wins = [b]
    m = b
    while m < N:
        e = min(m + d, N)
        wins.append(e - max(m - b, 0))
        m += d
    B = len(wins)
    total = 0
    for M in range(B):
        uz = 2 if M <= B - 2 else 1
        for Mp in range(B):
            uy = 2 if Mp <= B - 2 else 1
            k = wins[M] * wins[Mp]
            total += uz * uy * N * k * k * esz
    # dependent steps per apply: each quasi-1D solve runs its two elimination
    # halves concurrently (left chain m steps, right chain N-1-m, middle, back)
    m = (N - 1) // 2
    steps = (2 * B - 1) ** 2 * (2 * max(m, N - 1 - m) + 1)
    return B, total, steps


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_per_launch(n: int):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "sweep_traffic.txt")
    src = os.path.join(ROOT, "paper_1502_07266_gb300", "csrc", "sweep.cu")
    try:
        digest = hashlib.sha1(open(src, "rb").read()).hexdigest()
        fields = {}
        for line in open(path):
            if ":" in line:
                key, val = line.split(":", 1)
                fields[key.strip()] = val.strip()
        if fields.get("sweep.cu sha1") != digest or int(fields.get("n", -1)) != n:
            return None
        return float(fields["dram bytes per launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU oracle

def _slab_task(task):
    """One oracle slab solve (Algorithm 4 on slab M for one right-hand side,
    refactoring its quasi-1D problems), timed inside the worker process."""
    n, M, seed, schedule, b_aux = task
    import numpy as np

    from oracle.operator import Grid
    from oracle.sweep import SweepPreconditioner
    wl = _workload(n, 1)
    P = SweepPreconditioner(wl.c.astype(np.float32).astype(np.float64), Grid(wl.n, wl.b, wl.omega), d=wl.d,
                            b_aux=b_aux or None, keep_factors=False, schedule=schedule)
    pz, (za, zb) = P.zwin[M]
    rng = np.random.default_rng(seed)
    alpha = rng.standard_normal((1, zb - za, P.N, P.N)) + 1j * rng.standard_normal((1, zb - za, P.N, P.N))
    t0 = time.perf_counter()
    P.slab_apply(M, alpha)
    return time.perf_counter() - t0


def _warm_task(_):
    import numpy  # noqa: F401
    import scipy.sparse.linalg  # noqa: F401

    import oracle.sweep  # noqa: F401
    return os.getpid()


def _nblocks(n: int, schedule: str, b_aux: int) -> int:
    """Swept-axis blocks B of the workload's grid (b = 6, d = 1) under a schedule."""
    return len(_axis_windows(n + 12, 6, 1, b_aux or 6, schedule)[0])


def cpu_sample(n: int, rounds: int = 1, workers: int | None = None, schedule: str = "one_front", b_aux: int = 0):
    """Times the FP64 oracle as it stands on a bounded sample of the workload:
    `workers` interior slab solves at once (one per host core, each a
    single-threaded process started with spawn), `rounds` times.  Returns
    (slab solves per second over the whole pool, workers, seconds per round)."""
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    B = _nblocks(n, schedule, b_aux)
    with ctx.Pool(workers) as pool:
        pool.map(_warm_task, range(workers))
        walls = []
        for r in range(rounds):
            tasks = [(n, B // 2 - workers // 2 + i, 10 * r + i, schedule, b_aux) for i in range(workers)]
            t0 = time.perf_counter()
            pool.map(_slab_task, tasks, chunksize=1)
            walls.append(time.perf_counter() - t0)
    per_round = sum(walls) / len(walls)
    return workers / per_round, workers, per_round


def oracle_rate(n: int, slabs_per_s: float, iters: float, schedule: str = "one_front", b_aux: int = 0):
    """RHS-solves/s and preconditioner applies/s (per RHS) of the oracle from
    its slab throughput: an apply is 2B-1 slab solves (Algorithm 6), a solve
    `iters` applies (the GMRES vector work is not counted)."""
    B = _nblocks(n, schedule, b_aux)
    applies = slabs_per_s / (2 * B - 1)
    return applies / iters, applies


def sample_text(n: int, workers: int, iters: float, schedule: str = "one_front", b_aux: int = 0):
    B = _nblocks(n, schedule, b_aux)
    sched = "two fronts" if schedule == "two_front" else "one front"
    return (f"FP64 oracle as it stands ({sched}, b_aux={b_aux or 6}), {workers} interior slab solves of "
            f"Algorithm 4 at once for 1 RHS each "
            f"(one spawned single-threaded process per host core, each refactoring its slab's {B} quasi-1D "
            f"problems) at n={n}; throughput scaled by {2 * B - 1} slab solves per apply and {iters:g} GMRES "
            f"iterations per RHS-solve (the GPU's measured count; GMRES vector work not counted)")


# ------------------------------------------------------- replica logic

def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over all ranks: a replicated job takes as long as its
    slowest replica.  dist is torch.distributed (None for one process)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, units_per_replica: int, steps: int, elapsed_max: float) -> float:
    """Whole-job throughput: every replica processes units_per_replica per step."""
    return world * units_per_replica * steps / elapsed_max


# ----------------------------------------------------------------- arms

def run_reference(args):
    """The oracle arm: the FP64 oracle on the host cores, each step one round
    of slab solves (one per core), on the GPU arm's workload, metric and unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    workers = os.cpu_count() or 1
    walls = []
    sched, b_aux = args.schedule, args.b_aux
    iters = NOMINAL_ITERS[sched]
    for s in range(args.warmup + args.steps):
        _, workers, wall = cpu_sample(n, rounds=1, workers=workers, schedule=sched, b_aux=b_aux)
        if s >= args.warmup:
            walls.append(wall)
    per_round = sum(walls) / len(walls)
    slabs_per_s = workers / per_round
    solves_s, applies_s = oracle_rate(n, slabs_per_s, iters, sched, b_aux)
    line = {
        "impl": "reference", "metric": METRIC, "value": solves_s, "unit": "RHS-solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_round * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": f"n={n} b=6 d=1 random velocity, 64 sources (8x8, z=0.1), tol 1e-6",
                   "schedule": sched, "b_aux": b_aux or 6,
                   "step": f"{workers} oracle slab solves at once (one round)", "l2": "host run"},
        "precond_applies_per_s": applies_s,
        "cpu_baseline": {"value": solves_s, "unit": "RHS-solves/s", "cores": workers, "kind": "oracle",
                         "sample": sample_text(n, workers, iters, sched, b_aux)},
        "e2e": {"value": solves_s, "unit": "RHS-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _axis_windows(N: int, b: int, d: int, b_aux: int, schedule: str):
    """(block start, block end, window length) of a swept axis in axis order,
    and the centre block's index: the block decomposition and windows of the
    library (one front: the boundary slab, blocks of d, the last block ends the
    forward pass; two fronts: the boundary slabs, q = (N-2b-1)//(2d) blocks of d
    from each end, a centre of 1..2d layers; a side eliminated towards gets
    b_aux layers, clipped at the faces)."""
    if schedule == "two_front":
        q = (N - 2 * b - 1) // (2 * d)
        blocks = [(0, b, "L")] + [(b + i * d, b + (i + 1) * d, "L") for i in range(q)]
        blocks += [(b + q * d, N - b - q * d, "C")]
        blocks += [(N - b - (i + 1) * d, N - b - i * d, "U") for i in reversed(range(q))] + [(N - b, N, "U")]
    else:
        blocks = [(0, b, "L")] + [(m, min(m + d, N), "L") for m in range(b, N, d)]
        blocks[-1] = (blocks[-1][0], blocks[-1][1], "C")
    out = []
    for m, e, role in blocks:
        lo = max(m - b_aux, 0) if (role != "U" and m > 0) else m
        hi = min(e + b_aux, N) if (role != "L" and e < N) else e
        out.append((m, e, hi - lo))
    return out, [r for _, _, r in blocks].index("C")


def _dense_model(n: int, b: int, d: int, entry_bytes: int = 8, schedule: str = "one_front", b_aux: int = 0):
    """Work of one apply in the dense form: the (2B-1)^2 quasi-1D solves of
    Algorithm 6 over Algorithm 4 each read their stored operator once
    (n_out x n_in entries).  Each slab is visited forward and backward except
    the centre slab (once); in a visit every line block is solved forward and
    every one but the centre backward.  Returns (solves, operator bytes per
    apply, complex multiply-adds per right-hand side and apply)."""
    N = n + 2 * b
    wins, c = _axis_windows(N, b, d, b_aux or b, schedule)
    B = len(wins)
    two = schedule == "two_front"
    total = macs = 0
    for M in range(B):
        visits = 1 if M == c else 2
        m, e, Lz = wins[M]
        dz = e - m
        for Mp in range(B):
            for bwd in ((0,) if Mp == c else (0, 1)):
                if Mp == 0:
                    n_in, n_out = ((b * dz * N, ((b - 1) * dz + Lz) * N) if not bwd else (Lz * N, b * dz * N))
                elif two and Mp == B - 1:
                    n_in, n_out = ((b * dz * N, ((b - 1) * dz + Lz) * N) if not bwd else (Lz * N, b * dz * N))
                else:
                    nl = wins[Mp][1] - wins[Mp][0]
                    n_in = n_out = nl * Lz * N
                total += visits * n_out * n_in * entry_bytes
                macs += visits * n_out * n_in
    return (2 * B - 1) ** 2, total, macs


def _dense_setup_model(n: int, b: int, d: int, schedule: str = "one_front", b_aux: int = 0):
    """Algorithmic work of the dense form's setup in real flops (a complex
    multiply-add counted as 8): the block LDU factorisation of every quasi-1D
    problem (M, M') (Alg. 3 per slab, Alg. 5: N blocks of k = Lz Ly, k^3 complex
    multiply-adds each) and its restricted operators (one forward and one
    backward block substitution, 2 N k^2 multiply-adds, per input column of
    every stored operator: the line block's own, and the separate backward maps
    of the boundary blocks).  Returns (factor flops, operator flops)."""
    N = n + 2 * b
    wins, c = _axis_windows(N, b, d, b_aux or b, schedule)
    B = len(wins)
    two = schedule == "two_front"
    fac = ops = 0
    for M in range(B):
        m, e, Lz = wins[M]
        dz = e - m
        for Mp in range(B):
            k = Lz * wins[Mp][2]
            fac += 8 * k ** 3 * N
            boundary = Mp == 0 or (two and Mp == B - 1)
            if boundary:
                cols = [b * dz * N, Lz * N]               # forward map, then the backward map
            else:
                cols = [(wins[Mp][1] - wins[Mp][0]) * Lz * N]
            ops += sum(8 * 2 * N * k * k * n_in for n_in in cols)
    return fac, ops


DENSE_ENTRY_BYTES = {"fp32": 8, "split_fp16": 8, "fp16": 4}


def _dense_traffic(n: int, precision: str, schedule: str, b_aux: int):
    """DRAM bytes per dense apply launch from the committed ncu summary, if it
    was taken on the current kernel source and the same schedule (else None)."""
    path = os.path.join(ROOT, "profiles", "dense_traffic.txt")
    csrc = os.path.join(ROOT, "paper_1502_07266_gb300", "csrc")
    try:
        digest = hashlib.sha1(open(os.path.join(csrc, "dense.cu"), "rb").read()).hexdigest()
        digest_s = hashlib.sha1(open(os.path.join(csrc, "dense_sched.h"), "rb").read()).hexdigest()
        fields = {}
        for line in open(path):
            if ":" in line:
                key, val = line.split(":", 1)
                fields[key.strip()] = val.strip()
        if (fields.get("dense.cu sha1") != digest or fields.get("dense_sched.h sha1") != digest_s
                or fields.get("precision") != precision
                or fields.get("schedule") != schedule or int(fields.get("b_aux", -1)) != (b_aux or 6)):
            return None
        return float(fields["dram bytes per full-size launch"])
    except Exception:
        return None


def run_gpu(args):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = _workload(args.n, 8)
    R = wl.R
    N = wl.N
    c_host = torch.from_numpy(wl.c.astype(np.float32)).pin_memory()
    f_host = torch.from_numpy(wl.f.astype(np.complex64)).pin_memory()
    c_dev = c_host.to(dev)
    f_dev = f_host.to(dev)
    u_dev = torch.empty_like(f_dev)
    st = torch.cuda.current_stream()

    def make(form, precision, c_t, schedule=args.schedule, b_aux=args.b_aux):
        opts = helm.helm_default_opts()
        opts.precision = helm.PRECISIONS[precision]
        opts.apply_form = helm.APPLY_FORMS[form]
        if form == "dense":  # the chain form runs one front with b_aux = b only
            opts.schedule = helm.SCHEDULES[schedule]
            opts.b_aux = b_aux
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h = helm.helm_setup(c_t.data_ptr(), wl.omega, wl.n, wl.b, wl.d, opts, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        return h, e0.elapsed_time(e1) / 1e3

    def solve(h, f_t, u_t):
        return helm.helm_solve(h, f_t.data_ptr(), u_t.data_ptr(), R, TOL, st.cuda_stream)

    # ---------------- the timed steps: 64-RHS solves on one set-up handle ----------------
    h, setup_s = make(args.form, args.precision, c_dev)
    helm.helm_enable_timing(h, True)
    for _ in range(args.warmup):
        solve(h, f_dev, u_dev)
    helm.helm_reset_stats(h)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    barrier()
    l0 = helm.helm_launch_count(h)
    t_start.record(st)
    runs = [solve(h, f_dev, u_dev) for _ in range(args.steps)]
    t_stop.record(st)
    barrier()
    clk = clocks.stop()
    launches = helm.helm_launch_count(h) - l0
    elapsed = max_over_ranks(t_start.elapsed_time(t_stop) / 1e3, dist, dev)
    stats = helm.helm_get_stats(h)
    stored = helm.helm_factor_bytes(h)
    codes = sorted({r[0] for r in runs})
    its = runs[-1][1]
    relmax = max(max(r[2]) for r in runs)
    sample_rhs = [0, 21, 42, 63]
    u_sample = u_dev[sample_rhs].cpu().numpy() if rank == 0 else None
    helm.helm_destroy(h)

    # ---------------- the plain complex-FP32 form of the same method ----------------
    plain = None
    if not args.no_plain and (args.form, args.precision) != ("dense", "fp32") and args.form == "dense":
        hp, setup_p = make("dense", "fp32", c_dev)
        helm.helm_enable_timing(hp, True)
        solve(hp, f_dev, u_dev)
        helm.helm_reset_stats(hp)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kp = 2
        p0.record(st)
        pr = [solve(hp, f_dev, u_dev) for _ in range(kp)]
        p1.record(st)
        torch.cuda.synchronize()
        tp = p0.elapsed_time(p1) / 1e3
        sp = helm.helm_get_stats(hp)
        plain = {"form": "dense operators in complex FP32, FP32 SIMT products", "value": R * kp / tp,
                 "unit": "RHS-solves/s", "setup_s": setup_p, "steps": kp,
                 "gmres_iters": {"min": min(pr[-1][1]), "max": max(pr[-1][1])},
                 "relres_fp64_max": max(max(r[2]) for r in pr),
                 "precond_applies_per_s": sp.rhs_applied / (sp.sweep_ms / 1e3) if sp.sweep_ms else None,
                 "apply_ms": sp.sweep_ms / max(sp.sweep_launches, 1)}
        helm.helm_destroy(hp)

    # ---------------- one front with b_aux = b, the schedule of Section 4.2 ----------------
    onefront = None
    if not args.no_plain and args.form == "dense" and (args.schedule, args.b_aux) != ("one_front", 0):
        ho, setup_o = make("dense", args.precision, c_dev, "one_front", 0)
        helm.helm_enable_timing(ho, True)
        solve(ho, f_dev, u_dev)
        helm.helm_reset_stats(ho)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ko = 2
        p0.record(st)
        orr = [solve(ho, f_dev, u_dev) for _ in range(ko)]
        p1.record(st)
        torch.cuda.synchronize()
        to = p0.elapsed_time(p1) / 1e3
        so = helm.helm_get_stats(ho)
        onefront = {"schedule": "one_front", "b_aux": wl.b, "value": R * ko / to, "unit": "RHS-solves/s",
                    "setup_s": setup_o, "steps": ko,
                    "gmres_iters": {"min": min(orr[-1][1]), "max": max(orr[-1][1])},
                    "relres_fp64_max": max(max(r[2]) for r in orr),
                    "apply_ms": so.sweep_ms / max(so.sweep_launches, 1)}
        helm.helm_destroy(ho)

    # ---------------- e2e: the user's whole path from pinned host buffers ----------------
    e2e = None
    if not args.no_e2e:
        u_host = torch.empty_like(f_host).pin_memory()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        c_t = c_host.to(dev, non_blocking=True)
        f_t = f_host.to(dev, non_blocking=True)
        u_t = torch.empty_like(f_t)
        he, _ = make(args.form, args.precision, c_t)
        solve(he, f_t, u_t)
        u_host.copy_(u_t, non_blocking=True)
        e1.record(st)
        barrier()
        helm.helm_destroy(he)
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        e2e = {"value": replica_rate(world, R, 1, te), "unit": "RHS-solves/s",
               "h2d_bytes_per_step": c_host.numel() * 4 + f_host.numel() * 8,
               "d2h_bytes_per_step": u_host.numel() * 8,
               "includes": "host-to-device copy of velocity and sources, helm_setup, helm_solve, "
                           "device-to-host copy of the solutions"}
        del c_t, f_t, u_t

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    per_launch_ms = stats.sweep_ms / max(stats.sweep_launches, 1)
    peak, peak_kind = _peaks()
    if args.form == "dense":
        nsolves, alg_bytes, macs = _dense_model(wl.n, wl.b, wl.d, DENSE_ENTRY_BYTES[args.precision],
                                                args.schedule, args.b_aux)
        kernel = {"fp32": "k_dense<FP32 SIMT>", "split_fp16": "k_dense<FP16 hi+lo, tcgen05>",
                  "fp16": "k_dense<FP16 hi, tcgen05>"}[args.precision]
        traffic = _dense_traffic(wl.n, args.precision, args.schedule, args.b_aux)
        chain = {"dependent_solves_per_apply": nsolves, "us_per_solve": per_launch_ms * 1e3 / nsolves}
        flops = 8.0 * macs * R
    else:
        _, alg_bytes, chain_steps = _blocks_and_bytes(wl.n, wl.b, wl.d, args.precision)
        kernel = "k_sweep (block substitution chain)"
        traffic = _traffic_per_launch(wl.n)
        chain = {"dependent_steps_per_apply": chain_steps, "ns_per_step": per_launch_ms * 1e6 / chain_steps}
        flops = None
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    value = replica_rate(world, R, args.steps, elapsed)
    setup_work = None
    if args.form == "dense":
        fac_f, op_f = _dense_setup_model(wl.n, wl.b, wl.d, args.schedule, args.b_aux)
        setup_work = {"factor_flops": fac_f, "operator_flops": op_f,
                      "tflops": (fac_f + op_f) / setup_s / 1e12 if setup_s > 0 else None,
                      "note": "block LDU of every quasi-1D problem plus one forward and one backward "
                              "substitution per input column of every stored operator (FP32 SIMT)"}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "RHS-solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "c64", "split_fp16": "fp16 hi+lo -> fp32", "fp16": "fp16 -> fp32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"n={wl.n} b={wl.b} d={wl.d} ({N}^3), random velocity seed 0, "
                               f"{R} Gaussian sources (8x8, z=0.1), GMRES(30) tol {TOL}",
                   "step": "one helm_solve of the 64 right-hand sides on a set-up handle (setup excluded)",
                   "form": args.form,
                   "schedule": args.schedule if args.form == "dense" else "one_front",
                   "b_aux": (args.b_aux or wl.b) if args.form == "dense" else wl.b,
                   "precision": PRECISION_TEXT[args.precision] if args.form == "chain" else DENSE_TEXT[args.precision],
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (%.1f GB stored operators)" % (stored / 1e9)},
        "setup_s": setup_s,
        "setup_work": setup_work,
        "precond_applies_per_s": world * stats.rhs_applied / (stats.sweep_ms / 1e3) if stats.sweep_ms else None,
        "apply_ms": per_launch_ms,
        "gmres_iters": {"min": min(its), "max": max(its)},
        "relres_fp64_max": relmax,
        "status_codes": codes,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                     "peak_kind": peak_kind + " (copy bandwidth)",
                     "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": per_launch_ms},
        "chain": chain,
        "clocks": clk,
        "gpu_launches": launches,
        "stored_bytes": stored,
    }
    if flops is not None:
        line["tensor"] = {"flops_per_launch": flops, "tflops": flops / (per_launch_ms / 1e3) / 1e12,
                          "note": "complex multiply-adds x 8 (4M), per stored product term"}
    if plain is not None:
        plain["ratio_split_vs_plain"] = value / plain["value"]
        line["plain_fp32"] = plain
    if onefront is not None:
        line["one_front_b_aux_b"] = onefront
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        try:
            iters = float(np.mean(its))
            sched, b_aux = (args.schedule, args.b_aux) if args.form == "dense" else ("one_front", 0)
            slabs_per_s, workers, wall = cpu_sample(wl.n, rounds=1, schedule=sched, b_aux=b_aux)
            solves_s, applies_s = oracle_rate(wl.n, slabs_per_s, iters, sched, b_aux)
            cb = {"value": solves_s, "unit": "RHS-solves/s", "cores": workers, "kind": "oracle",
                  "sample": sample_text(wl.n, workers, iters, sched, b_aux), "seconds_per_round": wall,
                  "precond_applies_per_s": applies_s}
            # the oracle's FP64 operator on four of the GPU's solutions: their true residual
            from oracle.operator import Grid, apply_full
            g = Grid(wl.n, wl.b, wl.omega)
            c64 = wl.c.astype(np.float32).astype(np.float64)
            f64 = wl.f.astype(np.complex64).astype(np.complex128)
            res = []
            for k, r in enumerate(sample_rhs):
                ru = f64[r] - apply_full(u_sample[k].astype(np.complex128), c64, g)
                res.append(float(np.linalg.norm(ru) / np.linalg.norm(f64[r])))
            cb["oracle_residual"] = {"rhs": sample_rhs, "relres_fp64": res,
                                     "note": "||f - A u||/||f|| with the oracle's FP64 operator (Eq. system)"}
            line["cpu_baseline"] = cb
        except Exception as exc:  # keep the bench line even if the baseline fails
            line["cpu_baseline"] = {"value": None, "unit": "RHS-solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": "failed: " + str(exc)[-200:]}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_apply_only(args):
    """Setup once, then W warm-up and K timed preconditioner applies on the
    64-RHS batch (a bounded command for profiling the sweep kernel)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm
    wl = _workload(args.n, 8)
    dev = torch.device("cuda", 0)
    c = torch.from_numpy(wl.c.astype(np.float32)).to(dev)
    f = torch.from_numpy(wl.f.astype(np.complex64)).to(dev)
    z = torch.empty_like(f)
    st = torch.cuda.current_stream()
    opts = helm.helm_default_opts()
    opts.precision = helm.PRECISIONS[args.precision]
    opts.apply_form = helm.APPLY_FORMS[args.form]
    if args.form == "dense":
        opts.schedule = helm.SCHEDULES[args.schedule]
        opts.b_aux = args.b_aux
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    h = helm.helm_setup(c.data_ptr(), wl.omega, wl.n, wl.b, wl.d, opts, st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    setup_s = e0.elapsed_time(e1) / 1e3
    for _ in range(args.warmup):
        helm.helm_apply_precond(h, f.data_ptr(), z.data_ptr(), wl.R, st.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        helm.helm_apply_precond(h, f.data_ptr(), z.data_ptr(), wl.R, st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    helm.helm_status(h, st.cuda_stream)
    ms = e0.elapsed_time(e1) / args.steps
    if args.form == "dense":
        chain, alg, _ = _dense_model(wl.n, wl.b, wl.d, DENSE_ENTRY_BYTES[args.precision], args.schedule, args.b_aux)
        per = {"schedule": args.schedule, "b_aux": args.b_aux or wl.b, "us_per_solve": ms * 1e3 / chain}
    else:
        _, alg, chain = _blocks_and_bytes(wl.n, wl.b, wl.d, args.precision)
        per = {"ns_per_step": ms * 1e6 / chain}
    print(json.dumps({"mode": "apply-only", "form": args.form, "precision": args.precision, "setup_s": setup_s,
                      "stored_gb": helm.helm_factor_bytes(h) / 1e9, "n": wl.n, "rhs": wl.R, "ms_per_apply": ms,
                      "precond_applies_per_s": wl.R / (ms / 1e3), "hbm_gbs": alg / (ms / 1e3) / 1e9, **per}),
          flush=True)
    helm.helm_destroy(h)


def run_schedules(args):
    """Sweep schedules at the 64-source workload (Section 4.2's third
    modification): one front with b_aux = b, one front with a thinner
    auxiliary PML, and two fronts in both loops (b_aux = 2 is the headline) (whose centre windows
    extend b_aux to both sides, so b_aux <= 3 keeps the quasi-1D blocks <= 64;
    the two inner fronts run side by side).
    One JSON line per configuration: setup, stored bytes, GMRES iterations,
    FP64 residual, solve time of the 64 right-hand sides."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm
    wl = _workload(args.n, 8)
    dev = torch.device("cuda", 0)
    c = torch.from_numpy(wl.c.astype(np.float32)).to(dev)
    f = torch.from_numpy(wl.f.astype(np.complex64)).to(dev)
    u = torch.empty_like(f)
    st = torch.cuda.current_stream()
    for sched, b_aux in (("one_front", 0), ("one_front", 3), ("two_front", 3), ("two_front", 2)):
        opts = helm.helm_default_opts()
        opts.precision = helm.PRECISIONS[args.precision]
        opts.apply_form = helm.APPLY_FORMS["dense"]
        opts.schedule = helm.SCHEDULES[sched]
        opts.b_aux = b_aux
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        h = helm.helm_setup(c.data_ptr(), wl.omega, wl.n, wl.b, wl.d, opts, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        setup_s = e0.elapsed_time(e1) / 1e3
        helm.helm_solve(h, f.data_ptr(), u.data_ptr(), wl.R, TOL, st.cuda_stream)      # warm-up
        helm.helm_enable_timing(h, True)
        helm.helm_reset_stats(h)
        e1.record(st)
        code, its, rel = helm.helm_solve(h, f.data_ptr(), u.data_ptr(), wl.R, TOL, st.cuda_stream)
        e2.record(st)
        torch.cuda.synchronize()
        sp = helm.helm_get_stats(h)
        solve_s = e1.elapsed_time(e2) / 1e3
        print(json.dumps({"mode": "schedule", "schedule": sched, "b_aux": b_aux or wl.b, "n": wl.n, "rhs": wl.R,
                          "precision": args.precision, "setup_s": setup_s,
                          "stored_gb": helm.helm_factor_bytes(h) / 1e9, "gmres_iters": [int(min(its)), int(max(its))],
                          "relres_fp64_max": float(max(rel)), "status": int(code), "solve_s": solve_s,
                          "rhs_solves_per_s": wl.R / solve_s,
                          "apply_ms": sp.sweep_ms / max(sp.sweep_launches, 1)}), flush=True)
        helm.helm_destroy(h)


def run_batch(args):
    """Six uneven problems (n = 63..159, b = 5, 8-32 sources each): one batched
    preconditioner launch over all of them against the six separate applies
    issued one after the other on the same stream."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm, workloads as W
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()
    opts = helm.helm_default_opts()
    opts.precision = helm.PRECISIONS[args.precision]
    hs, fs, zs, setup_s, fbytes, shapes = [], [], [], 0.0, 0, []
    for wl in W.uneven_batch():
        shapes.append([wl.n, wl.b, wl.R])
        c = torch.from_numpy(wl.c.astype(np.float32)).to(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h = helm.helm_setup(c.data_ptr(), wl.omega, wl.n, wl.b, wl.d, opts, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        setup_s += e0.elapsed_time(e1) / 1e3
        fbytes += helm.helm_factor_bytes(h)
        f = torch.from_numpy(wl.f.astype(np.complex64)).to(dev)
        hs.append(h), fs.append(f), zs.append(torch.empty_like(f))
        del c
    nrhs = [f.shape[0] for f in fs]

    def batched():
        helm.helm_apply_batch(hs, [f.data_ptr() for f in fs], [z.data_ptr() for z in zs], nrhs, st.cuda_stream)

    def separate():
        for h, f, z, r in zip(hs, fs, zs, nrhs):
            helm.helm_apply_precond(h, f.data_ptr(), z.data_ptr(), r, st.cuda_stream)

    out = {}
    for name, fn in (("batched", batched), ("separate", separate)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / args.steps / 1e3
    codes = [helm.helm_status(h, st.cuda_stream) for h in hs]
    for h in hs:
        helm.helm_destroy(h)
    R = sum(nrhs)
    print(json.dumps({"mode": "batch", "problems": shapes,
                      "rhs_total": R, "precision": args.precision, "factor_gb": fbytes / 1e9,
                      "setup_s_total": setup_s, "batched_s_per_apply": out["batched"],
                      "separate_s_per_apply": out["separate"],
                      "batched_precond_applies_per_s": R / out["batched"],
                      "separate_precond_applies_per_s": R / out["separate"],
                      "status_codes": codes}), flush=True)


def run_stencil(args):
    """The PML stencil matvec (a2) on the 64-source workload in c64 and c128:
    CUDA-event time per launch and achieved HBM bandwidth for its algorithmic
    bytes (read x, write y per point and right-hand side; kappa once)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm
    wl = _workload(args.n, 8)
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()
    c = torch.from_numpy(wl.c.astype(np.float32)).to(dev)
    h = helm.helm_setup(c.data_ptr(), wl.omega, wl.n, wl.b, wl.d, None, st.cuda_stream)
    n3 = wl.N ** 3
    peak, peak_kind = _peaks()
    out = {"mode": "stencil", "n": wl.n, "rhs": wl.R, "peak_gbs": peak, "peak_kind": peak_kind}
    for name, dt, fp64, kbytes in (("c64", torch.complex64, 0, 4), ("c128", torch.complex128, 1, 8)):
        x = torch.randn(wl.R, wl.N, wl.N, wl.N, dtype=dt, device=dev)
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            helm.helm_matvec(h, x.data_ptr(), y.data_ptr(), wl.R, fp64, st.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(args.steps, 10)
        e0.record(st)
        for _ in range(reps):
            helm.helm_matvec(h, x.data_ptr(), y.data_ptr(), wl.R, fp64, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        alg = 2 * wl.R * n3 * x.element_size() + n3 * kbytes
        out[name] = {"ms_per_launch": ms, "algorithmic_bytes": alg, "achieved_gbs": alg / (ms / 1e3) / 1e9,
                     "frac": alg / (ms / 1e3) / 1e9 / peak}
        del x, y
    helm.helm_destroy(h)
    print(json.dumps(out), flush=True)


def run_grad(args):
    """Differentiation pattern: loss 1/2 sum |u_rec - d|^2 over 16 sources at
    n = 63 (lens plus a bump; data from the unperturbed lens, receivers on the
    z = 0.9 plane) and its velocity gradient through the autograd wrapper
    (forward setup + solve, adjoint solve, fused gradient kernel)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import workloads as W
    from paper_1502_07266_gb300.autograd import helmholtz_solve
    wl = W.lens_bump_16_sources()
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()
    f = torch.from_numpy(wl.f.astype(np.complex64)).to(dev)
    c_obs = torch.from_numpy(wl.meta["c_obs"].astype(np.float32)).to(dev)
    rec = wl.meta["rec_plane"]
    with torch.no_grad():
        d_obs = helmholtz_solve(c_obs, f, wl.omega, wl.n, wl.b, wl.d)[:, rec].clone()
    c0 = torch.from_numpy(wl.c.astype(np.float32)).to(dev)

    def step():
        c = c0.clone().requires_grad_(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(st)
        u = helmholtz_solve(c, f, wl.omega, wl.n, wl.b, wl.d)
        loss = 0.5 * (u[:, rec] - d_obs).abs().pow(2).sum()
        ev[1].record(st)
        loss.backward()
        ev[2].record(st)
        return ev, loss, c.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    runs = [step() for _ in range(args.steps)]
    e1.record(st)
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1) / args.steps / 1e3
    fwd = sum(r[0][0].elapsed_time(r[0][1]) for r in runs) / args.steps / 1e3
    bwd = sum(r[0][1].elapsed_time(r[0][2]) for r in runs) / args.steps / 1e3
    g = runs[-1][2]
    print(json.dumps({"mode": "grad", "n": wl.n, "b": wl.b, "sources": wl.R, "receiver_plane": rec,
                      "s_per_gradient": total, "gradients_per_s": 1.0 / total,
                      "forward_s": fwd, "backward_s": bwd, "loss": float(runs[-1][1].detach()),
                      "grad_norm": float(g.norm()), "grad_finite": bool(torch.isfinite(g).all())}),
          flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=127, help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=sorted(ENTRY_BYTES), default="split_fp16",
                    help="stored form of the factors or operators (the precision pattern)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain complex-FP32 comparison")
    ap.add_argument("--form", choices=["chain", "dense"], default="dense",
                    help="apply form: block substitution chain or dense restricted operators")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", choices=["one_front", "two_front"], default=DEFAULT_SCHEDULE,
                    help="sweep schedule of the dense form (two fronts: Section 5's)")
    ap.add_argument("--b-aux", type=int, default=DEFAULT_B_AUX,
                    help="auxiliary PML thickness of the moving windows (0: b)")
    ap.add_argument("--stencil", action="store_true",
                    help="stencil matvec bandwidth at n=127, 64 RHS (prints its own JSON)")
    ap.add_argument("--grad", action="store_true",
                    help="loss and velocity gradient for 16 sources at n=63 (prints its own JSON)")
    ap.add_argument("--schedules", action="store_true",
                    help="one front (b_aux = b and 3) against two fronts (b_aux = 3 and 2) at the 64-source workload")
    ap.add_argument("--batch", action="store_true",
                    help="six uneven problems: one batched apply vs separate applies (prints its own JSON)")
    ap.add_argument("--apply-only", action="store_true",
                    help="setup once, then time preconditioner applies only (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.stencil:
        run_stencil(args)
    elif args.grad:
        run_grad(args)
    elif args.schedules:
        run_schedules(args)
    elif args.batch:
        run_batch(args)
    elif args.apply_only:
        run_apply_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
