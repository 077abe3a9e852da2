"""Benchmark: RHS-solves/s and preconditioner applies/s for the recursive
moving-PML sweeping preconditioner with GMRES, on the 64-source workload.

Workload (the configuration the headline metric is quoted on): n = 127
interior points per axis, b = 6 PML layers on every face (139^3 unknowns),
d = 1, omega = 2 pi 127 / 8 (8 points per wavelength), smooth random velocity
in [1, 2] (seed 0), 64 Gaussian sources on an 8 x 8 grid of the z = 0.1 plane,
GMRES(30) to a true relative residual of 1e-6.  Synthetic inputs, seeded.

A step is one pass of the whole hot path over the 64-RHS batch: helm_setup
(coefficients, every quasi-1D factorisation) then helm_solve (GMRES with the
recursive sweep, stencil and FP64 residuals).  Inputs are resident in HBM for
`value`; `e2e` repeats one step through pinned host buffers.  The factors
(56.5 GB in FP32, 29 GB in FP16) exceed L2, so no flush is needed between steps.

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
# GMRES iterations the GPU path takes on this workload (measured); used only
# to scale the CPU oracle's timed sample to RHS-solves/s.
NOMINAL_ITERS = 22


def _workload(n: int, per_side: int):
    from paper_1502_07266_gb300 import workloads as W
    return W.random_64_sources(n=n, b=6, d=1, seed=0, per_side=per_side)


ENTRY_BYTES = {"fp32": 8, "fp16": 4, "split_fp16": 8}   # stored bytes per complex factor entry
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

def cpu_sample(n: int, slabs: int, seed: int = 3):
    """Times the FP64 oracle on a bounded sample of the workload: the quasi-2D
    solve (Algorithm 4, refactoring its quasi-1D problems) of `slabs` interior
    slabs for one right-hand side.  Returns seconds per slab."""
    import numpy as np

    from oracle.operator import Grid
    from oracle.sweep import SweepPreconditioner
    wl = _workload(n, 1)
    g = Grid(wl.n, wl.b, wl.omega)
    c64 = wl.c.astype(np.float32).astype(np.float64)
    P = SweepPreconditioner(c64, g, d=wl.d, keep_factors=False)
    rng = np.random.default_rng(seed)
    mid = P.B // 2
    t0 = time.perf_counter()
    for s in range(slabs):
        M = mid + s
        pz, (za, zb) = P.zwin[M]
        alpha = rng.standard_normal((1, zb - za, P.N, P.N)) + 1j * rng.standard_normal((1, zb - za, P.N, P.N))
        P.slab_apply(M, alpha)
    return (time.perf_counter() - t0) / slabs


def cpu_baseline_subprocess(n: int, slabs: int):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--n", str(n),
                          "--slabs", str(slabs)], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return float(out.stdout.strip().splitlines()[-1])


def oracle_rate(n: int, t_slab: float):
    B, _, _ = _blocks_and_bytes(n, 6, 1)
    per_apply = (2 * B - 1) * t_slab            # seconds per single-RHS preconditioner apply
    return 1.0 / (NOMINAL_ITERS * per_apply), 1.0 / per_apply


def sample_text(n: int, slabs: int):
    B, _, _ = _blocks_and_bytes(n, 6, 1)
    return (f"FP64 oracle, {slabs} interior slab(s) of Algorithm 4 for 1 RHS (each refactoring its {B} "
            f"quasi-1D problems) at n={n}; scaled by {2 * B - 1} slab solves per apply and "
            f"{NOMINAL_ITERS} GMRES iterations per RHS-solve (GMRES vector work not counted)")


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
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    times = []
    for s in range(args.warmup + args.steps):
        t = cpu_baseline_subprocess(n, 1)
        if s >= args.warmup:
            times.append(t)
    t_slab = sum(times) / len(times)
    solves_s, applies_s = oracle_rate(n, t_slab)
    line = {
        "impl": "reference", "metric": METRIC, "value": solves_s, "unit": "RHS-solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_slab * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": f"n={n} b=6 d=1 random velocity, 64 sources (8x8, z=0.1), tol 1e-6",
                   "l2": "inputs larger than L2"},
        "precond_applies_per_s": applies_s,
        "cpu_baseline": {"value": solves_s, "unit": "RHS-solves/s", "cores": 1, "kind": "oracle",
                         "sample": sample_text(n, 1)},
        "e2e": {"value": solves_s, "unit": "RHS-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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

    results = {}

    opts = helm.helm_default_opts()
    opts.precision = helm.PRECISIONS[args.precision]

    def step(c_t, f_t, u_t, timing=False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(st)
        h = helm.helm_setup(c_t.data_ptr(), wl.omega, wl.n, wl.b, wl.d, opts, st.cuda_stream)
        ev[1].record(st)
        if timing:
            helm.helm_enable_timing(h, True)
        code, its, rel = helm.helm_solve(h, f_t.data_ptr(), u_t.data_ptr(), R, TOL, st.cuda_stream)
        ev[2].record(st)
        stats = helm.helm_get_stats(h) if timing else None
        launches = helm.helm_launch_count(h)
        fb = helm.helm_factor_bytes(h)
        helm.helm_destroy(h)
        return dict(code=code, its=its, rel=rel, ev=ev, stats=stats, launches=launches, factor_bytes=fb)

    for _ in range(args.warmup):
        step(c_dev, f_dev, u_dev)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    barrier()
    t_start.record(st)
    runs = [step(c_dev, f_dev, u_dev, timing=True) for _ in range(args.steps)]
    t_stop.record(st)
    barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(t_start.elapsed_time(t_stop) / 1e3, dist, dev)

    setup_s = sum(r["ev"][0].elapsed_time(r["ev"][1]) for r in runs) / len(runs) / 1e3
    solve_s = sum(r["ev"][1].elapsed_time(r["ev"][2]) for r in runs) / len(runs) / 1e3
    sweep_launches = sum(r["stats"].sweep_launches for r in runs)
    sweep_ms = sum(r["stats"].sweep_ms for r in runs)
    rhs_applied = sum(r["stats"].rhs_applied for r in runs)
    launches = sum(r["launches"] for r in runs)
    its = runs[-1]["its"]
    relmax = max(max(r["rel"]) for r in runs)
    codes = sorted({r["code"] for r in runs})

    # e2e: the same step from pinned host buffers, copies inside the timed region
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
        step(c_t, f_t, u_t)
        u_host.copy_(u_t, non_blocking=True)
        e1.record(st)
        barrier()
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        e2e = {"value": replica_rate(world, R, 1, te), "unit": "RHS-solves/s",
               "h2d_bytes_per_step": c_host.numel() * 4 + f_host.numel() * 8,
               "d2h_bytes_per_step": u_host.numel() * 8}
        del c_t, f_t, u_t

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    B, alg_bytes, chain_steps = _blocks_and_bytes(wl.n, wl.b, wl.d, args.precision)
    per_launch_ms = sweep_ms / max(sweep_launches, 1)
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    value = replica_rate(world, R, args.steps, elapsed)
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
        "dtype": "c64",
        "data": "synthetic",
        "config": {"workload": f"n={wl.n} b={wl.b} d={wl.d} ({N}^3), random velocity seed 0, "
                               f"{R} Gaussian sources (8x8, z=0.1), GMRES(30) tol {TOL}",
                   "precision": PRECISION_TEXT[args.precision],
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (%.1f GB factors)" % (runs[-1]["factor_bytes"] / 1e9)},
        "precond_applies_per_s": world * rhs_applied / (sweep_ms / 1e3) if sweep_ms else None,
        "setup_s": setup_s,
        "solve_s": solve_s,
        "gmres_iters": {"min": min(its), "max": max(its)},
        "relres_fp64_max": relmax,
        "status_codes": codes,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _traffic_per_launch(wl.n),
                     "kernel": "k_sweep (preconditioner apply)", "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": per_launch_ms},
        "chain": {"dependent_steps_per_apply": chain_steps,
                  "ns_per_step": per_launch_ms * 1e6 / chain_steps},
        "clocks": clk,
        "gpu_launches": launches,
        "factor_bytes": runs[-1]["factor_bytes"],
    }
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world >= 1:
        try:
            slabs = args.cpu_slabs
            t_slab = cpu_baseline_subprocess(wl.n, slabs)
            solves_s, applies_s = oracle_rate(wl.n, t_slab)
            line["cpu_baseline"] = {"value": solves_s, "unit": "RHS-solves/s", "cores": 1, "kind": "oracle",
                                    "sample": sample_text(wl.n, slabs), "seconds_per_slab": t_slab,
                                    "precond_applies_per_s": applies_s}
        except Exception as exc:  # keep the bench line even if the baseline fails
            line["cpu_baseline"] = {"value": None, "unit": "RHS-solves/s", "cores": 1, "kind": "oracle",
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
    h = helm.helm_setup(c.data_ptr(), wl.omega, wl.n, wl.b, wl.d, opts, st.cuda_stream)
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
    B, alg, chain = _blocks_and_bytes(wl.n, wl.b, wl.d, args.precision)
    print(json.dumps({"mode": "apply-only", "n": wl.n, "rhs": wl.R, "ms_per_apply": ms,
                      "precond_applies_per_s": wl.R / (ms / 1e3), "hbm_gbs": alg / (ms / 1e3) / 1e9,
                      "ns_per_step": ms * 1e6 / chain}), flush=True)
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
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=127, help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=sorted(ENTRY_BYTES), default="fp32",
                    help="stored form of the quasi-1D factors (the precision pattern)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-slabs", type=int, default=3)
    ap.add_argument("--stencil", action="store_true",
                    help="stencil matvec bandwidth at n=127, 64 RHS (prints its own JSON)")
    ap.add_argument("--grad", action="store_true",
                    help="loss and velocity gradient for 16 sources at n=63 (prints its own JSON)")
    ap.add_argument("--batch", action="store_true",
                    help="six uneven problems: one batched apply vs separate applies (prints its own JSON)")
    ap.add_argument("--apply-only", action="store_true",
                    help="setup once, then time preconditioner applies only (profiling)")
    ap.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--slabs", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3 and not args.cpu_worker:
        ap.error("--warmup must be at least 3")
    if args.cpu_worker:
        print(cpu_sample(args.n, args.slabs))
        return
    if args.stencil:
        run_stencil(args)
    elif args.grad:
        run_grad(args)
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
