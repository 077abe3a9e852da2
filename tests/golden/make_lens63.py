"""Writes lens63_solution.json: the FP64 oracle's solution of the lens workload
(n = 63, b = 6, d = 1, 8 points per wavelength, one Gaussian source at
(0.5, 0.5, 0.25)) sampled at seeded grid points.

Calls only the oracle (the discretisation of Sec. 2, the sweep of Alg. 6 over
Alg. 4, right-preconditioned GMRES of Sec. 5) and the seeded input generators.
The velocity is rounded to FP32 first, as the GPU path receives it.  About
20 minutes on one host core:  python tests/golden/make_lens63.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.krylov import gmres                       # noqa: E402
from oracle.operator import Grid, apply_full          # noqa: E402
from oracle.sweep import SweepPreconditioner          # noqa: E402
from paper_1502_07266_gb300 import workloads as W    # noqa: E402

SAMPLES = 2048
TOL = 1e-10


def main():
    wl = W.lens_one_source(63, 6, 1)
    c = wl.c.astype(np.float32).astype(np.float64)
    f = wl.f[0].astype(np.complex64).astype(np.complex128)
    g = Grid(wl.n, wl.b, wl.omega)
    t0 = time.time()
    P = SweepPreconditioner(c, g, d=wl.d).setup()
    t_setup = time.time() - t0
    t0 = time.time()
    u, its, hist = gmres(lambda v: apply_full(v, c, g), P.apply, f, tol=TOL)
    t_solve = time.time() - t0
    relres = float(np.linalg.norm(f - apply_full(u, c, g)) / np.linalg.norm(f))
    N = wl.N
    rng = np.random.default_rng(63)
    flat = rng.choice(N ** 3, size=SAMPLES, replace=False)
    flat = np.union1d(flat, [int(np.argmax(np.abs(u)))])
    uf = u.ravel()
    out = {
        "what": "FP64 oracle solution, lens n=63 b=6 d=1, 8 ppw, Gaussian source at (0.5,0.5,0.25), "
                "velocity rounded to FP32; values at seeded flat indices of the (N,N,N) padded grid (z,y,x)",
        "n": wl.n, "b": wl.b, "d": wl.d, "omega": wl.omega, "N": N,
        "gmres_tol": TOL, "restart": 30, "iterations": int(its), "relres_fp64": relres,
        "norm_u": float(np.linalg.norm(uf)), "norm_f": float(np.linalg.norm(f)),
        "oracle_seconds": {"setup": round(t_setup, 1), "solve": round(t_solve, 1)},
        "index": [int(i) for i in flat],
        "re": [float(uf[i].real) for i in flat],
        "im": [float(uf[i].imag) for i in flat],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lens63_solution.json"), "w") as fh:
        json.dump(out, fh, indent=0)
    print("iterations", its, "relres", relres, "setup", t_setup, "solve", t_solve)


if __name__ == "__main__":
    main()
