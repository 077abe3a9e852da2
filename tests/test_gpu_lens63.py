"""The lens workload (n = 63, b = 6, d = 1, 8 points per wavelength, one
Gaussian source at (0.5, 0.5, 0.25)) solved on the GPU and compared with the
FP64 oracle's solution.

The oracle's solution (right-preconditioned GMRES of Sec. 5 with the sweep of
Alg. 6 over Alg. 4, tolerance 1e-10, FP64) takes about ten minutes on a host
core, so it is stored: `tests/golden/lens63_solution.json`, written by
`tests/golden/make_lens63.py` (oracle calls only), holds its values at 2049
seeded grid points and its 2-norm.  The GPU solves at the workload's tolerance
1e-6 in every stored form; the comparison is on the sampled points (relative
2-norm error <= 1e-5) and on the norm, plus the true FP64 residual of the
whole GPU solution under the oracle's operator (Eq. system).
"""
import json
import os
import time

import numpy as np
import pytest

from oracle.operator import Grid, apply_full
from paper_1502_07266_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lens63_solution.json")


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm as H
    return H


@pytest.fixture(scope="module")
def case():
    gold = json.load(open(GOLDEN))
    wl = W.lens_one_source(gold["n"], gold["b"], gold["d"])
    assert wl.N == gold["N"] and abs(wl.omega - gold["omega"]) < 1e-12
    return wl, gold


@pytest.mark.parametrize("form,precision", [("chain", "fp32"), ("dense", "fp32"), ("dense", "split_fp16")])
def test_lens63_solution_matches_fp64_oracle(helm, case, form, precision):
    wl, gold = case
    c32 = wl.c.astype(np.float32)
    f = torch.from_numpy(wl.f.astype(np.complex64)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = helm.Solver(torch.from_numpy(c32).cuda(), wl.omega, wl.n, wl.b, wl.d, precision=precision,
                    apply_form=form)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    try:
        u, its, rel, code = S.solve(f, tol=1e-6)
        assert code == helm.HELM_OK
        ug = u.cpu().numpy()[0].astype(np.complex128)
    finally:
        S.close()
    idx = np.asarray(gold["index"])
    uo = np.asarray(gold["re"]) + 1j * np.asarray(gold["im"])
    us = ug.ravel()[idx]
    err_sample = np.linalg.norm(us - uo) / np.linalg.norm(uo)
    err_norm = abs(np.linalg.norm(ug) - gold["norm_u"]) / gold["norm_u"]
    g = Grid(wl.n, wl.b, wl.omega)
    f64 = wl.f[0].astype(np.complex64).astype(np.complex128)
    relres = np.linalg.norm(f64 - apply_full(ug, c32.astype(np.float64), g)) / np.linalg.norm(f64)
    print(f"\nlens63 {form}/{precision}: setup {t_setup:.2f} s, {int(its[0])} iterations "
          f"(oracle {gold['iterations']} at 1e-10), sampled error vs FP64 oracle {err_sample:.2e}, "
          f"norm error {err_norm:.2e}, FP64 residual of the FP32 solution {relres:.2e}")
    assert err_sample <= 1e-5
    assert err_norm <= 1e-5
    assert relres <= 3e-6
