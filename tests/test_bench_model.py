"""The bench's work model against the oracle: the algorithmic factor bytes of
one preconditioner apply (the roofline numerator) and the number of quasi-1D
solves are counted from the sweeps themselves, independently of the closed
form in bench.py."""
import collections

import numpy as np
import pytest

import bench
from oracle.operator import Grid
from oracle.sweep import Quasi1D, SweepPreconditioner
from paper_1502_07266_gb300 import workloads as W


@pytest.mark.parametrize("n,b,d", [(5, 2, 1), (6, 3, 2), (7, 3, 1)])
def test_factor_bytes_and_solves_per_apply(monkeypatch, n, b, d):
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    P = SweepPreconditioner(c, g, d=d).setup()
    uses = collections.Counter()
    orig = Quasi1D.restricted_apply

    def counting(self, alpha):
        uses[(self.Ly, self.Lz, id(self))] += 1
        return orig(self, alpha)

    monkeypatch.setattr(Quasi1D, "restricted_apply", counting)
    P.apply(W.random_rhs(1, n, b, seed=1))
    N = g.N
    solves = sum(uses.values())
    bytes_counted = sum(cnt * N * (Ly * Lz) ** 2 * 8 for (Ly, Lz, _), cnt in uses.items())
    B, alg, chain = bench._blocks_and_bytes(n, b, d)
    assert B == P.B
    assert solves == (2 * B - 1) ** 2            # every outer slab visit runs 2B-1 inner solves
    assert bytes_counted == alg                  # each solve reads its N blocks of k x k once
    m = (N - 1) // 2
    assert chain == solves * (2 * max(m, N - 1 - m) + 1)
    # FP16 storage halves the bytes
    assert bench._blocks_and_bytes(n, b, d, "fp16")[1] * 2 == alg
