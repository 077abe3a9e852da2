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


@pytest.mark.parametrize("n,b,d", [(5, 2, 1), (6, 3, 2), (7, 3, 1), (4, 1, 1)])
def test_dense_operator_bytes_per_apply(monkeypatch, n, b, d):
    """The dense form's work model: one stored operator read per quasi-1D
    solve of the oracle's Algorithm 6, sized from the oracle's own windows:
    line blocks M' >= 1 map their lines x every z row of the slab window to
    themselves; the first line block maps its lines x the slab's own layers
    to those entries plus the line that couples to M' = 1 (forward), and
    that line to its lines x own layers (backward)."""
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    P = SweepPreconditioner(c, g, d=d).setup()
    ident = {id(q): (M, Mp) for M in range(P.B) for Mp, q in enumerate(P.slab_problems(M))}
    calls = []
    orig = Quasi1D.restricted_apply

    def counting(self, alpha):
        calls.append(ident[id(self)])
        return orig(self, alpha)

    monkeypatch.setattr(Quasi1D, "restricted_apply", counting)
    P.apply(W.random_rhs(1, n, b, seed=1))
    N, B = g.N, P.B
    per = 2 * B - 1
    total = macs = 0
    for s, (M, Mp) in enumerate(calls):
        bwd = (s % per) >= B                      # each slab visit: B forward solves, then B-1 backward
        assert Mp == ((s % per) if not bwd else 2 * B - 2 - (s % per))
        pz, (za, zb) = P.zwin[M]
        py, (ia, ib) = P.ywin[Mp]
        if Mp >= 1:
            n_in = n_out = (ib - ia) * pz.L * N
        elif not bwd:
            n_in = b * (zb - za) * N
            n_out = ((b - 1) * (zb - za) + pz.L) * N
        else:
            n_in = pz.L * N
            n_out = b * (zb - za) * N
        total += n_out * n_in * 8
        macs += n_out * n_in
    nsolves, alg, mc = bench._dense_model(n, b, d)
    assert nsolves == len(calls) == per ** 2
    assert (alg, mc) == (total, macs)
    assert bench._dense_model(n, b, d, entry_bytes=4)[1] * 2 == alg


@pytest.mark.parametrize("n,b,d,b_aux", [(5, 2, 1, 2), (7, 3, 1, 2), (8, 2, 2, 1)])
def test_dense_operator_bytes_two_front(monkeypatch, n, b, d, b_aux):
    """The same model for the two-front schedule, counted on the oracle's
    two-front sweep: both boundary line blocks have the reduced forward and
    backward maps, the centre line block has no backward solve, and the
    centre slab is visited once."""
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    P = SweepPreconditioner(c, g, d=d, b_aux=b_aux, schedule="two_front").setup()
    ident = {id(q): (M, Mp) for M in range(P.B) for Mp, q in enumerate(P.slab_problems(M))}
    calls = []
    orig = Quasi1D.restricted_apply

    def counting(self, alpha):
        calls.append(ident[id(self)])
        return orig(self, alpha)

    monkeypatch.setattr(Quasi1D, "restricted_apply", counting)
    P.apply(W.random_rhs(1, n, b, seed=1))
    N, B = g.N, P.B
    per = 2 * B - 1
    total = 0
    for s, (M, Mp) in enumerate(calls):
        bwd = (s % per) >= B                      # each visit: B forward solves, then B-1 backward
        pz, (za, zb) = P.zwin[M]
        py, (ia, ib) = P.ywin[Mp]
        if 0 < Mp < B - 1:
            n_in = n_out = (ib - ia) * pz.L * N
        elif not bwd:
            n_in = b * (zb - za) * N
            n_out = ((b - 1) * (zb - za) + pz.L) * N
        else:
            n_in = pz.L * N
            n_out = b * (zb - za) * N
        total += n_out * n_in * 8
    nsolves, alg, _ = bench._dense_model(n, b, d, schedule="two_front", b_aux=b_aux)
    assert nsolves == len(calls) == per ** 2
    assert alg == total


@pytest.mark.parametrize("schedule,b_aux", [("one_front", 0), ("two_front", 2), ("two_front", 3)])
def test_cpu_baseline_scaling_follows_the_schedule(schedule, b_aux):
    """The oracle baseline scales a slab solve to an apply by the slab visits of
    Algorithm 6 under the schedule: 2B - 1 with B the oracle's own block count on
    the workload's z axis (b = 6, d = 1)."""
    from oracle.sweep import axis_schedule
    n = 127
    blocks, roles, c = axis_schedule(n + 12, 6, 1, schedule)
    B = len(blocks)
    assert bench._nblocks(n, schedule, b_aux) == B
    # the oracle's own outer sweep visits 2B - 1 slabs (counted on a small grid of the same rule)
    ns = 9
    P = SweepPreconditioner(W.velocity_lens(ns, 6), Grid(ns, 6, W.omega_for(ns)), d=1, b_aux=b_aux or None,
                            schedule=schedule)
    visits = []
    P.sweep(lambda M, rhs: visits.append(M) or np.zeros_like(rhs), np.zeros((ns + 12,) * 3, dtype=np.complex128), axis=0)
    assert len(visits) == 2 * bench._nblocks(ns, schedule, b_aux) - 1
    solves, applies = bench.oracle_rate(n, 514.0, 2.0, schedule, b_aux)
    assert applies == pytest.approx(514.0 / (2 * B - 1)) and solves == pytest.approx(applies / 2.0)
    text = bench.sample_text(n, 16, 24.0, schedule, b_aux)
    assert f"{2 * B - 1} slab solves per apply" in text and f"b_aux={b_aux or 6}" in text


def test_dense_setup_model():
    """The factorisation term reproduces the a4 setup count (8 k^3 N_x per
    problem, 2.35e12 flops at n = 127 with one front and b_aux = b, where the
    interior blocks have k = 49); the thin two-front windows need far less."""
    fac, ops = bench._dense_setup_model(127, 6, 1, "one_front", 0)
    assert fac == pytest.approx(2.35e12, rel=0.01)
    # restricted operators: 2 N k^2 complex multiply-adds per input column, k = 49, 973 columns
    assert ops > 17000 * 16 * 139 * 49 ** 2 * 973
    fac2, ops2 = bench._dense_setup_model(127, 6, 1, "two_front", 2)
    assert fac2 + ops2 < (fac + ops) / 20
