"""Host-side test of the dense apply's step schedule (csrc/dense_sched.h).

The kernel walks Algorithm 6 over Algorithm 4 as a sequence of steps, two
quasi-1D solves side by side in the two-front schedule (Sec. 4.2, third
modification).  The schedule header is compiled for the host here and its
step list is checked against the oracle's own sweep (oracle.sweep.sweep):
the same outer order, every inner solve exactly once, each solve after the
solves whose values its right-hand side reads, and the cluster split of a
step between the lower and the upper front.  No GPU is needed."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.operator import Grid
from oracle.sweep import SweepPreconditioner
from paper_1502_07266_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1502_07266_gb300", "csrc", "dense_sched.h")

DRIVER = r'''
#define __host__
#define __device__
#define __forceinline__ inline
#include <cstdio>
#include <cstdlib>
namespace {
#include "dense_sched.h"
}
int main(int argc, char** argv) {
    const int B = atoi(argv[1]), c = atoi(argv[2]), two = atoi(argv[3]), nclus = atoi(argv[4]);
    const int spv = inner_steps(B, c, two) + 1;
    const int nsteps = (2 * B - 1) * spv + 1;
    printf("%d %d %d\n", spv, nsteps, dense_nops(B));
    for (int j = 0; j < 2 * B - 1; ++j) {
        const PassPos q = pass_pos(j, B, c);
        printf("P %d %d %d %d\n", j, q.M, q.bwd, q.role);
    }
    for (int s = 0; s < nsteps; ++s)
        for (int cid = 0; cid < nclus; ++cid) {
            const StepInfo t = step_info(s, B, c, two, cid, nclus);
            printf("S %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", s, cid, t.phase, t.jo, t.k, t.o.M, t.o.Mp,
                   t.o.od, t.o.id, t.o.rz, t.o.ry, t.o.p, t.mcid, t.mncl);
        }
    return 0;
}
'''


@pytest.fixture(scope="module")
def driver():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "sched.cpp")
    open(src, "w").write(DRIVER)
    exe = os.path.join(d, "sched")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.dirname(HDR), src, "-o", exe], check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run(exe, B, c, two, nclus):
    out = subprocess.run([exe, str(B), str(c), str(two), str(nclus)], capture_output=True, text=True,
                         check=True).stdout.split("\n")
    spv, nsteps, nops = map(int, out[0].split())
    passes, steps = [], []
    for line in out[1:]:
        if line.startswith("P "):
            passes.append(tuple(map(int, line.split()[1:])))
        elif line.startswith("S "):
            steps.append(tuple(map(int, line.split()[1:])))
    return spv, nsteps, nops, passes, steps


def oracle_order(n, b, schedule):
    """(block, direction) sequence of one sweep of the oracle along an axis, and
    its block count and centre."""
    P = SweepPreconditioner(W.velocity_lens(n, b), Grid(n, b, W.omega_for(n)), d=1, b_aux=1,
                            schedule=schedule)
    seq = []
    P.sweep(lambda M, rhs: seq.append(M) or np.zeros_like(rhs), np.zeros((n + 2 * b,) * 3, np.complex128), axis=0)
    B, c = P.B, P.centre
    return [(M, 0 if q < B else 1) for q, M in enumerate(seq)], B, c


def deps(Mp, bwd, B, c):
    """Solves whose values the right-hand side of solve (Mp, bwd) reads in the
    oracle's sweep: forward, the neighbour swept before it (below for the lower
    front and the centre, above for the upper front and the centre); backward,
    the block's own forward value and the neighbour its pass comes from."""
    if not bwd:
        out = []
        if 0 < Mp <= c:
            out.append((Mp - 1, 0))
        if c <= Mp < B - 1:
            out.append((Mp + 1, 0))
        return out
    nb = Mp + 1 if Mp < c else Mp - 1
    return [(Mp, 0), (nb, 0 if nb == c else 1)]


@pytest.mark.parametrize("n,b,schedule,nclus", [(9, 3, "two_front", 15), (9, 3, "two_front", 2),
                                                (10, 2, "two_front", 3), (7, 3, "one_front", 15),
                                                (6, 2, "one_front", 4)])
def test_kernel_schedule_follows_the_oracle_sweep(driver, n, b, schedule, nclus):
    order, B, c = oracle_order(n, b, schedule)
    two = schedule == "two_front"
    spv, nsteps, nops, passes, steps = run(driver, B, c, int(two), nclus)
    # the outer order: pass positions are the oracle's sweep order
    assert [(M, bwd) for _, M, bwd, _ in passes] == order
    assert nsteps == (2 * B - 1) * spv + 1
    by_step = {}
    for (s, cid, phase, jo, k, M, Mp, od, iid, rz, ry, p, mcid, mncl) in steps:
        assert jo == s // spv and k == s % spv and phase == (k == 0)
        by_step.setdefault(s, []).append((cid, phase, M, Mp, od, iid, rz, ry, p, mcid, mncl))
    ncA = (nclus + 1) // 2
    seen_p = {}
    for jo in range(2 * B - 1):
        M_o, od_o = order[jo]
        when = {}                                   # inner solve -> step
        for k in range(1, spv):
            s = jo * spv + k
            rows = by_step[s]
            solves = {}
            for (cid, phase, M, Mp, od, iid, rz, ry, p, mcid, mncl) in rows:
                assert not phase and (M, od) == (M_o, od_o)
                assert 0 <= p < nops
                assert seen_p.setdefault((M, Mp, iid), p) == p
                solves.setdefault((Mp, iid), []).append((cid, mcid, mncl))
            assert 1 <= len(solves) <= (2 if two else 1)
            if len(solves) == 2:
                lower, upper = sorted(solves, key=lambda t: min(x[0] for x in solves[t]))
                assert sorted(x[0] for x in solves[lower]) == list(range(ncA))
                assert all(m == cid and nc == ncA for cid, m, nc in solves[lower])
                assert all(m == cid - ncA and nc == nclus - ncA for cid, m, nc in solves[upper])
            else:
                (only,) = solves
                assert all(m == cid and nc == nclus for cid, m, nc in solves[only])
            for sol in solves:
                assert sol not in when, f"solve {sol} twice in visit {jo}"
                when[sol] = s
        # every inner solve of the oracle's sweep once, after the solves it reads
        assert sorted(when) == sorted(order)
        for (Mp, bwd), s in when.items():
            for dep in deps(Mp, bwd, B, c):
                assert when[dep] < s, (jo, (Mp, bwd), dep)
        # the visit's boundary phase comes first
        assert all(r[1] for r in by_step[jo * spv])
    assert all(r[1] for r in by_step[nsteps - 1])
    # one operator per (slab, block, direction) slot; the forward and backward
    # solves of an interior block share it
    assert len(set(seen_p.values())) == len(seen_p) - sum(
        1 for (M, Mp, iid) in seen_p if iid == 1 and 0 < Mp < B - 1)
