"""Local factor update (Section 6: a velocity change on a subdomain touches only
the quasi-1D problems whose windows meet it).

The CPU test pins the C library's affected-problem query (helm_affected_problems,
host only) against the oracle by brute force: every quasi-1D matrix H~_{M,M'}
(Alg. 3's problems, assembled by the oracle) is built for the old and the new
velocity, and the problems whose matrices differ must be exactly the ranges the
query returns.  The GPU tests (test_gpu_local_update.py) check that the update
equals a fresh setup.
"""
import numpy as np
import pytest

from oracle.operator import Grid
from oracle.sweep import SweepPreconditioner
from paper_1502_07266_gb300 import workloads as W

CASES = [  # n, b, d, b_aux, box (x0, x1, y0, y1, z0, z1)
    (7, 3, 1, 0, (4, 6, 5, 7, 5, 7)),
    (7, 3, 1, 0, (0, 13, 0, 1, 12, 13)),
    (8, 2, 2, 0, (3, 4, 2, 9, 7, 8)),
    (8, 3, 2, 2, (0, 2, 10, 14, 0, 3)),
    (6, 2, 3, 1, (1, 9, 4, 5, 2, 10)),
]


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm as H
    return H


def _changed(P0, P1):
    out = set()
    for M in range(P0.B):
        for Mp in range(P0.B):
            a, b = P0.quasi1d(M, Mp), P1.quasi1d(M, Mp)
            if not (np.array_equal(a.D, b.D) and np.array_equal(a.lower, b.lower)
                    and np.array_equal(a.upper, b.upper)):
                out.add((M, Mp))
    return out


@pytest.mark.parametrize("n,b,d,b_aux,box", CASES)
def test_affected_problems_are_the_changed_quasi1d_matrices(helm, n, b, d, b_aux, box):
    g = Grid(n, b, W.omega_for(n))
    c0 = W.velocity_random(n, b, seed=5)
    c1 = c0.copy()
    x0, x1, y0, y1, z0, z1 = box
    c1[z0:z1, y0:y1, x0:x1] *= 1.1                 # arrays are (z, y, x)
    ba = b_aux if b_aux > 0 else None
    changed = _changed(SweepPreconditioner(c0, g, d=d, b_aux=ba), SweepPreconditioner(c1, g, d=d, b_aux=ba))
    r = helm.helm_affected_problems(n, b, d, box, b_aux=b_aux)
    want = {(M, Mp) for M in range(r[0], r[1] + 1) for Mp in range(r[2], r[3] + 1)} if r[0] >= 0 else set()
    assert changed == want
    assert 0 < len(changed) < SweepPreconditioner(c0, g, d=d).B ** 2     # a strict subset


@pytest.mark.parametrize("n,b,d,b_aux,box", [(7, 3, 1, 3, (4, 6, 5, 7, 5, 7)), (9, 3, 2, 2, (0, 15, 11, 14, 1, 4)),
                                             (8, 2, 1, 2, (2, 5, 6, 7, 0, 12))])
def test_affected_problems_two_front(helm, n, b, d, b_aux, box):
    """The same brute-force pin for the two-front schedule (its upper front's
    and centre's windows extend above their blocks)."""
    g = Grid(n, b, W.omega_for(n))
    c0 = W.velocity_random(n, b, seed=7)
    c1 = c0.copy()
    x0, x1, y0, y1, z0, z1 = box
    c1[z0:z1, y0:y1, x0:x1] *= 1.1
    P0 = SweepPreconditioner(c0, g, d=d, b_aux=b_aux, schedule="two_front")
    P1 = SweepPreconditioner(c1, g, d=d, b_aux=b_aux, schedule="two_front")
    changed = _changed(P0, P1)
    r = helm.helm_affected_problems(n, b, d, box, b_aux=b_aux, schedule=helm.HELM_TWO_FRONT)
    want = {(M, Mp) for M in range(r[0], r[1] + 1) for Mp in range(r[2], r[3] + 1)} if r[0] >= 0 else set()
    assert changed == want
    assert 0 < len(changed) < P0.B ** 2


def test_affected_problems_rejects_bad_boxes(helm):
    for box in [(0, 14, 0, 1, 0, 1), (3, 3, 0, 1, 0, 1), (-1, 2, 0, 1, 0, 1), (0, 1, 5, 4, 0, 1)]:
        with pytest.raises(helm.HelmError):
            helm.helm_affected_problems(7, 3, 1, box)
