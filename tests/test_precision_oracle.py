"""Pins for the oracle's precision pattern: the twisted quasi-1D factorisation
and the reduced-precision storage of its factors (oracle/precision.py).

The twisted form must reproduce a sparse direct solve exactly (up to FP64
rounding): a wrong chain index, a dropped Schur term at the middle block or a
swapped coupling fails it.  The storage forms are pinned by the bounds that
follow from IEEE round-to-nearest in binary16 (10 stored significand bits):
a wrong scale exponent overflows or loses bits, a low part formed from the
wrong remainder or a swapped real/imaginary part breaks the bounds.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.krylov import gmres
from oracle.operator import Grid, apply_full, assemble_box, global_profile, kappa_field
from oracle.precision import block_exponent, fp16_parts, round_factor, split_fp16_parts
from oracle.sweep import SweepPreconditioner
from paper_1502_07266_gb300 import workloads as W


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _wide_blocks(seed, count=6, k=49):
    """Complex blocks whose entries span six decades, at overall scales from 1e-20 to 1e20."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        mag = 10.0 ** rng.uniform(-6, 0, (k, k))
        z = (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))) * mag
        out.append(z * 10.0 ** rng.uniform(-20, 20))
    return out


# ------------------------------------------------- twisted factorisation ---

@pytest.mark.parametrize("n,b,M,Mp", [(7, 3, 0, 0), (7, 3, 2, 3), (8, 2, 4, 1), (1, 1, 1, 1)])
def test_twisted_factorisation_matches_sparse_solve(n, b, M, Mp):
    """Both-ends elimination meeting at m = (Nx-1)//2 solves the quasi-1D problem
    exactly; Nx = 3 (n = 1, b = 1) has one-block chains on each side."""
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=2)
    P = SweepPreconditioner(c, g, d=1, factor_format="fp64")
    q1 = P.quasi1d(M, Mp).factor()
    assert q1.fmt == "fp64"
    pz, _ = P.zwin[M]
    py, _ = P.ywin[Mp]
    kap = kappa_field(c, g.omega)[pz.lo:pz.lo + pz.L, py.lo:py.lo + py.L, :]
    H = assemble_box(kap, global_profile(g), py, pz, g.h).tocsc()
    rng = np.random.default_rng(6)
    q = rng.standard_normal((g.N, q1.k, 2)) + 1j * rng.standard_normal((g.N, q1.k, 2))
    x = q1.solve(q)
    Lz, Ly = q1.Lz, q1.Ly
    for r in range(2):
        qn = q[:, :, r].reshape(g.N, Ly, Lz).transpose(2, 1, 0).ravel()
        xn = spla.spsolve(H, qn)
        assert _rel(x[:, :, r].reshape(g.N, Ly, Lz).transpose(2, 1, 0).ravel(), xn) < 1e-11


def test_twisted_preconditioner_equals_one_sided():
    """The whole apply with twisted FP64 factors equals the one-sided LDU form."""
    n, b = 7, 3
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    f = W.random_rhs(2, n, b, seed=7)
    z0 = SweepPreconditioner(c, g, d=1).apply(f)
    z1 = SweepPreconditioner(c, g, d=1, factor_format="fp64").apply(f)
    assert _rel(z1, z0) < 1e-12


# ------------------------------------------------------ stored formats ---

def test_block_exponent_places_largest_part_below_2_15():
    for T in _wide_blocks(1):
        e = block_exponent(T)
        mx = max(np.abs(T.real).max(), np.abs(T.imag).max()) / 2.0 ** e
        assert 2.0 ** 14 <= mx < 2.0 ** 15
    assert block_exponent(np.zeros((3, 3), complex)) == 0


def test_fp16_parts_are_fp16_values_within_half_an_ulp():
    for T in _wide_blocks(2):
        q, e = fp16_parts(T)
        for part, zpart in ((q.real, (T / 2.0 ** e).real), (q.imag, (T / 2.0 ** e).imag)):
            assert np.array_equal(part.astype(np.float16).astype(np.float64), part)
            err = np.abs(part - zpart)
            normal = np.abs(zpart) >= 2.0 ** -14
            assert np.all(err[normal] <= 2.0 ** -11 * np.abs(zpart[normal]))
            assert np.all(err[~normal] <= 2.0 ** -25)        # half the subnormal spacing
        # every entry carries at most the fp16 relative rounding of the block's scale
        assert _rel(round_factor(T, "fp16"), T) < 2.0 ** -11


def test_split_parts_reach_22_bits():
    for T in _wide_blocks(3):
        hi, lo, e = split_fp16_parts(T)
        z = T / 2.0 ** e
        for h, l, zp in ((hi.real, lo.real, z.real), (hi.imag, lo.imag, z.imag)):
            assert np.array_equal(h.astype(np.float16).astype(np.float64), h)
            assert np.array_equal(l.astype(np.float16).astype(np.float64), l)
            assert np.all(np.abs(h + l - zp) <= 2.0 ** -22 * np.abs(zp) + 2.0 ** -25)
        # the low part is the rounded remainder: it never exceeds half an ulp of hi
        assert np.all(np.abs(lo.real) <= 2.0 ** -11 * np.abs(hi.real) + 2.0 ** -25)


def test_split_product_error_within_analytical_bound():
    """(round(T) - T) w for the split form stays inside the entrywise bound
    sum_j 2^e (2^-22 (|Re z|+|Im z|) + 2^-24) |w_j|, far below the fp16 one."""
    rng = np.random.default_rng(4)
    for T in _wide_blocks(5, count=4, k=64):
        w = rng.standard_normal(64) + 1j * rng.standard_normal(64)
        e = block_exponent(T)
        z = T / 2.0 ** e
        bound = 2.0 ** e * ((2.0 ** -22) * (np.abs(z.real) + np.abs(z.imag)) + 2.0 ** -24) @ np.abs(w)
        err = np.abs(round_factor(T, "split_fp16") @ w - T @ w)
        assert np.all(err <= bound)
        err16 = np.abs(round_factor(T, "fp16") @ w - T @ w)
        assert np.linalg.norm(err) < 2.0 ** -9 * np.linalg.norm(err16)   # 11 more bits


def test_fp16_factors_keep_gmres_iterations():
    """With FP16-stored factors the preconditioner changes by about 2^-11 and
    GMRES (FP64 true residual) reaches the same tolerance in as many iterations."""
    n, b = 7, 3
    om = W.omega_for(n)
    g = Grid(n, b, om)
    c = W.velocity_random(n, b, seed=0)
    f = W.gaussian_sources(n, b, om, [(0.5, 0.5, 0.3)])[0]
    P64 = SweepPreconditioner(c, g, d=1)
    P16 = SweepPreconditioner(c, g, d=1, factor_format="fp16")
    z64, z16 = P64.apply(f), P16.apply(f)
    assert 1e-6 < _rel(z16, z64) < 1e-2
    _, it64, h64 = gmres(lambda x: apply_full(x, c, g), P64.apply, f, tol=1e-8)
    _, it16, h16 = gmres(lambda x: apply_full(x, c, g), P16.apply, f, tol=1e-8)
    assert h16[-1] <= 1e-8 and h64[-1] <= 1e-8
    assert it16 <= it64 + 1
