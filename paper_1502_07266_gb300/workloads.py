"""Seeded synthetic inputs for the Helmholtz problems (velocity fields and sources).

This module holds input recipes only: it samples velocity fields c(x) and
source terms f(x) on the PML-padded grid.  It contains none of the solver's
arithmetic (no PML stretching, no stencil, no sweep), so both the CUDA path
and the FP64 oracle draw their inputs from here without sharing method code.

Grid convention (Section 2 of the paper, padded on every face): with ``n``
interior points per axis and ``b`` PML layers on each face, the padded axis
has ``N = n + 2b`` nodes ``g = 0..N-1`` at coordinate ``(g - b + 1) h`` with
``h = 1/(n+1)``.  The physical nodes ``g = b..b+n-1`` sit at ``h..n h``.
Arrays are ``(N, N, N)`` indexed ``[z, y, x]`` (x fastest, the paper's
column-major order), multi-RHS arrays ``(R, N, N, N)``.

Recipes (the paper names the fields of its Section 4 but does not give their
formulas; these are the stated synthetic stand-ins):
  * constant:   c = 1
  * lens:       c = 4/3 (1 - 0.5 exp(-32 |x - (1/2,1/2,1/2)|^2))
  * waveguide:  c = 0.7 where |x1 - 1/2| < 0.1 and |x2 - 1/2| < 0.1, else 1
                (a vertical guide along x3)
  * random:     i.i.d. N(0,1) on a 16^3 lattice at nodes j/15 per axis
                (numpy default_rng(seed)), trilinear onto the grid, then
                mapped affinely to [1, 2] by the lattice min and max
  * bump:       lens + 0.05 exp(-32 |x - x_b|^2), x_b ~ U[0.35, 0.65]^3 (seed)
  * Gaussian source at x_s: f = exp(-(4 omega / pi)^2 |x - x_s|^2) on the
    physical nodes, zero in the PML padding (the force lies outside the PML).
  * wave packet (the paper's second force: a Gaussian wave packet centred at
    (1/2, 1/4, 1/4) travelling along (0, 1/sqrt2, 1/sqrt2); its formula is not
    in the paper, so this definition is this library's own):
        f = exp(-|x - x_0|^2 / (2 w^2)) exp(i omega e.(x - x_0)),
    e the unit direction, w = one wavelength 2 pi / omega at c = 1 divided by 2,
    zero in the PML padding and below 1e-12 of the peak.
Velocity in the padding is the nearest physical value (clamped index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def omega_for(n: int, ppw: float = 8.0) -> float:
    """Angular frequency giving ``ppw`` points per wavelength at c = 1: 2 pi n / ppw."""
    return 2.0 * math.pi * n / ppw


def padded_coords(n: int, b: int) -> np.ndarray:
    """Coordinates of the padded axis nodes, clamped to the physical range.

    Node g maps to (g - b + 1) h; padding nodes take the coordinate of the
    nearest physical node, which realises the nearest-value clamp of fields.
    """
    N = n + 2 * b
    h = 1.0 / (n + 1)
    g = np.arange(N)
    gc = np.clip(g, b, b + n - 1)
    return (gc - b + 1) * h


def physical_coords(n: int, b: int) -> np.ndarray:
    """Unclamped coordinates (g - b + 1) h of all padded nodes."""
    N = n + 2 * b
    h = 1.0 / (n + 1)
    return (np.arange(N) - b + 1) * h


def _mesh(n: int, b: int, clamp: bool = True):
    x = padded_coords(n, b) if clamp else physical_coords(n, b)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def velocity_constant(n: int, b: int, value: float = 1.0) -> np.ndarray:
    N = n + 2 * b
    return np.full((N, N, N), value, dtype=np.float64)


def velocity_lens(n: int, b: int) -> np.ndarray:
    X, Y, Z = _mesh(n, b)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    return (4.0 / 3.0) * (1.0 - 0.5 * np.exp(-32.0 * r2))


def velocity_waveguide(n: int, b: int) -> np.ndarray:
    X, Y, _ = _mesh(n, b)
    inside = (np.abs(X - 0.5) < 0.1) & (np.abs(Y - 0.5) < 0.1)
    return np.where(inside, 0.7, 1.0)


def _trilinear_lattice(vals: np.ndarray, X, Y, Z) -> np.ndarray:
    """Trilinear interpolation of a lattice on nodes j/(L-1) in [0,1]^3 (indexed [x,y,z])."""
    L = vals.shape[0]

    def split(t):
        u = np.clip(t, 0.0, 1.0) * (L - 1)
        i0 = np.minimum(np.floor(u).astype(np.int64), L - 2)
        return i0, u - i0

    ix, fx = split(X)
    iy, fy = split(Y)
    iz, fz = split(Z)
    out = np.zeros(X.shape)
    for dx in (0, 1):
        wx = fx if dx else 1.0 - fx
        for dy in (0, 1):
            wy = fy if dy else 1.0 - fy
            for dz in (0, 1):
                wz = fz if dz else 1.0 - fz
                out += wx * wy * wz * vals[ix + dx, iy + dy, iz + dz]
    return out


def velocity_random(n: int, b: int, seed: int = 0, lattice: int = 16) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((lattice, lattice, lattice))
    X, Y, Z = _mesh(n, b)
    w = _trilinear_lattice(v, X, Y, Z)
    return 1.0 + (w - v.min()) / (v.max() - v.min())


def velocity_bump(n: int, b: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    xb = rng.uniform(0.35, 0.65, size=3)
    X, Y, Z = _mesh(n, b)
    r2 = (X - xb[0]) ** 2 + (Y - xb[1]) ** 2 + (Z - xb[2]) ** 2
    return velocity_lens(n, b) + 0.05 * np.exp(-32.0 * r2)


def gaussian_sources(n: int, b: int, omega: float, centers) -> np.ndarray:
    """Gaussian point sources exp(-(4 omega/pi)^2 |x - x_s|^2), zero in the padding.

    Returns complex128 array (R, N, N, N).
    """
    N = n + 2 * b
    X, Y, Z = _mesh(n, b, clamp=False)
    alpha = (4.0 * omega / math.pi) ** 2
    phys = np.zeros(N, dtype=bool)
    phys[b:b + n] = True
    mask = phys[:, None, None] & phys[None, :, None] & phys[None, None, :]
    out = np.zeros((len(centers), N, N, N), dtype=np.complex128)
    for s, (cx, cy, cz) in enumerate(centers):
        r2 = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2
        out[s] = np.where(mask, np.exp(-alpha * r2), 0.0)
    return out


def wave_packet(n: int, b: int, omega: float, center=(0.5, 0.25, 0.25),
                direction=(0.0, 1.0 / math.sqrt(2.0), 1.0 / math.sqrt(2.0)), width=None) -> np.ndarray:
    """Gaussian wave packet exp(-|x-x0|^2/(2 w^2)) exp(i omega e.(x-x0)), zero in
    the padding; w defaults to half a wavelength at c = 1 (pi / omega).
    Returns complex128 (1, N, N, N)."""
    N = n + 2 * b
    X, Y, Z = _mesh(n, b, clamp=False)
    e = np.asarray(direction, dtype=np.float64)
    e = e / np.linalg.norm(e)
    w = (math.pi / omega) if width is None else float(width)
    cx, cy, cz = center
    r2 = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2
    phase = omega * (e[0] * (X - cx) + e[1] * (Y - cy) + e[2] * (Z - cz))
    f = np.exp(-r2 / (2.0 * w * w)) * np.exp(1j * phase)
    phys = np.zeros(N, dtype=bool)
    phys[b:b + n] = True
    mask = phys[:, None, None] & phys[None, :, None] & phys[None, None, :]
    f = np.where(mask & (np.abs(f) >= 1e-12), f, 0.0)
    return f[None].astype(np.complex128)


def plane_grid_centers(per_side: int, z: float):
    """per_side x per_side source centres ((i+1/2)/p, (j+1/2)/p, z)."""
    return [((i + 0.5) / per_side, (j + 0.5) / per_side, z)
            for j in range(per_side) for i in range(per_side)]


def rect_grid_centers(nx: int, ny: int, z: float):
    """nx x ny source centres ((i+1/2)/nx, (j+1/2)/ny, z)."""
    return [((i + 0.5) / nx, (j + 0.5) / ny, z) for j in range(ny) for i in range(nx)]


def random_rhs(R: int, n: int, b: int, seed: int) -> np.ndarray:
    """Seeded complex Gaussian vectors on the full padded grid, (R, N, N, N)."""
    N = n + 2 * b
    rng = np.random.default_rng(seed)
    return rng.standard_normal((R, N, N, N)) + 1j * rng.standard_normal((R, N, N, N))


@dataclass
class Workload:
    name: str
    n: int
    b: int
    d: int
    omega: float
    c: np.ndarray            # (N, N, N) float64 velocity on the padded grid
    f: np.ndarray            # (R, N, N, N) complex128 sources
    C: float = 10.0
    tol: float = 1e-6
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n + 2 * self.b

    @property
    def R(self) -> int:
        return self.f.shape[0]


def lens_wave_packet(n: int = 63, b: int = 6, d: int = 1) -> Workload:
    """The lens with the wave-packet source (the paper's force (b))."""
    om = omega_for(n)
    return Workload("lens, wave packet", n, b, d, om, velocity_lens(n, b), wave_packet(n, b, om))


def small_constant(n: int = 31, b: int = 6, d: int = 1) -> Workload:
    """Constant c = 1, one centred Gaussian source, 8 points per wavelength."""
    w = omega_for(n)
    return Workload("constant-c n=%d b=%d" % (n, b), n, b, d, w,
                    velocity_constant(n, b), gaussian_sources(n, b, w, [(0.5, 0.5, 0.5)]))


def lens_one_source(n: int = 63, b: int = 6, d: int = 1) -> Workload:
    w = omega_for(n)
    return Workload("lens n=%d b=%d" % (n, b), n, b, d, w,
                    velocity_lens(n, b), gaussian_sources(n, b, w, [(0.5, 0.5, 0.25)]))


def random_64_sources(n: int = 127, b: int = 6, d: int = 1, seed: int = 0,
                      per_side: int = 8) -> Workload:
    """Smooth random velocity in [1,2], per_side^2 sources on the z = 0.1 plane."""
    w = omega_for(n)
    return Workload("random-c n=%d b=%d %dx%d sources" % (n, b, per_side, per_side),
                    n, b, d, w, velocity_random(n, b, seed),
                    gaussian_sources(n, b, w, plane_grid_centers(per_side, 0.1)),
                    meta={"seed": seed})


def receiver_plane_index(n: int, b: int, z: float = 0.9) -> int:
    """Padded index of the grid plane nearest x3 = z (the receiver plane)."""
    return b - 1 + int(round(z * (n + 1)))


def lens_bump_16_sources(n: int = 63, b: int = 6, d: int = 1, seed: int = 0) -> Workload:
    """Lens perturbed by a 0.05 Gaussian bump, 4 x 4 sources on z = 0.1; the
    unperturbed lens provides the observed data (meta['c_obs'])."""
    w = omega_for(n)
    wl = Workload("lens+bump n=%d b=%d 4x4 sources" % (n, b), n, b, d, w,
                  velocity_bump(n, b, seed), gaussian_sources(n, b, w, plane_grid_centers(4, 0.1)),
                  meta={"c_obs": velocity_lens(n, b), "rec_plane": receiver_plane_index(n, b)})
    return wl


def uneven_batch(b: int = 5, d: int = 1, seed: int = 0):
    """Six uneven problems served together: n = 63, 95, 127, 159, 127, 95 with
    lens / waveguide / random velocities in turn (random seeded per problem) and
    8, 16, 32, 8, 16, 32 Gaussian sources on the z = 0.1 plane (4x2, 4x4, 8x4
    grids), 8 points per wavelength each."""
    ns = [63, 95, 127, 159, 127, 95]
    grids = {8: (4, 2), 16: (4, 4), 32: (8, 4)}
    counts = [8, 16, 32, 8, 16, 32]
    out = []
    for q, (n, R) in enumerate(zip(ns, counts)):
        w = omega_for(n)
        kind = ("lens", "waveguide", "random")[q % 3]
        c = {"lens": lambda: velocity_lens(n, b), "waveguide": lambda: velocity_waveguide(n, b),
             "random": lambda: velocity_random(n, b, seed=seed + q)}[kind]()
        f = gaussian_sources(n, b, w, rect_grid_centers(*grids[R], 0.1))
        out.append(Workload("%s n=%d b=%d %d sources" % (kind, n, b, R), n, b, d, w, c, f,
                            meta={"kind": kind, "seed": seed + q}))
    return out
