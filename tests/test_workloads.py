"""The seeded input recipes: the wave-packet source (the paper's force (b),
defined here since the paper gives no formula)."""
import math

import numpy as np

from paper_1502_07266_gb300 import workloads as W


def test_wave_packet_shape_and_direction():
    n, b = 31, 4
    om = W.omega_for(n)
    f = W.wave_packet(n, b, om)[0]
    N = n + 2 * b
    x = W.padded_coords(n, b)
    # zero in the padding, unit peak at the centre node nearest (1/2, 1/4, 1/4)
    pad = np.ones(N, bool)
    pad[b:b + n] = False
    assert np.all(f[pad, :, :] == 0) and np.all(f[:, pad, :] == 0) and np.all(f[:, :, pad] == 0)
    k = [int(np.argmin(np.abs(x - v))) for v in (0.25, 0.25, 0.5)]       # [z, y, x]
    assert abs(abs(f[k[0], k[1], k[2]]) - np.abs(f).max()) < 1e-12
    # the phase advances by omega h e_d per node along each axis (e = (0, 1, 1)/sqrt 2)
    h = 1.0 / (n + 1)
    z0, y0, x0 = k
    dphi_y = np.angle(f[z0, y0 + 1, x0] / f[z0, y0, x0])
    dphi_z = np.angle(f[z0 + 1, y0, x0] / f[z0, y0, x0])
    dphi_x = np.angle(f[z0, y0, x0 + 1] / f[z0, y0, x0])
    assert abs(dphi_y - om * h / math.sqrt(2)) < 1e-12 and abs(dphi_z - om * h / math.sqrt(2)) < 1e-12
    assert abs(dphi_x) < 1e-12
    # envelope: exp(-1/2) one width (half a wavelength) away from the centre along x
    w = math.pi / om
    r = np.abs(f[z0, y0, :])
    xs = x - x[x0]
    inside = (np.abs(xs) <= 3 * w) & ~pad
    np.testing.assert_allclose(r[inside], np.exp(-xs[inside] ** 2 / (2 * w * w)) * r[x0], rtol=1e-12)
