"""The 3D Taylor-Green input generator (workloads.taylor_green_3d / _box): the analytic velocity gradient
against central differences of the sampled field (which for a single Fourier mode differ by exactly
sin(k) / k), zero divergence, and the cubic form equal to the box form."""
import numpy as np

from paper_1704_04413_gb300 import workloads as wl


def test_gradient_matches_central_differences_and_divergence_vanishes():
    nx, ny, nz, u0 = 24, 16, 12, 0.07
    rho, u, g = wl.taylor_green_3d_box(nx, ny, nz, u0)
    assert np.all(rho == 1.0)
    n = {0: nx, 1: ny, 2: nz}
    axis = {0: 2, 1: 1, 2: 0}  # arrays are [z][y][x]
    for a in range(3):
        for b in range(3):
            k = 2 * np.pi / n[b]
            fd = (np.roll(u[a], -1, axis=axis[b]) - np.roll(u[a], 1, axis=axis[b])) / 2.0
            assert np.max(np.abs(fd - g[3 * a + b] * np.sin(k) / k)) < 1e-14
    assert np.max(np.abs(g[0] + g[4] + g[8])) < 1e-15


def test_cube_equals_box():
    a = wl.taylor_green_3d(16, 0.05)
    b = wl.taylor_green_3d_box(16, 16, 16, 0.05)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=0, atol=1e-16)
