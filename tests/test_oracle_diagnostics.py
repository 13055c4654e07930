"""Pins of the oracle's flow diagnostics (Sec. III.B): the vorticity from fourth-order centred differences
and the domain mean / standard deviation of u^2 and of the enstrophy density omega^2 / 2, checked against
closed forms on trigonometric fields (no GPU)."""
import numpy as np
import pytest

from oracle import oracle as orc


def fields(L, m, U, V):
    """u_x = U cos(k y), u_y = V sin(k x) on an L x L periodic grid, k = 2 pi m / L (grid units)."""
    k = 2 * np.pi * m / L
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    return k, U * np.cos(k * y), V * np.sin(k * x)


def symbol(k):
    """Fourier symbol of the fourth-order centred first derivative, (8 sin k - sin 2k) / 6."""
    return (8 * np.sin(k) - np.sin(2 * k)) / 6.0


@pytest.mark.parametrize("L,m", [(16, 1), (32, 3), (64, 5)])
def test_vorticity_is_the_fourth_order_difference(L, m):
    k, ux, uy = fields(L, m, 0.7, -1.3)
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    # omega = d_x u_y - d_y u_x; the stencil maps sin / cos(k x) to symbol(k) times cos / -sin(k x)
    expect = -1.3 * symbol(k) * np.cos(k * x) + 0.7 * symbol(k) * np.sin(k * y)
    assert np.max(np.abs(orc.vorticity(ux, uy) - expect)) <= 1e-13


def test_vorticity_converges_at_fourth_order():
    """Against the exact derivative of the same continuous field: halving the spacing divides the
    error by 2^4 (a second-order stencil would give 4, a wrong sign or index no convergence at all)."""
    errs = []
    for L in (16, 32, 64, 128):
        k, ux, uy = fields(L, 1, 1.0, 1.0)
        y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
        exact = k * np.cos(k * x) + k * np.sin(k * y)
        errs.append(np.max(np.abs(orc.vorticity(ux, uy) - exact)) / k)
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 14.5) & (ratios < 17.5)), ratios


def test_vorticity_orientation():
    """Solid-body rotation counter-clockwise (u = (-y, x) locally) has omega = +2: checked on a periodic
    field whose first harmonic is that rotation near the origin."""
    L = 64
    k, ux, uy = fields(L, 1, 1.0, 1.0)
    # u_x = cos(k y) has d_y u_x = -k sin(k y); at y = L/4 (sin = 1) and x = 0 (d_x u_y = k):
    w = orc.vorticity(ux, uy)
    assert w[L // 4, 0] > 0 and abs(w[L // 4, 0] - 2 * symbol(k)) < 1e-13


@pytest.mark.parametrize("L,m,U,V", [(32, 1, 0.1, 0.05), (48, 2, 0.03, 0.08), (64, 3, 1.0, 1.0)])
def test_diagnostics_closed_forms(L, m, U, V):
    """u^2 = U^2 cos^2(ky) + V^2 sin^2(kx) and omega = s (V cos(kx) + U sin(ky)) with s = symbol(k): over a
    grid that samples whole periods, the x and y phases are independent and uniform, so
    <u^2> = (U^2 + V^2) / 2, var(u^2) = (U^4 + V^4) / 8, <omega^2/2> = s^2 (U^2 + V^2) / 4, and with
    A = V cos, B = U sin: var(omega^2 / 2) = s^4 / 4 (E(A+B)^4 - (E(A+B)^2)^2),
    E(A+B)^4 = 3 V^4 / 8 + 6 (V^2 / 2)(U^2 / 2) + 3 U^4 / 8."""
    k, ux, uy = fields(L, m, U, V)
    rho = np.ones_like(ux)
    d = orc.diagnostics(rho, ux, uy)
    s = symbol(k)
    e2 = (U ** 2 + V ** 2) / 2
    e4 = 3 * V ** 4 / 8 + 6 * (V ** 2 / 2) * (U ** 2 / 2) + 3 * U ** 4 / 8
    expect = np.array([e2, np.sqrt((U ** 4 + V ** 4) / 8), s ** 2 * e2 / 2, s ** 2 / 2 * np.sqrt(e4 - e2 ** 2)])
    assert np.allclose(d, expect, rtol=1e-12, atol=0), (d, expect)


def test_diagnostics_of_a_uniform_flow():
    """Uniform flow: <u^2> = |u|^2, no spread, no vorticity."""
    ux = np.full((20, 24), 0.04)
    uy = np.full((20, 24), -0.03)
    d = orc.diagnostics(np.ones_like(ux), ux, uy)
    assert abs(d[0] - 0.0025) < 1e-17 and d[1] < 1e-17 and d[2] < 1e-30 and d[3] < 1e-30
