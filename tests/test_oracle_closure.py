"""Pins of the oracle's closure-corrected collision (no GPU).

The learned closure adds Delta a1^(2) to the projected a1^(2) of the RR collision before the recursion
(Eq. MalaspinasRecursiveRelation) builds the higher orders.  The collision is linear in a1 at fixed rho
and u, so the difference of the corrected and the plain collision of the same populations is
(1 - 1/tau) times the Hermite expansion of the correction and of what the recursion builds from it; its
Hermite moments are checked against closed forms: the order-2 moments are (1 - 1/tau) Delta, and on the
complete D2Q9 basis the order-3 and order-4 ones are the isothermal closed forms
a1_xxy = u_y a1_xx + 2 u_x a1_xy, a1_xyy = u_x a1_yy + 2 u_y a1_xy,
a1_xxyy = u_y^2 a1_xx + u_x^2 a1_yy + 4 u_x u_y a1_xy applied to Delta."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl


def cell_state(name, seed):
    """Non-equilibrium populations of one cell: f^(0) of a random (rho, u) times a 2 % noise."""
    L = orc.lattice(name)
    rng = np.random.default_rng(seed)
    rho, ux, uy = 1.0 + 0.05 * rng.standard_normal(), 0.08 * rng.standard_normal(), 0.08 * rng.standard_normal()
    op = orc.params(name, 1, 1, 0.7, "bgk", L.nmax)
    f = orc.init(op, np.array([[rho]]), np.array([[ux]]), np.array([[uy]]))[:, 0, 0]
    return L, f * (1.0 + 0.02 * rng.uniform(-1, 1, L.V))


def hermite_moments(L, g):
    """Hermite moments of g: order 2 (xx, xy, yy), order 3 (xxy, xyy), order 4 (xxyy), with the
    probabilists' polynomials in xi / cs written out."""
    x, y, c = L.cx.astype(float), L.cy.astype(float), L.cs2
    return {"xx": np.sum((x * x - c) * g), "xy": np.sum(x * y * g), "yy": np.sum((y * y - c) * g),
            "xxy": np.sum((x * x - c) * y * g), "xyy": np.sum(x * (y * y - c) * g),
            "xxyy": np.sum((x * x - c) * (y * y - c) * g)}


@pytest.mark.parametrize("name", ["D2Q9", "D2V17", "D2V37"])
def test_zero_correction_is_the_rr_collision(name):
    L, f = cell_state(name, 1)
    op = orc.params(name, 1, 1, 0.62, "rr", L.nmax)
    assert np.array_equal(orc.collide_delta(op, f, [0.0, 0.0, 0.0]), orc.collide(op, f))


@pytest.mark.parametrize("name", ["D2Q9", "D2V17", "D2V37"])
def test_corrected_collision_conserves_mass_and_momentum(name):
    L, f = cell_state(name, 2)
    op = orc.params(name, 1, 1, 0.58, "rr", L.nmax)
    g = orc.collide_delta(op, f, [3e-3, -2e-3, 1.5e-3])
    for w in (np.ones(L.V), L.cx, L.cy):
        assert abs(np.sum(w * (g - f))) <= 1e-15


@pytest.mark.parametrize("name", ["D2Q9", "D2V17", "D2V37"])
def test_correction_enters_the_second_order_moments(name):
    """Order-2 Hermite moments of f*(Delta) - f*(0) = (1 - 1/tau) Delta on every lattice."""
    L, f = cell_state(name, 3)
    tau, d = 0.58, np.array([3e-3, -2e-3, 1.5e-3])
    op = orc.params(name, 1, 1, tau, "rr", L.nmax)
    m = hermite_moments(L, orc.collide_delta(op, f, d) - orc.collide(op, f))
    om1 = 1.0 - 1.0 / tau
    assert np.allclose([m["xx"], m["xy"], m["yy"]], om1 * d, rtol=1e-12, atol=1e-17)


def test_recursion_carries_the_correction_to_orders_three_and_four():
    """D2Q9 RR-4 (complete basis): the order-3 and order-4 moments of f*(Delta) - f*(0) follow the
    isothermal closed forms applied to Delta, with u the cell's velocity."""
    L, f = cell_state("D2Q9", 4)
    tau, (dxx, dxy, dyy) = 0.61, (2e-3, 1e-3, -1.2e-3)
    op = orc.params("D2Q9", 1, 1, tau, "rr", 4, 4)
    m = hermite_moments(L, orc.collide_delta(op, f, [dxx, dxy, dyy]) - orc.collide(op, f))
    rho = f.sum()
    ux, uy = np.sum(L.cx * f) / rho, np.sum(L.cy * f) / rho
    om1 = 1.0 - 1.0 / tau
    assert abs(m["xxy"] - om1 * (uy * dxx + 2 * ux * dxy)) <= 1e-15
    assert abs(m["xyy"] - om1 * (ux * dyy + 2 * uy * dxy)) <= 1e-15
    assert abs(m["xxyy"] - om1 * (uy * uy * dxx + ux * ux * dyy + 4 * ux * uy * dxy)) <= 1e-15


def test_closure_scaling_makes_the_relaxed_stress_the_prediction():
    """With Delta = u0^2 y / (1 - 1/tau), the post-collision second-order non-equilibrium moments move by
    exactly u0^2 y: the relaxed state carries the predicted subgrid stress."""
    name, nx, ny, tau, u0 = "D2Q9", 7, 5, 0.57, 0.05
    L = orc.lattice(name)
    fl = wl.random_fields(nx, ny, 3, u_scale=0.05)
    op = orc.params(name, nx, ny, tau, "rr", 4)
    f = orc.init(op, fl.rho, fl.ux, fl.uy) * (1.0 + wl.population_noise(L.V, nx, ny, 4, 0.02))
    y = np.random.default_rng(5).normal(size=(nx * ny, 8))
    d = orc.closure_delta(y, u0, tau, nx, ny)
    g = orc.step_delta(op, f, d) - orc.step(op, f)
    x, yv, c = L.cx.astype(float), L.cy.astype(float), L.cs2
    got = np.stack([np.tensordot(x * x - c, g, 1), np.tensordot(x * yv, g, 1), np.tensordot(yv * yv - c, g, 1)])
    assert np.allclose(got.reshape(3, -1).T, u0 * u0 * y[:, :3], rtol=1e-11, atol=1e-18)


def test_step_delta_matches_per_cell_collisions():
    """The grid step with a per-cell correction = pull streaming, then the cell collision with that
    cell's own Delta (checked on a ragged periodic grid against orc.step's streaming)."""
    name, nx, ny, tau = "D2V17", 9, 7, 0.66
    L = orc.lattice(name)
    fl = wl.random_fields(nx, ny, 8, u_scale=0.06)
    op = orc.params(name, nx, ny, tau, "rr", 3)
    f = orc.init(op, fl.rho, fl.ux, fl.uy) * (1.0 + wl.population_noise(L.V, nx, ny, 9, 0.02))
    d = np.random.default_rng(10).normal(size=(3, ny, nx)) * 1e-3
    out = orc.step_delta(op, f, d)
    # pull streaming by index: f_i(x) <- f_i(x - xi_i), periodic
    for (yy, xx) in [(0, 0), (3, 4), (ny - 1, nx - 1), (2, 8)]:
        fc = np.array([f[i, (yy - L.cy[i]) % ny, (xx - L.cx[i]) % nx] for i in range(L.V)])
        assert np.allclose(out[:, yy, xx], orc.collide_delta(op, fc, d[:, yy, xx]), rtol=0, atol=0)


def test_correction_is_rejected_outside_isothermal_rr():
    L, f = cell_state("D2V37", 6)
    for coll, thermal in (("pr", False), ("bgk", False), ("rr", True)):
        op = orc.params("D2V37", 1, 1, 0.7, coll, 4, thermal=thermal)
        with pytest.raises(ValueError):
            orc.collide_delta(op, f, [0.0, 0.0, 0.0])
