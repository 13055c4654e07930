"""Pins of the oracle's collision and streaming (Sec. II.A, II.E, II.F, III.A, III.B).

Invariants fixed by the paper: collision invariants (Eq. CollisionInvariant /
NullityOfa1); PR on the complete D2Q9 basis is BGK (Sec. II.F, Sec. III.B);
RR = PR for N = 2 isothermal (Sec. II.F); equilibrium is a fixed point; the
streaming of Sec. III.A moves population i by xi_i.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl

MODES = [("D2Q9", 2, 0), ("D2Q9", 4, 0), ("D2V17", 3, 0), ("D2V37", 4, 0), ("D2V37", 4, 3), ("D2V37", 2, 2)]


def noisy_cell(name, seed, theta=1.0, eps=0.05):
    L = orc.lattice(name)
    rng = np.random.default_rng(seed)
    rho, ux, uy = rng.uniform(0.8, 1.2), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)
    f0 = orc.expand(name, 0, L.nmax, orc.a0(L.cs2, rho, ux, uy, theta))
    return f0 * (1.0 + rng.uniform(-eps, eps, L.V)), L


@pytest.mark.parametrize("coll", ["bgk", "pr", "rr"])
@pytest.mark.parametrize("name,neq,nreg", MODES)
def test_collision_conserves_mass_and_momentum(coll, name, neq, nreg):
    for seed in range(4):
        f, L = noisy_cell(name, seed)
        p = orc.params(name, 1, 1, 0.6, coll, neq, nreg)
        g = orc.collide(p, f)
        for h in (np.ones(L.V), L.cx, L.cy):
            assert abs(np.dot(g - f, h)) < 2e-15


@pytest.mark.parametrize("coll", ["bgk", "pr", "rr"])
def test_thermal_collision_conserves_energy(coll):
    L = orc.lattice("D2V37")
    e = (L.cx ** 2 + L.cy ** 2).astype(float)
    for seed in range(4):
        f, _ = noisy_cell("D2V37", seed, theta=1.15)
        g = orc.collide(orc.params("D2V37", 1, 1, 0.7, coll, 4, 0, thermal=True), f)
        for h in (np.ones(L.V), L.cx, L.cy, e):
            assert abs(np.dot(g - f, h)) < 1e-14


def test_thermal_projected_a1_is_traceless():
    """Eq. (NullityOfa1): Tr a1^(2) = 0 when f^(0) carries the cell's own temperature."""
    L = orc.lattice("D2V37")
    f, _ = noisy_cell("D2V37", 9, theta=0.9)
    rho, jx, jy = f.sum(), (f * L.cx).sum(), (f * L.cy).sum()
    ux, uy = jx / rho, jy / rho
    th = ((f * (L.cx ** 2 + L.cy ** 2)).sum() / rho - ux * ux - uy * uy) / (2 * L.cs2)
    f0 = orc.expand("D2V37", 0, 4, orc.a0(L.cs2, rho, ux, uy, th))
    tr = sum(np.dot([orc.hermite(2, t, x, y, L.cs2) for x, y in zip(L.cx, L.cy)], f - f0) for t in (0, 3))
    assert abs(tr) < 1e-15


def test_pr_on_complete_d2q9_basis_is_bgk():
    """Sec. II.F / Sec. III.B: PR 4 with f^(0) on the complete D2Q9 basis gives exactly BGK."""
    for seed in range(5):
        f, _ = noisy_cell("D2Q9", seed, eps=0.1)
        a = orc.collide(orc.params("D2Q9", 1, 1, 0.57, "pr", 4, 4), f)
        b = orc.collide(orc.params("D2Q9", 1, 1, 0.57, "bgk", 4, 4), f)
        assert np.max(np.abs(a - b)) < 1e-15


@pytest.mark.parametrize("name,neq", [("D2Q9", 2), ("D2Q9", 4), ("D2V17", 3), ("D2V37", 4)])
def test_rr2_equals_pr2_isothermal(name, neq):
    """Sec. II.F: a1,RR^(n) = a1,PR^(n) for n <= 2 in the isothermal case, so N = 2 gives the same step."""
    for seed in range(3):
        f, _ = noisy_cell(name, seed)
        a = orc.collide(orc.params(name, 1, 1, 0.8, "rr", neq, 2), f)
        b = orc.collide(orc.params(name, 1, 1, 0.8, "pr", neq, 2), f)
        assert np.max(np.abs(a - b)) < 1e-15


@pytest.mark.parametrize("coll", ["bgk", "pr", "rr"])
@pytest.mark.parametrize("name,neq,nreg", MODES)
def test_equilibrium_is_fixed_point(coll, name, neq, nreg):
    L = orc.lattice(name)
    f0 = orc.expand(name, 0, neq, orc.a0(L.cs2, 1.05, 0.04, -0.03, 1.0))
    g = orc.collide(orc.params(name, 1, 1, 0.6, coll, neq, nreg), f0)
    assert np.max(np.abs(g - f0)) < 1e-15


def test_rr_filters_non_hydrodynamic_content_d2q9():
    """RR removes every non-equilibrium component not of Chapman-Enskog form: two cells with the same
    rho, u and a1^(2) but different higher projections collide to the same RR populations (Sec. II.F)."""
    L = orc.lattice("D2Q9")
    f, _ = noisy_cell("D2Q9", 3)
    # add a multiple of the order-3 tensor H_xxy (orthogonal to everything up to order 2)
    h = np.array([orc.hermite(3, 0b100, x, y, L.cs2) for x, y in zip(L.cx, L.cy)]) * L.w
    g = f + 1e-3 * h
    p = orc.params("D2Q9", 1, 1, 0.7, "rr", 2, 4)
    assert np.max(np.abs(orc.collide(p, f) - orc.collide(p, g))) < 1e-15
    pbgk = orc.params("D2Q9", 1, 1, 0.7, "bgk", 2, 4)
    assert np.max(np.abs(orc.collide(pbgk, f) - orc.collide(pbgk, g))) > 1e-5


@pytest.mark.parametrize("name", ["D2Q9", "D2V17", "D2V37"])
def test_streaming_moves_population_by_its_velocity(name):
    """Sec. III.A: f_i(x + xi_i, t + 1) is built from f_i(x, t); a perturbation of population i at x
    reaches, after one step, only the cell x + xi_i (periodic)."""
    L = orc.lattice(name)
    nx, ny = 11, 9
    p = orc.params(name, nx, ny, 0.9, "bgk", 2)
    base = orc.init(p, np.ones((ny, nx)), np.full((ny, nx), 0.02), np.zeros((ny, nx)))
    ref = orc.step(p, base)
    x0, y0 = 5, 4
    for i in range(L.V):
        f = base.copy()
        f[i, y0, x0] += 1e-3
        d = np.abs(orc.step(p, f) - ref).sum(axis=0)
        changed = set(zip(*np.nonzero(d > 1e-14)))
        assert changed == {((y0 + L.cy[i]) % ny, (x0 + L.cx[i]) % nx)}


@pytest.mark.parametrize("coll", ["bgk", "pr", "rr"])
@pytest.mark.parametrize("bc", [orc.PERIODIC, orc.ZERO_GRADIENT])
def test_uniform_flow_is_invariant(coll, bc):
    for name, neq in (("D2Q9", 2), ("D2V17", 3), ("D2V37", 4)):
        nx, ny = 7, 5
        p = orc.params(name, nx, ny, 0.55, coll, neq, bc_x=bc, bc_y=bc)
        f = orc.init(p, np.full((ny, nx), 1.1), np.full((ny, nx), 0.05), np.full((ny, nx), -0.02))
        g = orc.step(p, f, 3)
        assert np.max(np.abs(g - f)) < 1e-15


def test_zero_gradient_reads_clamped_source():
    """Boundary reading: a pulled source outside [0, nx-1] is replaced by the clamped edge cell."""
    name = "D2V37"
    L = orc.lattice(name)
    nx, ny = 8, 3
    p = orc.params(name, nx, ny, 0.8, "bgk", 4, bc_x=orc.ZERO_GRADIENT)
    fl = wl.random_fields(nx, ny, 5)
    f = orc.init(p, fl.rho, fl.ux, fl.uy)
    out = orc.step(p, f)
    # rebuild the pulled cell (x=0,y=1) by hand and collide it
    x, y = 0, 1
    pulled = np.array([f[i, (y - L.cy[i]) % ny, min(max(x - L.cx[i], 0), nx - 1)] for i in range(L.V)])
    assert np.max(np.abs(out[:, y, x] - orc.collide(p, pulled))) < 1e-16


def test_step_cells_matches_full_step():
    name = "D2V17"
    nx, ny = 13, 6
    p = orc.params(name, nx, ny, 0.7, "rr", 3)
    fl = wl.random_fields(nx, ny, 2)
    f = orc.init(p, fl.rho, fl.ux, fl.uy)
    full = orc.step(p, f)
    cells = np.array([0, 5, 40, nx * ny - 1])
    part = orc.step_cells(p, f, cells)
    for k, c in enumerate(cells):
        assert np.array_equal(part[k], full[:, c // nx, c % nx])


def test_rejects_invalid_parameters():
    with pytest.raises(ValueError):
        orc.collide(orc.params("D2Q9", 1, 1, 0.5, "rr", 2), np.ones(9))
    with pytest.raises(ValueError):
        orc.collide(orc.params("D2V17", 1, 1, 0.7, "rr", 4), np.ones(17))
    with pytest.raises(ValueError):
        orc.collide(orc.params("D2Q9", 1, 1, 0.7, "rr", 2, thermal=True), np.ones(9))


@pytest.mark.parametrize("name,neq,thermal", [("D2Q9", 2, False), ("D2V17", 3, False), ("D2V37", 4, False),
                                              ("D2V37", 4, True)])
def test_init_nonequilibrium_matches_chapman_enskog_stress(name, neq, thermal):
    """Sec. III.B initial state f = f^(0) + f^(1): projecting f - f^(0) on H^(2) returns the CE stress
    -tau rho cs^2 theta (S - (2/D) div u delta) (thermal) or -tau rho cs^2 S (isothermal) (App. A)."""
    L = orc.lattice(name)
    nx, ny, tau = 3, 2, 0.74
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.9, 1.1, (ny, nx))
    ux, uy = rng.uniform(-0.05, 0.05, (2, ny, nx))
    th = rng.uniform(0.9, 1.1, (ny, nx)) if thermal else None
    grad = rng.normal(size=(4, ny, nx)) * 1e-3
    p = orc.params(name, nx, ny, tau, "rr", neq, thermal=thermal)
    f = orc.init(p, rho, ux, uy, th, grad)
    f0 = orc.init(p, rho, ux, uy, th, None)
    for y in range(ny):
        for x in range(nx):
            du = np.array([[grad[0, y, x], grad[1, y, x]], [grad[2, y, x], grad[3, y, x]]])  # du[a][b] = d_b u_a
            t = th[y, x] if thermal else 1.0
            for a in range(2):
                for b in range(2):
                    S = du[a, b] + du[b, a] - ((du[0, 0] + du[1, 1]) if (thermal and a == b) else 0.0)
                    h = np.array([orc.hermite(2, a | (b << 1), cx, cy, L.cs2) for cx, cy in zip(L.cx, L.cy)])
                    got = np.dot(h, f[:, y, x] - f0[:, y, x])
                    assert abs(got + tau * rho[y, x] * L.cs2 * t * S) < 1e-15
