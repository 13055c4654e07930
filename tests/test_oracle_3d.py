"""Pins of the three-dimensional oracle (oracle/lbm3d.py) against what Tab. II and the mathematics fix: the
printed lattices (golden file), their quadrature degree against the Gaussian moments, the Gram matrix of
the kept Hermite tensors (orthonormal, also for the reading that keeps H_xxyz on D3Q27), the equilibrium
moments, the recursive a1 against its closed form, conservation, PR on the complete D3Q27 basis = BGK,
RR at order 2 = PR-2, streaming, and the viscous decay of a shear wave."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import hermite_e

from oracle import lbm3d as o

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_lattices.json")))
NAMES = ["D3Q19", "D3Q27", "D3V39", "D3Q103"]
# column order of the printed basis table: exponent triples
COLUMNS = [(0, 0, 0), (1, 0, 0), (2, 0, 0), (1, 1, 0), (3, 0, 0), (2, 1, 0), (1, 1, 1), (4, 0, 0), (3, 1, 0),
           (2, 2, 0), (2, 1, 1), (2, 2, 1), (2, 2, 2)]


def value(s):
    if s.startswith("sqrt("):
        return math.sqrt(float(Fraction(s[5:-1])))
    return float(Fraction(s)) if "/" in s else float(s)


@pytest.mark.parametrize("name", NAMES)
def test_lattice_matches_table2(name):
    g, L = GOLD[name], o.lattice(name)
    assert L.V == sum(g["p"])
    for rep, p, w in zip(g["groups"], g["p"], g["weights"]):
        sel = [i for i in range(L.V) if sorted(np.abs(L.xi[i])) == sorted(rep)]
        assert len(sel) == p
        assert np.allclose(L.w[sel], value(w), rtol=0, atol=1e-18)
    assert abs(1.0 / math.sqrt(L.cs2) - value(g["inv_cs"])) < 1e-14
    assert abs(L.w.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("name", NAMES)
def test_quadrature_degree(name):
    """sum_i w_i xi^a eta^b zeta^c equals the Gaussian moment cs^(a+b+c) (a-1)!!(b-1)!!(c-1)!! up to the
    degree Q of Tab. II, and fails at some moment of degree Q + 1 or Q + 2 for the standard lattices."""
    L, Q = o.lattice(name), GOLD[name]["Q"]
    xi = L.xi.astype(float)

    def gauss(a):
        return 0.0 if a % 2 else float(np.prod(np.arange(a - 1, 0, -2))) if a else 1.0

    for e in itertools.product(range(Q + 1), repeat=3):
        if sum(e) > Q:
            continue
        lhs = np.dot(L.w, xi[:, 0] ** e[0] * xi[:, 1] ** e[1] * xi[:, 2] ** e[2])
        rhs = L.cs2 ** (sum(e) / 2) * gauss(e[0]) * gauss(e[1]) * gauss(e[2])
        assert abs(lhs - rhs) < 1e-12, e


@pytest.mark.parametrize("name", NAMES)
def test_hermite_tensors_are_products_of_1d_hermite_polynomials(name):
    L, H = o.lattice(name), o.hermite(name)
    cs = math.sqrt(L.cs2)
    for n in range(5):
        for alpha in o.tuples(n):
            e = o.exponents(alpha)
            ref = np.prod([hermite_e.hermeval(L.xi[:, d] / cs, [0] * e[d] + [1]) * cs ** e[d] for d in range(3)],
                          axis=0)
            assert np.allclose(H[alpha], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", NAMES)
def test_gram_matrix_of_kept_tensors(name):
    """sum_i w_i H_a H_b = delta_ab a_x! a_y! a_z! cs^(2n) on the kept basis (canonical tuples), which is
    what makes the projections and the rebuild exact, except for D3Q19's six pairs of third-order tensors
    noted below; the printed basis column agrees except where the reading differs (H_xxyz on D3Q27)."""
    L, H = o.lattice(name), o.hermite(name)
    canon = [e for n in range(o.NMAX[name] + 1) for e in itertools.product(range(n + 1), repeat=3)
             if sum(e) == n and o.kept(name, e)]
    tup = lambda e: (0,) * e[0] + (1,) * e[1] + (2,) * e[2]
    def partners(a, b):
        # D3Q19 only: two third-order tensors with the same odd axis and different even axes (H_xxy and
        # H_yzz, ...) are not orthogonal on 19 velocities: their product sums to -cs^6
        if name != "D3Q19" or sum(a) != 3 or sum(b) != 3 or a == b:
            return False
        return [d for d in range(3) if a[d] == 1] == [d for d in range(3) if b[d] == 1]

    for a in canon:
        for b in canon:
            g = np.dot(L.w, H[tup(a)] * H[tup(b)])
            if a == b:
                want = math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2]) * L.cs2 ** sum(a)
            else:
                want = -L.cs2 ** 3 if partners(a, b) else 0.0
            assert abs(g - want) < 1e-12, (a, b)
    printed = GOLD[name]["basis_as_printed"]
    for col, flag in zip(COLUMNS, printed):
        if name == "D3Q27" and col == (2, 1, 1):
            assert not flag and o.kept(name, col)
            continue
        assert o.kept(name, col) == bool(flag), col


def random_state(name, N, seed, eps=0.02, neq=2):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * rng.standard_normal(N)
    u = 0.05 * rng.standard_normal((3, N))
    f = o.expand(name, o.equilibrium_coefficients(rho, u, neq), 0, neq)
    return f * (1 + rng.uniform(-eps, eps, f.shape))


@pytest.mark.parametrize("name", NAMES)
def test_equilibrium_moments(name):
    rng = np.random.default_rng(1)
    rho, u = 1 + 0.1 * rng.random(20), 0.1 * rng.standard_normal((3, 20))
    L = o.lattice(name)
    xi = L.xi.astype(float)
    f0 = o.expand(name, o.equilibrium_coefficients(rho, u, 2), 0, 2)
    assert np.allclose(f0.sum(0), rho, atol=1e-14)
    assert np.allclose(xi.T @ f0, rho * u, atol=1e-14)
    for a, b in o.tuples(2):
        pi = (xi[:, a] * xi[:, b]) @ f0
        assert np.allclose(pi, rho * u[a] * u[b] + rho * L.cs2 * (a == b), atol=1e-14)


def test_recursive_a1_equals_the_isothermal_closed_form():
    """a1^(n)_alpha = sum over position pairs i < j of a1_{alpha_i alpha_j} prod_{k != i, j} u_{alpha_k}."""
    rng = np.random.default_rng(2)
    rho, u = 1 + 0.1 * rng.random(7), 0.1 * rng.standard_normal((3, 7))
    a0 = o.equilibrium_coefficients(rho, u, 6)
    m = rng.standard_normal((3, 3, 7))
    a1 = {(a, b): m[a, b] + m[b, a] for a, b in o.tuples(2)}
    o.a1_recursive(rho, u, a0, a1, 6)
    for n in (3, 4, 5, 6):
        for alpha in o.tuples(n):
            ref = 0.0
            for i, j in itertools.combinations(range(n), 2):
                rest = [alpha[k] for k in range(n) if k not in (i, j)]
                ref = ref + a1[(alpha[i], alpha[j])] * np.prod([u[d] for d in rest], axis=0)
            assert np.allclose(a1[alpha], ref, atol=1e-14), alpha


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("coll", ["bgk", "pr", "rr"])
def test_collision_conserves_mass_and_momentum(name, coll):
    L = o.lattice(name)
    f = random_state(name, 50, 3)
    p = o.Params3(name, 50, 1, 1, 0.7, coll, hermite_order=min(3, L.nmax))
    g = o.collide(p, f)
    xi = L.xi.astype(float)
    assert np.allclose(g.sum(0), f.sum(0), atol=1e-14)
    assert np.allclose(xi.T @ g, xi.T @ f, atol=1e-14)


def test_pr_on_the_complete_d3q27_basis_is_bgk():
    f = random_state("D3Q27", 40, 4, neq=6)
    pr = o.collide(o.Params3("D3Q27", 40, 1, 1, 0.7, "pr", hermite_order=6, reg_order=6), f)
    bgk = o.collide(o.Params3("D3Q27", 40, 1, 1, 0.7, "bgk", hermite_order=6), f)
    assert np.allclose(pr, bgk, atol=1e-14)


@pytest.mark.parametrize("name", NAMES)
def test_rr_at_order_2_is_pr_2(name):
    f = random_state(name, 30, 5)
    rr = o.collide(o.Params3(name, 30, 1, 1, 0.7, "rr", reg_order=2), f)
    pr = o.collide(o.Params3(name, 30, 1, 1, 0.7, "pr", reg_order=2), f)
    assert np.allclose(rr, pr, atol=1e-15)


@pytest.mark.parametrize("name", ["D3Q19", "D3V39"])
def test_streaming_moves_a_perturbation_along_its_velocity(name):
    L = o.lattice(name)
    p = o.Params3(name, 9, 8, 7, 0.8, "bgk")
    f = np.zeros((L.V, 7, 8, 9))
    f[:, 3, 4, 4] = 1.0
    g = o.stream(p, f)
    for i in range(L.V):
        cx, cy, cz = L.xi[i]
        assert g[i, (3 + cz) % 7, (4 + cy) % 8, (4 + cx) % 9] == 1.0 and g[i].sum() == 1.0


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("coll", ["bgk", "rr"])
def test_shear_wave_decays_at_nu_k2(name, coll):
    """u_x = A sin(2 pi z / nz): amplitude decays as exp(-nu k^2 t), nu = cs^2 (tau - 1/2) (32 cells per
    wavelength on the standard lattices, 64 on the high-order ones, whose velocities reach 3 cells)."""
    L = o.lattice(name)
    nz, tau = (32 if name in ("D3Q19", "D3Q27") else 64), 0.8
    p = o.Params3(name, 2, 2, nz, tau, coll, hermite_order=2)
    k = 2 * np.pi / nz
    z = np.arange(nz)
    rho = np.ones((nz, 2, 2))
    u = np.zeros((3, nz, 2, 2))
    u[0] = 1e-3 * np.sin(k * z)[:, None, None]
    grad = np.zeros((3, 3, nz, 2, 2))
    grad[0, 2] = 1e-3 * k * np.cos(k * z)[:, None, None]
    f = o.init(p, rho, u, grad)
    nu = L.cs2 * (tau - 0.5)
    n = int(0.5 / (nu * k * k))
    a0 = np.abs(o.moments(p, f)[1][0]).max()
    f = o.step(p, f, n)
    rate = np.log(a0 / np.abs(o.moments(p, f)[1][0]).max()) / n
    assert rate == pytest.approx(nu * k * k, rel=0.04)
