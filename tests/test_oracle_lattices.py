"""Pins of the oracle's lattice tables and Hermite tensors (App. C, App. D, Tab. I).

The expected values come from the printed table (tests/golden/table1_lattices.json),
from quadrature identities that any lattice of Tab. I must satisfy, and from
numpy's probabilists' Hermite polynomials; none from the oracle itself.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

from oracle import oracle as orc

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_lattices.json")))


def _eval(expr):
    return eval(expr, {"sqrt": math.sqrt})


def _orbit(p, q):
    return {(sp * a, sq * b) for a, b in ((p, q), (q, p)) for sp in (1, -1) for sq in (1, -1)}


@pytest.mark.parametrize("name", ["D2Q9", "D2V17", "D2V37"])
def test_groups_and_weights_match_table1(name):
    L = orc.lattice(name)
    g = GOLD[name]
    if name == "D2Q9":
        weights = [_eval(w) for w in g["weights_reading"]]
    elif name == "D2V17":
        weights = [_eval(w) for w in g["weights_closed_form"]]
    else:
        weights = [float(w) for w in g["weights"]]
    vel = {(int(a), int(b)): w for a, b, w in zip(L.cx, L.cy, L.w)}
    assert len(vel) == L.V == sum(g["p"])
    for (p, q), count, w in zip(g["groups"], g["p"], weights):
        orbit = _orbit(p, q)
        assert len(orbit) == count
        for v in orbit:
            assert abs(vel[v] - w) <= 1e-15
    assert abs(1.0 / math.sqrt(L.cs2) - _eval(g["inv_cs"])) <= 1e-14


@pytest.mark.parametrize("name,order", [("D2Q9", 5), ("D2V17", 7), ("D2V37", 9)])
def test_quadrature_reproduces_gaussian_moments(name, order):
    """sum_i w_i xi_x^p xi_y^q equals the moment of the weight function up to the quadrature degree (Eq. 29)."""
    L = orc.lattice(name)
    cs2 = L.cs2

    def gauss_moment(k):  # E[X^k], X ~ N(0, cs2)
        return 0.0 if k % 2 else cs2 ** (k // 2) * math.prod(range(k - 1, 0, -2))

    for p in range(order + 1):
        for q in range(order + 1 - p):
            lhs = np.sum(L.w * L.cx.astype(float) ** p * L.cy.astype(float) ** q)
            assert abs(lhs - gauss_moment(p) * gauss_moment(q)) < 1e-13, (p, q)


def test_d2q9_printed_alignment_fails_isotropy():
    """Reading of the shifted D2Q9 column: the as-printed alignment breaks sum w xi_x^2 = cs^2."""
    rows = GOLD["D2Q9"]["weights_as_printed_rows"]
    w = {(0, 0): _eval(rows["(0,0)"]), (1, 0): _eval(rows["(1,0)"]), (1, 1): _eval(rows["(1,1)"])}
    tot = sum(w[g] * len(_orbit(*g)) for g in w)
    second = sum(w[g] * sum(v[0] ** 2 for v in _orbit(*g)) for g in w)
    assert abs(tot - 1.0) > 0.1 or abs(second - 1.0 / 3.0) > 0.05


def _herm_lib(nx, ny, xx, xy, cs2):
    """c^n He_nx(xi_x/c) He_ny(xi_y/c) from numpy's probabilists' Hermite series."""
    c = math.sqrt(cs2)
    ex = He.hermeval(xx / c, [0] * nx + [1]) * c ** nx
    ey = He.hermeval(xy / c, [0] * ny + [1]) * c ** ny
    return ex * ey


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4])
def test_hermite_tensors_match_library(n):
    rng = np.random.default_rng(n)
    for t in range(1 << n):
        ny = bin(t).count("1")
        for _ in range(5):
            xx, xy, cs2 = rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(0.2, 1.0)
            assert abs(orc.hermite(n, t, xx, xy, cs2) - _herm_lib(n - ny, ny, xx, xy, cs2)) < 1e-12


def test_hermite_2d_printed_forms():
    """App. C 2D forms (H_xx, H_xxy, H_xxxx, H_xxxy, H_xxyy) at an arbitrary point."""
    x, y, c2 = 1.3, -0.7, 0.41
    T = lambda *a: sum(v << k for k, v in enumerate(a))
    assert abs(orc.hermite(2, T(0, 0), x, y, c2) - (x * x - c2)) < 1e-14
    assert abs(orc.hermite(3, T(0, 0, 1), x, y, c2) - (x * x - c2) * y) < 1e-14
    assert abs(orc.hermite(3, T(0, 0, 0), x, y, c2) - (x * x - 3 * c2) * x) < 1e-14
    assert abs(orc.hermite(4, T(0, 0, 0, 0), x, y, c2) - (x ** 4 - 6 * c2 * x * x + 3 * c2 * c2)) < 1e-13
    assert abs(orc.hermite(4, T(0, 0, 0, 1), x, y, c2) - (x * x - 3 * c2) * x * y) < 1e-14
    assert abs(orc.hermite(4, T(0, 0, 1, 1), x, y, c2) - (x * x - c2) * (y * y - c2)) < 1e-14


def _kept_basis(L):
    return [(a, b) for a in range(5) for b in range(5) if L.keep[a, b]]


@pytest.mark.parametrize("name", ["D2Q9", "D2V17", "D2V37"])
def test_gram_matrix_diagonal_on_kept_basis(name):
    """sum_i w_i H_(a,b) H_(c,d) = cs^{2(a+b)} a! b! delta (App. D orthogonality), on the kept basis of Tab. I."""
    L = orc.lattice(name)
    basis = _kept_basis(L)
    expect_size = {"D2Q9": 9, "D2V17": 10, "D2V37": 15}[name]
    assert len(basis) == expect_size
    H = np.array([[_herm_lib(a, b, x, y, L.cs2) for (a, b) in basis] for x, y in zip(L.cx, L.cy)])
    G = H.T @ (L.w[:, None] * H)
    D = np.diag([L.cs2 ** (a + b) * math.factorial(a) * math.factorial(b) for a, b in basis])
    assert np.max(np.abs(G - D)) < 1e-13


@pytest.mark.parametrize("name,excluded", [("D2Q9", [(3, 0), (4, 0), (3, 1)]), ("D2V17", [(4, 0), (3, 1), (2, 2)])])
def test_excluded_tensors_are_not_in_basis(name, excluded):
    """Tab. I bottom: the tensors marked as outside the basis are absent from the oracle's kept set."""
    L = orc.lattice(name)
    for a, b in excluded:
        assert not L.keep[a, b] and not L.keep[b, a]
