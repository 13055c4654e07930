"""Pins of the oracle's Hermite coefficients a0^(n) (App. B) and a1^(n) (Sec. II.E, App. A, App. C).

Expected values come from: the closed forms of Eq. (HermiteCoeffEq); Gaussian
quadrature of the continuous Maxwellian; the Chapman-Enskog expansion of the
Hermite-projected Boltzmann equation (Eq. LBK_ProjectedOnH) closed with Euler's
equations, derived symbolically; the isothermal closed form
a1^(n) = sum_{i<j} (prod_{k != i,j} u_k) a1^(2)_{ij}; and the printed 2D forms of App. C.
"""
import itertools
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

from oracle import oracle as orc


def tup(*alpha):
    return sum(a << k for k, a in enumerate(alpha))


def alphas(n):
    return list(itertools.product((0, 1), repeat=n))


def closed_form_a0(alpha, rho, u, cs2, theta):
    """Eq. (HermiteCoeffEq) for n <= 4: rho [u^n + cs^2(theta-1) u^{n-2} delta + cs^4 (theta-1)^2 delta^2]."""
    n = len(alpha)
    d = lambda i, j: 1.0 if alpha[i] == alpha[j] else 0.0
    U = lambda *ks: math.prod(u[alpha[k]] for k in ks)
    e = cs2 * (theta - 1.0)
    if n == 0:
        return rho
    if n == 1:
        return rho * U(0)
    if n == 2:
        return rho * (U(0, 1) + e * d(0, 1))
    if n == 3:
        return rho * (U(0, 1, 2) + e * (U(0) * d(1, 2) + U(1) * d(0, 2) + U(2) * d(0, 1)))
    if n == 4:
        pair = U(0, 1) * d(2, 3) + U(0, 2) * d(1, 3) + U(0, 3) * d(1, 2) + U(1, 2) * d(0, 3) + U(1, 3) * d(0, 2) + U(2, 3) * d(0, 1)
        dd = d(0, 1) * d(2, 3) + d(0, 2) * d(1, 3) + d(0, 3) * d(1, 2)
        return rho * (U(0, 1, 2, 3) + e * pair + e * e * dd)
    raise ValueError


def herm_lib(alpha, xx, xy, cs2):
    ny = sum(alpha)
    nx = len(alpha) - ny
    c = math.sqrt(cs2)
    return He.hermeval(xx / c, [0] * nx + [1]) * c ** nx * He.hermeval(xy / c, [0] * ny + [1]) * c ** ny


def quadrature_a0(alpha, rho, u, cs2, theta, npts=30):
    """a0_alpha = int H_alpha(xi) f^eq(xi) dxi, f^eq the Maxwellian of Eq. (feq) with r T = cs^2 theta."""
    z, wz = He.hermegauss(npts)
    wz = wz / math.sqrt(2 * math.pi)
    s = math.sqrt(cs2 * theta)
    tot = 0.0
    for zi, wi in zip(z, wz):
        for zj, wj in zip(z, wz):
            tot += wi * wj * herm_lib(alpha, u[0] + s * zi, u[1] + s * zj, cs2)
    return rho * tot


RNG = np.random.default_rng(1234)
CASES = [(RNG.uniform(0.5, 2.0), RNG.uniform(-0.4, 0.4, 2), RNG.uniform(0.3, 0.8), th)
         for th in (1.0, 0.7, 1.3, 1.0, 0.9)]


@pytest.mark.parametrize("rho,u,cs2,theta", CASES)
def test_a0_recursion_matches_closed_form_and_quadrature(rho, u, cs2, theta):
    a0 = orc.a0(cs2, rho, u[0], u[1], theta)
    for n in range(5):
        for al in alphas(n):
            cf = closed_form_a0(al, rho, u, cs2, theta)
            q = quadrature_a0(al, rho, u, cs2, theta)
            assert abs(a0[n, tup(*al)] - cf) < 1e-13 * max(1, abs(cf))
            assert abs(a0[n, tup(*al)] - q) < 1e-12 * max(1, abs(q))


@pytest.mark.parametrize("name,neq", [("D2Q9", 2), ("D2Q9", 4), ("D2V17", 3), ("D2V37", 4)])
def test_equilibrium_reproduces_conserved_moments(name, neq):
    """sum f^(0) = rho, sum f^(0) xi = rho u, sum f^(0) xi^2 = rho u^2 + D rho cs^2 theta (Sec. II.A, II.D)."""
    L = orc.lattice(name)
    thetas = (1.0, 0.8, 1.2) if name == "D2V37" else (1.0,)
    for theta in thetas:
        rho, ux, uy = 1.1, 0.07, -0.05
        f = orc.expand(name, 0, neq, orc.a0(L.cs2, rho, ux, uy, theta))
        assert abs(f.sum() - rho) < 1e-14
        assert abs((f * L.cx).sum() - rho * ux) < 1e-14
        assert abs((f * L.cy).sum() - rho * uy) < 1e-14
        e2 = (f * (L.cx ** 2 + L.cy ** 2)).sum()
        assert abs(e2 - rho * (ux * ux + uy * uy + 2 * L.cs2 * theta)) < 1e-13


def random_sym2(rng):
    m = rng.normal(size=(2, 2))
    m = m + m.T
    return m


def tensor2(m):
    a = np.zeros((5, 16))
    for al in alphas(2):
        a[2, tup(*al)] = m[al[0], al[1]]
    return a


@pytest.mark.parametrize("seed", range(5))
def test_isothermal_recursion_matches_chapman_enskog_closed_form(seed):
    """Eq. (MalaspinasRecursiveRelation) with a0^(n) = rho u^n equals sum_{i<j} prod_{k!=i,j} u a1^(2)_ij."""
    rng = np.random.default_rng(seed)
    rho, u, cs2 = rng.uniform(0.5, 2), rng.uniform(-0.3, 0.3, 2), rng.uniform(0.3, 0.8)
    m = random_sym2(rng) * 1e-3
    a0 = orc.a0(cs2, rho, u[0], u[1], 1.0)
    a1 = orc.a1_recursive(cs2, rho, u[0], u[1], 1.0, False, 4, a0, tensor2(m))
    for n in (3, 4):
        for al in alphas(n):
            expect = 0.0
            for i, j in itertools.combinations(range(n), 2):
                expect += math.prod(u[al[k]] for k in range(n) if k not in (i, j)) * m[al[i], al[j]]
            assert abs(a1[n, tup(*al)] - expect) < 1e-15


def test_recursion_printed_2d_forms():
    """App. C 2D forms of a1_xxxx, a1_xxxy, a1_xxyy (thermal), given a1^(2), a1^(3)."""
    rng = np.random.default_rng(7)
    rho, (ux, uy), cs2, th = 1.3, rng.uniform(-0.3, 0.3, 2), 0.69, 1.17
    m = random_sym2(rng) * 1e-3
    a0 = orc.a0(cs2, rho, ux, uy, th)
    a1 = tensor2(m)
    # an a1^(3) of Chapman-Enskog form (symmetric) with a temperature-gradient part G
    G = rng.normal(size=2) * 1e-4
    u = (ux, uy)
    for al in alphas(3):
        a, b, g = al
        v = u[a] * m[b, g] + u[b] * m[a, g] + u[g] * m[a, b]
        v -= G[a] * (b == g) + G[b] * (a == g) + G[g] * (a == b)
        a1[3, tup(*al)] = v
    r = orc.a1_recursive(cs2, rho, ux, uy, th, True, 4, a0, a1)
    e = cs2 * (th - 1)
    xx, xy, yy = m[0, 0], m[0, 1], m[1, 1]
    xxx, xxy, xyy = a1[3, tup(0, 0, 0)], a1[3, tup(0, 0, 1)], a1[3, tup(0, 1, 1)]
    assert abs(r[4, tup(0, 0, 0, 0)] - (4 * ux * xxx + 6 * (e - ux * ux) * xx)) < 1e-15
    assert abs(r[4, tup(0, 0, 0, 1)] - ((3 * ux * xxy + uy * xxx) + 3 * (e - ux * ux) * xy - 3 * ux * uy * xx)) < 1e-15
    assert abs(r[4, tup(0, 0, 1, 1)] - (2 * (ux * xyy + uy * xxy) + (e - ux * ux) * yy + (e - uy * uy) * xx
                                        - 4 * ux * uy * xy)) < 1e-15


@pytest.mark.parametrize("seed", range(4))
def test_recursions_give_symmetric_tensors(seed):
    rng = np.random.default_rng(100 + seed)
    rho, u, cs2, th = 1.0, rng.uniform(-0.3, 0.3, 2), 0.7, rng.uniform(0.8, 1.2)
    m = random_sym2(rng) * 1e-3
    proj3 = rng.normal(size=8) * 1e-4  # arbitrary (non-symmetric) projected a1^(3)
    a1 = tensor2(m)
    a1[3, :8] = orc.a1_third_thermal(u[0], u[1], a1[2, :4], proj3)
    for thermal in (False, True):
        t = th if thermal else 1.0
        r = orc.a1_recursive(cs2, rho, u[0], u[1], t, thermal, 4, orc.a0(cs2, rho, u[0], u[1], t), a1)
        for n in (3, 4):
            for al in alphas(n):
                for perm in itertools.permutations(al):
                    assert abs(r[n, tup(*al)] - r[n, tup(*perm)]) < 1e-16


def test_thermal_third_order_reconstruction_is_a_projection():
    """App. C steps 1-4: an a1^(3) already of Chapman-Enskog form is returned unchanged; any input is mapped onto that form."""
    rng = np.random.default_rng(3)
    u = rng.uniform(-0.3, 0.3, 2)
    m = random_sym2(rng)
    G = rng.normal(size=2)

    def ce(Gv):
        out = np.zeros(8)
        for al in alphas(3):
            a, b, g = al
            out[tup(*al)] = (u[a] * m[b, g] + u[b] * m[a, g] + u[g] * m[a, b]
                             - Gv[a] * (b == g) - Gv[b] * (a == g) - Gv[g] * (a == b))
        return out

    a12 = tensor2(m)[2, :4]
    assert np.max(np.abs(orc.a1_third_thermal(u[0], u[1], a12, ce(G)) - ce(G))) < 1e-14
    rnd = rng.normal(size=8)
    out = orc.a1_third_thermal(u[0], u[1], a12, rnd)
    # the output is of CE form with the averaged estimates of Eq. (TempGradLBM)
    xx, xy, yy = m[0, 0], m[0, 1], m[1, 1]
    Gx = 0.5 * ((u[0] * xx - rnd[tup(0, 0, 0)] / 3) + (2 * u[1] * xy + u[0] * yy - rnd[tup(1, 1, 0)]))
    Gy = 0.5 * ((u[1] * yy - rnd[tup(1, 1, 1)] / 3) + (2 * u[0] * xy + u[1] * xx - rnd[tup(0, 0, 1)]))
    assert np.max(np.abs(out - ce(np.array([Gx, Gy])))) < 1e-14


# --------------------------------------------------------------------------------------------
# Chapman-Enskog derivation (symbolic): a1^(n) = -tau [d_t a0^(n) + d_g a0^(n+1)_{..g} + cs^2 sum_i d_{a_i} a0^(n-1)_{beta_i}]
# with time derivatives removed by Euler's equations (App. A), then compared with the recursions.
# --------------------------------------------------------------------------------------------

def _pairing_a0(sp, alpha, rho, u, e):
    """rho * sum over partial pairings of alpha: prod(pairs) e delta * prod(unpaired) u  (generalises Eq. HermiteCoeffEq)."""
    def rec(idx):
        if not idx:
            return sp.Integer(1)
        first, rest = idx[0], idx[1:]
        tot = u[alpha[first]] * rec(rest)
        for k, other in enumerate(rest):
            if alpha[first] == alpha[other]:
                tot += e * rec(rest[:k] + rest[k + 1:])
        return tot
    return rho * rec(list(range(len(alpha))))


def test_pairing_form_matches_quadrature_to_order_five():
    sp = pytest.importorskip("sympy")
    rho, u, cs2, th = 1.2, (0.11, -0.07), 0.55, 1.25
    for n in range(6):
        for al in alphas(n):
            v = float(_pairing_a0(sp, al, sp.Float(rho), [sp.Float(u[0]), sp.Float(u[1])], sp.Float(cs2 * (th - 1))))
            assert abs(v - quadrature_a0(al, rho, u, cs2, th)) < 1e-12


def _ce_a1(thermal, n_max=4, seed=0):
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(seed)
    rho, ux, uy, th, tau, cs2 = sp.symbols("rho ux uy th tau cs2", positive=True)
    q = [rho, ux, uy, th]
    # gradients of (rho, ux, uy, th) along x and y
    grad = {(v, g): sp.Symbol("d%d_%d" % (i, g)) for i, v in enumerate(q) for g in (0, 1)}
    u = [ux, uy]
    D = 2
    div = grad[(ux, 0)] + grad[(uy, 1)]
    # Euler time derivatives (App. A); isothermal: theta fixed, p = rho cs^2
    dt = {rho: -(ux * grad[(rho, 0)] + uy * grad[(rho, 1)]) - rho * div}
    for a, ua in enumerate(u):
        if thermal:
            dp = cs2 * (th * grad[(rho, a)] + rho * grad[(th, a)])
        else:
            dp = cs2 * grad[(rho, a)]
        dt[ua] = -(ux * grad[(ua, 0)] + uy * grad[(ua, 1)]) - dp / rho
    dt[th] = (-(ux * grad[(th, 0)] + uy * grad[(th, 1)]) - sp.Rational(2, D) * th * div) if thermal else 0
    e = cs2 * (th - 1) if thermal else 0
    thv = th if thermal else 1

    def a0(alpha):
        return _pairing_a0(sp, alpha, rho, u, e)

    def ddt(expr):
        return sum(sp.diff(expr, v) * dt[v] for v in q)

    def ddx(expr, g):
        return sum(sp.diff(expr, v) * grad[(v, g)] for v in q)

    a1 = {}
    for n in range(2, n_max + 1):
        for al in alphas(n):
            s = ddt(a0(al)) + sum(ddx(a0(al + (g,)), g) for g in (0, 1))
            s += cs2 * sum(ddx(a0(al[:i] + al[i + 1:]), al[i]) for i in range(n))
            a1[al] = -tau * s
    vals = {rho: rng.uniform(0.6, 1.6), ux: rng.uniform(-0.3, 0.3), uy: rng.uniform(-0.3, 0.3), tau: 0.8,
            cs2: 0.697953322019683, th: rng.uniform(0.7, 1.3) if thermal else 1}
    for k, s in grad.items():
        vals[s] = 0.0 if (not thermal and k[0] is th) else rng.normal() * 1e-2
    num = {al: float(sp.N(expr.subs(vals), 30)) for al, expr in a1.items()}
    env = {str(k): float(vals[k]) for k in (rho, ux, uy, tau, cs2)}
    env["th"] = float(vals[th]) if thermal else 1.0
    env["grad"] = {(str(k[0]), k[1]): float(vals[s]) for k, s in grad.items()}
    return num, env


def test_chapman_enskog_second_order_matches_viscous_stress():
    """The symbolic CE a1^(2) equals -tau rho cs^2 theta (S - (2/D) div u delta) (App. A) -- pins the derivation."""
    num, env = _ce_a1(True, n_max=2, seed=5)
    g = env["grad"]
    du = [[g[("ux", 0)], g[("ux", 1)]], [g[("uy", 0)], g[("uy", 1)]]]  # du[a][b] = d_b u_a
    div = du[0][0] + du[1][1]
    for al in alphas(2):
        a, b = al
        S = du[b][a] + du[a][b] - (div if a == b else 0.0)
        expect = -env["tau"] * env["rho"] * env["cs2"] * env["th"] * S
        assert abs(num[al] - expect) < 1e-14


@pytest.mark.parametrize("thermal,seed", [(False, 11), (True, 12), (True, 13)])
def test_recursion_matches_chapman_enskog_expansion(thermal, seed):
    """Eqs. (MalaspinasRecursiveRelation) / (RecursiveRelation_ThermalCase) reproduce the CE a1^(n) exactly."""
    num, env = _ce_a1(thermal, n_max=4, seed=seed)
    rho, ux, uy, cs2, th = env["rho"], env["ux"], env["uy"], env["cs2"], env["th"]
    a1 = np.zeros((5, 16))
    for al in alphas(2):
        a1[2, tup(*al)] = num[al]
    if thermal:
        for al in alphas(3):
            a1[3, tup(*al)] = num[al]
    a0 = orc.a0(cs2, rho, ux, uy, th)
    r = orc.a1_recursive(cs2, rho, ux, uy, th, thermal, 4, a0, a1)
    for n in ((3, 4) if not thermal else (4,)):
        for al in alphas(n):
            assert abs(r[n, tup(*al)] - num[al]) < 1e-13 * max(1.0, abs(num[al])), (n, al)
