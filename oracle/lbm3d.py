"""FP64 reference of the three-dimensional lattices of Tab. II (test infrastructure only: only tests/,
__graft_entry__.smoke() and bench.py's CPU legs use it; the product never imports it).

Plain numpy over all cells at once, in the paper's tensor-index notation: a Hermite tensor or a Hermite
coefficient of order n is stored for every index tuple alpha in {x, y, z}^n (3^n entries), so the
multiplicities A^(n) of App. C come from summing over all tuples, not from a table.  Steps, for
isothermal flows (theta = 1):
  - lattices built from Tab. II's group representatives by every permutation and reflection;
  - Hermite tensors by the recursion H^(n+1)_{alpha beta} = xi_beta H^(n)_alpha
    - cs^2 sum_k delta_{alpha_k beta} H^(n-1)_{alpha without k} (App. B);
  - a0^(n) by App. B's recursion with theta = 1: a0^(n)_{alpha_1..alpha_n} = u_{alpha_n} a0^(n-1);
  - f^(0) = w_i sum_n 1/(n! cs^2n) sum_alpha H_alpha a0_alpha over the lattice's kept tensors;
  - BGK f* = f - (f - f^(0))/tau; PR a1^(n) = sum_i H_alpha (f_i - f_i^(0)) for n = 2..N; RR a1^(2)
    projected and a1^(n >= 3) by Eq. MalaspinasRecursiveRelation, all rebuilt with (1 - 1/tau);
  - pull streaming f_i(x) <- f_i*(x - xi_i), periodic or clamped (zero-gradient) per axis.
Populations are f[V][nz][ny][nx].  Readings (kept tensors of Tab. II): D3Q19 keeps the orders <= 3 except
H_xxx-type and H_xyz; D3Q27 keeps every tensor whose exponents are all <= 2 (its complete basis, so
H_xxyz-type is kept although the table marks it out; the Gram-matrix pin shows it is orthonormal there);
D3V39 every tensor of order <= 3; D3Q103 every tensor of order <= 4.
"""
from __future__ import annotations

import functools
import itertools
import math
from dataclasses import dataclass

import numpy as np

# Tab. II: group representative, weight (per lattice), and 1/cs
GROUPS = {
    "D3Q19": [((0, 0, 0), 1 / 3), ((1, 0, 0), 1 / 18), ((1, 1, 0), 1 / 36)],
    "D3Q27": [((0, 0, 0), 8 / 27), ((1, 0, 0), 2 / 27), ((1, 1, 0), 1 / 54), ((1, 1, 1), 1 / 216)],
    "D3V39": [((0, 0, 0), 1 / 12), ((1, 0, 0), 1 / 12), ((1, 1, 1), 1 / 27), ((2, 0, 0), 2 / 135),
              ((2, 2, 0), 1 / 432), ((3, 0, 0), 1 / 1620)],
    "D3Q103": [((0, 0, 0), 0.032633351764471159466), ((1, 0, 0), 0.097656833590334574221),
               ((1, 1, 1), 0.028097750290257335627), ((2, 0, 0), 0.001045259560430061466),
               ((2, 1, 0), 0.005705329016894815990), ((2, 2, 0), 0.000611939269829747839),
               ((2, 2, 2), 0.000155964159374283722), ((3, 0, 0), 0.000284443251800055207),
               ((3, 1, 1), 0.000130698375985191585), ((3, 3, 3), 0.000001223194501323058)],
}
INV_CS = {"D3Q19": math.sqrt(3.0), "D3Q27": math.sqrt(3.0), "D3V39": math.sqrt(1.5),
          "D3Q103": 1.19697977039307435897239}
NMAX = {"D3Q19": 3, "D3Q27": 6, "D3V39": 3, "D3Q103": 4}
PERIODIC, ZERO_GRADIENT = 0, 1


def kept(lattice: str, e) -> bool:
    """Whether the Hermite tensor with exponents e = (n_x, n_y, n_z) belongs to the lattice's basis."""
    a = sorted(e, reverse=True)
    n = sum(a)
    if lattice == "D3Q19":
        return n <= 3 and a[0] <= 2 and a[2] == 0
    if lattice == "D3Q27":
        return a[0] <= 2
    if lattice == "D3V39":
        return n <= 3
    if lattice == "D3Q103":
        return n <= 4
    raise ValueError(lattice)


def orbit(rep):
    """Every permutation and reflection of a group representative (Tab. II)."""
    out = set()
    for p in itertools.permutations(rep):
        for s in itertools.product((1, -1), repeat=3):
            out.add(tuple(a * b for a, b in zip(p, s)))
    return sorted(out)


@dataclass(frozen=True)
class Lattice3:
    name: str
    xi: np.ndarray   # (V, 3) integer velocities
    w: np.ndarray    # (V,)
    cs2: float
    nmax: int

    @property
    def V(self):
        return self.xi.shape[0]


@functools.lru_cache(maxsize=None)
def lattice(name: str) -> Lattice3:
    xi, w = [], []
    for rep, wt in GROUPS[name]:
        o = orbit(rep)
        xi += o
        w += [wt] * len(o)
    return Lattice3(name, np.array(xi, dtype=np.int64), np.array(w, dtype=np.float64), 1.0 / INV_CS[name] ** 2,
                    NMAX[name])


def tuples(n):
    return itertools.product(range(3), repeat=n)


def exponents(alpha):
    return tuple(alpha.count(d) for d in range(3))


@functools.lru_cache(maxsize=None)
def hermite(name: str, nmax: int = 6):
    """H[alpha] = H^(n)_alpha(xi_i) for every tuple alpha of length <= nmax, each an array over the V
    velocities, by the recursion of App. B."""
    L = lattice(name)
    xi = L.xi.astype(np.float64)
    H = {(): np.ones(L.V)}
    for n in range(nmax):
        for alpha in tuples(n):
            for beta in range(3):
                v = xi[:, beta] * H[alpha]
                for k in range(n):
                    if alpha[k] == beta:
                        v = v - L.cs2 * H[alpha[:k] + alpha[k + 1:]]
                H[alpha + (beta,)] = v
    return H


@dataclass
class Params3:
    lattice: str
    nx: int
    ny: int
    nz: int
    tau: float                 # tau-bar of the discrete scheme (Sec. III.A)
    collision: str = "rr"      # "bgk", "pr", "rr"
    hermite_order: int = 2     # N of f^(0)
    reg_order: int = 0         # N of f^(1); 0 = lattice maximum
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)

    def orders(self):
        L = lattice(self.lattice)
        neq = self.hermite_order
        nreg = self.reg_order or L.nmax
        if not (1 <= neq <= L.nmax and 2 <= nreg <= L.nmax) or not self.tau > 0.5:
            raise ValueError("orders or tau out of range")
        return neq, nreg


def equilibrium_coefficients(rho, u, nmax):
    """a0^(n) for n <= nmax, isothermal (App. B with theta = 1): a0 = rho; a0^(n)_{alpha, beta} =
    u_beta a0^(n-1)_alpha.  rho (N,), u (3, N)."""
    a0 = {(): rho}
    for n in range(nmax):
        for alpha in tuples(n):
            for beta in range(3):
                a0[alpha + (beta,)] = u[beta] * a0[alpha]
    return a0


def expand(name, coef, nmin, nmax):
    """f_i = w_i sum_{n=nmin..nmax} 1/(n! cs^2n) sum_{alpha kept} H_alpha(xi_i) coef_alpha  -> (V, N)."""
    L = lattice(name)
    H = hermite(name)
    out = None
    for n in range(nmin, nmax + 1):
        scale = 1.0 / (math.factorial(n) * L.cs2 ** n)
        for alpha in tuples(n):
            if not kept(name, exponents(alpha)):
                continue
            term = np.outer(H[alpha], coef[alpha]) * scale
            out = term if out is None else out + term
    return L.w[:, None] * out


def cell_moments(name, f):
    """rho (N,) and u (3, N) of populations f (V, N) (Sec. II.A)."""
    L = lattice(name)
    rho = f.sum(axis=0)
    u = (L.xi.T.astype(np.float64) @ f) / rho
    return rho, u


def project(name, g, n):
    """sum_i H^(n)_alpha(xi_i) g_i for every tuple of length n -> dict alpha -> (N,)."""
    H = hermite(name)
    return {alpha: H[alpha] @ g for alpha in tuples(n)}


def a1_recursive(rho, u, a0, a1, nreg):
    """Eq. MalaspinasRecursiveRelation (isothermal): for n >= 3,
    a1_{alpha_1..alpha_n} = u_{alpha_n} a1_{alpha_1..alpha_{n-1}} + (1/rho) sum_{l<n} a0_{beta_l} a1_{alpha_l alpha_n},
    beta_l = alpha without positions l and n.  a1 holds the order-2 tuples on entry."""
    for n in range(3, nreg + 1):
        for alpha in tuples(n):
            v = u[alpha[-1]] * a1[alpha[:-1]]
            for l in range(n - 1):
                beta = alpha[:l] + alpha[l + 1:n - 1]
                v = v + a0[beta] * a1[(alpha[l], alpha[-1])] / rho
            a1[alpha] = v
    return a1


def collide(p: Params3, f):
    """One collision of every cell: f (V, N) -> (V, N)."""
    neq, nreg = p.orders()
    rho, u = cell_moments(p.lattice, f)
    a0 = equilibrium_coefficients(rho, u, max(neq, nreg))
    feq = expand(p.lattice, a0, 0, neq)
    if p.collision == "bgk":
        return f - (f - feq) / p.tau
    g = f - feq
    a1 = {}
    if p.collision == "pr":
        for n in range(2, nreg + 1):
            a1.update(project(p.lattice, g, n))
    elif p.collision == "rr":
        a1.update(project(p.lattice, g, 2))
        a1_recursive(rho, u, a0, a1, nreg)
    else:
        raise ValueError(p.collision)
    return feq + (1.0 - 1.0 / p.tau) * expand(p.lattice, a1, 2, nreg)


def _source(n, c, bc):
    s = np.arange(n) - c
    return np.mod(s, n) if bc == PERIODIC else np.clip(s, 0, n - 1)


def stream(p: Params3, f):
    """Pull streaming f_i(x) <- f_i(x - xi_i): f (V, nz, ny, nx)."""
    L = lattice(p.lattice)
    out = np.empty_like(f)
    for i in range(L.V):
        cx, cy, cz = (int(v) for v in L.xi[i])
        ix = _source(p.nx, cx, p.bc[0])
        iy = _source(p.ny, cy, p.bc[1])
        iz = _source(p.nz, cz, p.bc[2])
        out[i] = f[i][np.ix_(iz, iy, ix)]
    return out


def step(p: Params3, f, n=1):
    """n steps of pull streaming then collision on f (V, nz, ny, nx)."""
    L = lattice(p.lattice)
    for _ in range(n):
        g = stream(p, f)
        f = collide(p, g.reshape(L.V, -1)).reshape(g.shape)
    return f


def init(p: Params3, rho, u, grad=None):
    """f = f^(0) + f^(1) (Sec. III.B): rho (nz, ny, nx), u (3, nz, ny, nx); grad[a][b] = d u_a / d x_b
    (3, 3, nz, ny, nx) or None; a1^(2)_ab = -tau rho cs^2 (d_a u_b + d_b u_a) (isothermal), continued to
    every order of the lattice by Eq. MalaspinasRecursiveRelation (as in two dimensions)."""
    L = lattice(p.lattice)
    neq, _ = p.orders()
    shape = rho.shape
    r = rho.reshape(-1)
    uu = u.reshape(3, -1)
    f = expand(p.lattice, equilibrium_coefficients(r, uu, neq), 0, neq)
    if grad is not None:
        g = grad.reshape(3, 3, -1)
        a1 = {}
        for a, b in tuples(2):
            a1[(a, b)] = -p.tau * r * L.cs2 * (g[b, a] + g[a, b])
        a1_recursive(r, uu, equilibrium_coefficients(r, uu, L.nmax), a1, L.nmax)
        f = f + expand(p.lattice, a1, 2, L.nmax)
    return f.reshape((L.V,) + shape)


def moments(p: Params3, f):
    """rho (nz, ny, nx) and u (3, nz, ny, nx) of f (V, nz, ny, nx)."""
    L = lattice(p.lattice)
    rho, u = cell_moments(p.lattice, f.reshape(L.V, -1))
    return rho.reshape(f.shape[1:]), u.reshape((3,) + f.shape[1:])
