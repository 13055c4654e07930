"""Python access to the FP64 CPU oracle (oracle/lbm_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by the smoke check and by the
CPU-baseline / reference leg of bench.py; never by the product package.  It
shares no code with the CUDA path: arrays are plain numpy float64 in the
oracle's own velocity order, SoA [V][ny][nx].

The arithmetic lives in lbm_oracle.c (paper: Sec. II.E, Sec. III.A, App. A-D).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

D2Q9, D2V17, D2V37 = 0, 1, 2
BGK, PR, RR = 0, 1, 2
PERIODIC, ZERO_GRADIENT = 0, 1
LATTICE_NAMES = {"D2Q9": D2Q9, "D2V17": D2V17, "D2V37": D2V37}
COLLISION_NAMES = {"bgk": BGK, "pr": PR, "rr": RR}
MAXQ = 64
MAXN = 4


def build_oracle(force: bool = False) -> str:
    """Compile lbm_oracle.c into oracle/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcLattice(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int), ("cx", ctypes.c_int * MAXQ), ("cy", ctypes.c_int * MAXQ),
                ("w", ctypes.c_double * MAXQ), ("cs2", ctypes.c_double), ("nmax", ctypes.c_int),
                ("keep", (ctypes.c_int * (MAXN + 1)) * (MAXN + 1))]


class OrcParams(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("hermite_order", ctypes.c_int), ("reg_order", ctypes.c_int),
                ("collision", ctypes.c_int), ("thermal", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("tau", ctypes.c_double), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("tau3", ctypes.c_double), ("tau4", ctypes.c_double), ("a1_source", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.orc_hermite.restype = ctypes.c_double
        _lib.orc_hermite.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        _lib.orc_a0.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, dp]
        _lib.orc_a1_recursive.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_int, dp, dp]
        _lib.orc_a1_third_thermal.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp, dp]
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Lattice:
    V: int
    cx: np.ndarray
    cy: np.ndarray
    w: np.ndarray
    cs2: float
    nmax: int
    keep: np.ndarray


def lattice(lat) -> Lattice:
    lat = LATTICE_NAMES.get(lat, lat)
    L = OrcLattice()
    if lib().orc_lattice_get(int(lat), ctypes.byref(L)) != 0:
        raise ValueError("unknown lattice %r" % lat)
    V = L.V
    keep = np.array([[L.keep[a][b] for b in range(MAXN + 1)] for a in range(MAXN + 1)], dtype=bool)
    return Lattice(V, np.array(L.cx[:V]), np.array(L.cy[:V]), np.array(L.w[:V]), L.cs2, L.nmax, keep)


def hermite(n: int, tuple_: int, xx: float, xy: float, cs2: float) -> float:
    return lib().orc_hermite(n, tuple_, xx, xy, cs2)


def a0(cs2, rho, ux, uy, theta, nmax=4) -> np.ndarray:
    out = np.zeros((MAXN + 1, 16))
    lib().orc_a0(cs2, rho, ux, uy, theta, nmax, _dp(out))
    return out


def a1_recursive(cs2, rho, ux, uy, theta, thermal, nmax, a0_t, a1_t) -> np.ndarray:
    a0_t = np.ascontiguousarray(a0_t, dtype=np.float64)
    out = np.array(a1_t, dtype=np.float64, copy=True)
    lib().orc_a1_recursive(cs2, rho, ux, uy, theta, int(thermal), nmax, _dp(a0_t), _dp(out))
    return out


def a1_third_thermal(ux, uy, a1_2, a1_3_proj) -> np.ndarray:
    a1_2 = np.ascontiguousarray(a1_2, dtype=np.float64)
    a1_3_proj = np.ascontiguousarray(a1_3_proj, dtype=np.float64)
    out = np.zeros(8)
    lib().orc_a1_third_thermal(ux, uy, _dp(a1_2), _dp(a1_3_proj), _dp(out))
    return out


def params(lattice_, nx, ny, tau, collision="rr", hermite_order=2, reg_order=0, thermal=False,
           bc_x=PERIODIC, bc_y=PERIODIC, tau3=0.0, tau4=0.0, a1_source=0) -> OrcParams:
    """tau is the order-2 (viscous) relaxation time; tau3 / tau4 those of the order-3 / order-4
    coefficients of f^(1) (0 = tau).  a1_source (RR only): 0 projection, 1 finite differences."""
    return OrcParams(LATTICE_NAMES.get(lattice_, lattice_), hermite_order, reg_order,
                     COLLISION_NAMES.get(collision, collision), int(thermal), nx, ny, float(tau), bc_x, bc_y,
                     float(tau3), float(tau4), int(a1_source))


def expand(lat, nmin, nmax, coef) -> np.ndarray:
    L = OrcLattice()
    lib().orc_lattice_get(int(LATTICE_NAMES.get(lat, lat)), ctypes.byref(L))
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    out = np.zeros(L.V)
    lib().orc_expand(ctypes.byref(L), nmin, nmax, _dp(coef), _dp(out))
    return out


def collide(p: OrcParams, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    if lib().orc_collide(ctypes.byref(p), _dp(f), _dp(out)) != 0:
        raise ValueError("orc_collide rejected the parameters")
    return out


def collide_fd(p: OrcParams, f: np.ndarray, grad) -> np.ndarray:
    """One cell's collision with a1 from the given gradients (d ux/dx, d ux/dy, d uy/dx, d uy/dy, d theta/dx,
    d theta/dy); p.a1_source must be 1."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(grad, dtype=np.float64)
    out = np.empty_like(f)
    if lib().orc_collide_fd(ctypes.byref(p), _dp(f), _dp(g), _dp(out)) != 0:
        raise ValueError("orc_collide_fd rejected the parameters")
    return out


def step(p: OrcParams, f: np.ndarray, n: int = 1) -> np.ndarray:
    a = np.ascontiguousarray(f, dtype=np.float64).copy()
    b = np.empty_like(a)
    for _ in range(n):
        if lib().orc_step(ctypes.byref(p), _dp(a), _dp(b)) != 0:
            raise ValueError("orc_step rejected the parameters")
        a, b = b, a
    return a


def step_cells(p: OrcParams, f: np.ndarray, cells: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    V = f.shape[0]
    out = np.empty((len(cells), V))
    if lib().orc_step_cells(ctypes.byref(p), _dp(f), len(cells),
                            cells.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _dp(out)) != 0:
        raise ValueError("orc_step_cells rejected the parameters")
    return out


def collide_delta(p: OrcParams, f: np.ndarray, delta) -> np.ndarray:
    """One cell's isothermal RR collision with (xx, xy, yy) = delta added to the projected a1^(2) before the
    recursion (Eq. MalaspinasRecursiveRelation builds the higher orders from the corrected a1^(2))."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    out = np.empty_like(f)
    if lib().orc_collide_delta(ctypes.byref(p), _dp(f), _dp(d), _dp(out)) != 0:
        raise ValueError("orc_collide_delta rejected the parameters")
    return out


def step_delta(p: OrcParams, f: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """One step whose collision adds delta[3][ny][nx] = (xx, xy, yy) to each cell's projected a1^(2)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    if d.shape != (3, p.ny, p.nx):
        raise ValueError("delta must be [3][ny][nx]")
    out = np.empty_like(f)
    if lib().orc_step_delta(ctypes.byref(p), _dp(f), _dp(d), _dp(out)) != 0:
        raise ValueError("orc_step_delta rejected the parameters")
    return out


def closure_delta(y: np.ndarray, u0: float, tau: float, nx: int, ny: int) -> np.ndarray:
    """The learned closure's correction of a1^(2) from the network outputs y[nx*ny][>=3] (the subgrid stress
    (xx, xy, yy) / u0^2): Delta a1^(2) = u0^2 y / (1 - 1/tau), so that the relaxed non-equilibrium part
    (1 - 1/tau) a1^(2) of the post-collision state carries the predicted stress.  Returned as [3][ny][nx]."""
    y = np.asarray(y, dtype=np.float64)[:, :3]
    return (u0 * u0 * y / (1.0 - 1.0 / tau)).T.reshape(3, ny, nx)


def init(p: OrcParams, rho, ux, uy, T=None, grad_u=None) -> np.ndarray:
    V = lattice(p.lattice).V
    c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    rho, ux, uy, T, grad_u = c(rho), c(ux), c(uy), c(T), c(grad_u)
    f = np.empty((V, p.ny, p.nx))
    nul = ctypes.POINTER(ctypes.c_double)()
    rc = lib().orc_init(ctypes.byref(p), _dp(rho), _dp(ux), _dp(uy), _dp(T) if T is not None else nul,
                        _dp(grad_u) if grad_u is not None else nul, _dp(f))
    if rc != 0:
        raise ValueError("orc_init rejected the parameters")
    return f


def moments(p: OrcParams, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    shp = (p.ny, p.nx)
    rho, ux, uy, th = (np.empty(shp) for _ in range(4))
    lib().orc_moments(ctypes.byref(p), _dp(f), _dp(rho), _dp(ux), _dp(uy), _dp(th))
    return rho, ux, uy, th


def conservation(p: OrcParams, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_conservation(ctypes.byref(p), _dp(f), _dp(out))
    return out


def num_threads() -> int:
    return lib().orc_num_threads()


def tau_from_nu(cs2: float, nu: float, theta_ref: float = 1.0) -> float:
    """Shifted relaxation time of the discrete scheme: nu = cs^2 theta (tau - 1/2) (Sec. II.B, Sec. III.A)."""
    return nu / (cs2 * theta_ref) + 0.5


def vorticity(ux: np.ndarray, uy: np.ndarray) -> np.ndarray:
    """omega = d_x u_y - d_y u_x with fourth-order centred differences on a periodic grid (Sec. III.B)."""
    def d(g, axis):
        return (-np.roll(g, -2, axis) + 8 * np.roll(g, -1, axis) - 8 * np.roll(g, 1, axis) + np.roll(g, 2, axis)) / 12.0
    return d(uy, 1) - d(ux, 0)


def diagnostics(rho, ux, uy):
    """Domain mean and standard deviation of u^2 and of the enstrophy density omega^2/2 (Sec. III.B)."""
    u2 = ux * ux + uy * uy
    w = vorticity(ux, uy)
    ens = 0.5 * w * w
    return np.array([u2.mean(), u2.std(), ens.mean(), ens.std()])
