"""Seeded synthetic inputs: macroscopic fields and run parameters only.

This module is shared by the CUDA path's tests and benchmark and by the oracle
tests.  It holds none of the method's arithmetic (no lattice, no Hermite
expansion, no collision): it produces density / velocity / temperature fields,
their analytic velocity gradients, and the physical parameters (u0, nu, step
counts) of the workloads of Sec. III, given the sound speed of whichever
lattice the caller uses.

Gradients are returned as one [4, ny, nx] array in the order
d ux/dx, d ux/dy, d uy/dx, d uy/dy.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Fields:
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    theta: np.ndarray | None = None
    grad_u: np.ndarray | None = None


def _centres(n: int, length: float) -> np.ndarray:
    # cell-centred coordinate x* = (i + 1/2) / L
    return (np.arange(n, dtype=np.float64) + 0.5) / length


def double_shear_layer(L: int, u0: float, kappa: float = 80.0, delta: float = 0.05, ny: int | None = None) -> Fields:
    """Doubly periodic shear layer of Sec. III.B on an L x L grid.

    u_x = u0 tanh(kappa (y* - 1/4)) for y* <= 1/2, u0 tanh(kappa (3/4 - y*)) otherwise;
    u_y = u0 delta sin(2 pi (x* + 1/4)); rho = 1.  Gradients are analytic.
    """
    ny = L if ny is None else ny
    xs = _centres(L, L)
    ys = _centres(ny, L)
    X, Y = np.meshgrid(xs, ys)  # [ny, nx]
    lower = Y <= 0.5
    ux = np.where(lower, u0 * np.tanh(kappa * (Y - 0.25)), u0 * np.tanh(kappa * (0.75 - Y)))
    uy = u0 * delta * np.sin(2.0 * np.pi * (X + 0.25))
    sech2_lo = 1.0 / np.cosh(kappa * (Y - 0.25)) ** 2
    sech2_hi = 1.0 / np.cosh(kappa * (0.75 - Y)) ** 2
    dux_dy = np.where(lower, u0 * kappa * sech2_lo, -u0 * kappa * sech2_hi) / L
    duy_dx = u0 * delta * 2.0 * np.pi * np.cos(2.0 * np.pi * (X + 0.25)) / L
    grad = np.stack([np.zeros_like(ux), dux_dy, duy_dx, np.zeros_like(ux)])
    return Fields(np.ones_like(ux), ux, uy, None, grad)


def shear_layer_params(L: int, cs: float, mach: float, reynolds: float, convective_times: float = 1.0):
    """u0 = Ma cs, nu = u0 L / Re, and the step count of `convective_times` t_c = L / u0."""
    u0 = mach * cs
    nu = u0 * L / reynolds
    steps = int(round(convective_times * L / u0))
    return u0, nu, steps


def shear_wave(nx: int, ny: int, amplitude: float, mode: int = 1) -> Fields:
    """Transverse shear wave u_x = A sin(2 pi m y / ny), u_y = 0, rho = 1 (decays as exp(-nu k^2 t))."""
    ys = np.arange(ny, dtype=np.float64)
    k = 2.0 * np.pi * mode / ny
    ux = np.repeat((amplitude * np.sin(k * ys))[:, None], nx, axis=1)
    grad = np.zeros((4, ny, nx))
    grad[1] = np.repeat((amplitude * k * np.cos(k * ys))[:, None], nx, axis=1)
    return Fields(np.ones((ny, nx)), ux, np.zeros((ny, nx)), None, grad)


def taylor_green_3d_box(nx: int, ny: int, nz: int, u0: float):
    """The Taylor-Green vortex of taylor_green_3d on an nx x ny x nz periodic box (wavenumber 2 pi / n per
    axis), u_y scaled by kx / ky so that the field stays divergence-free; same layout of the returned arrays
    (equal to taylor_green_3d on a cube)."""
    kx, ky, kz = 2.0 * np.pi / nx, 2.0 * np.pi / ny, 2.0 * np.pi / nz
    X = np.arange(nx, dtype=np.float64)[None, None, :] * kx
    Y = np.arange(ny, dtype=np.float64)[None, :, None] * ky
    Z = np.arange(nz, dtype=np.float64)[:, None, None] * kz
    shape = (nz, ny, nx)
    sx, cx, sy, cy, sz, cz = np.sin(X), np.cos(X), np.sin(Y), np.cos(Y), np.sin(Z), np.cos(Z)
    u = np.zeros((3,) + shape)
    r = kx / ky
    u[0] = u0 * sx * cy * cz
    u[1] = -u0 * r * cx * sy * cz
    g = np.zeros((9,) + shape)
    g[0] = u0 * kx * cx * cy * cz
    g[1] = -u0 * ky * sx * sy * cz
    g[2] = -u0 * kz * sx * cy * sz
    g[3] = u0 * r * kx * sx * sy * cz
    g[4] = -u0 * r * ky * cx * cy * cz
    g[5] = u0 * r * kz * cx * sy * sz
    return np.ones(shape), u, g


def taylor_green_3d(n: int, u0: float):
    """Three-dimensional Taylor-Green vortex on a periodic n^3 box, rho = 1:
    u_x = u0 sin(kx) cos(ky) cos(kz), u_y = -u0 cos(kx) sin(ky) cos(kz), u_z = 0, k = 2 pi / n.
    Returns rho [n][n][n], u [3][n][n][n] and grad [9][n][n][n] with component 3a + b = d u_a / d x_b
    (arrays indexed [z][y][x])."""
    k = 2.0 * np.pi / n
    c = np.arange(n, dtype=np.float64) * k
    sx, cx = np.sin(c)[None, None, :], np.cos(c)[None, None, :]
    sy, cy = np.sin(c)[None, :, None], np.cos(c)[None, :, None]
    sz, cz = np.sin(c)[:, None, None], np.cos(c)[:, None, None]
    shape = (n, n, n)
    u = np.zeros((3,) + shape)
    u[0] = u0 * sx * cy * cz
    u[1] = -u0 * cx * sy * cz
    g = np.zeros((9,) + shape)
    g[0] = u0 * k * cx * cy * cz
    g[1] = -u0 * k * sx * sy * cz
    g[2] = -u0 * k * sx * cy * sz
    g[3] = u0 * k * sx * sy * cz
    g[4] = -u0 * k * cx * cy * cz
    g[5] = u0 * k * cx * sy * sz
    return np.ones(shape), u, g


def riemann_tube(nx: int, ny: int, left, right, x0: int | None = None) -> Fields:
    """Piecewise-constant states (rho, u, theta) left of x0 and right of it (x0 = nx/2 by default)."""
    x0 = nx // 2 if x0 is None else x0
    xs = np.arange(nx)
    sel = (xs < x0)[None, :].repeat(ny, axis=0)
    rho = np.where(sel, left[0], right[0]).astype(np.float64)
    ux = np.where(sel, left[1], right[1]).astype(np.float64)
    th = np.where(sel, left[2], right[2]).astype(np.float64)
    return Fields(rho, ux, np.zeros_like(rho), th, None)


def sod_states(pl=1.0, rhol=1.0, pr=0.1, rhor=0.125):
    """Left/right (rho, u, theta) with theta = (p/rho) / (p_L/rho_L): the left state sits at theta = 1."""
    t_ref = pl / rhol
    return (rhol, 0.0, (pl / rhol) / t_ref), (rhor, 0.0, (pr / rhor) / t_ref)


def random_fields(nx: int, ny: int, seed: int, u_scale: float = 0.05, rho_amp: float = 0.05,
                  theta_amp: float = 0.0) -> Fields:
    """Smooth random fields: a few random Fourier modes per component (periodic)."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny)

    def modes(amp):
        g = np.zeros((ny, nx))
        for _ in range(4):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            g += rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        return amp * g / 4.0

    rho = 1.0 + modes(rho_amp)
    ux, uy = modes(u_scale), modes(u_scale)
    th = 1.0 + modes(theta_amp) if theta_amp > 0 else None
    return Fields(rho, ux, uy, th, None)


def population_noise(V: int, nx: int, ny: int, seed: int, eps: float) -> np.ndarray:
    """Relative perturbation eta[V, ny, nx] uniform in [-eps, eps], to multiply populations by (1 + eta)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-eps, eps, size=(V, ny, nx))


@dataclass
class Instance:
    lattice: str
    L: int
    reynolds: float


def batched_sweep(n: int = 64, seed: int = 0, sizes=(128, 192, 256, 384, 512, 768, 1024),
                  re_range=(1e4, 1e6), lattices=("D2Q9", "D2V17")) -> list[Instance]:
    """Heterogeneous shear-layer instances: size uniform over `sizes`, Re log-uniform, lattices alternating."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.choice(sizes))
        re = float(math.exp(rng.uniform(math.log(re_range[0]), math.log(re_range[1]))))
        out.append(Instance(lattices[k % len(lattices)], L, re))
    return out


def perturbed_shear_layer(L: int, u0: float, seed: int, kappa_range=(60.0, 100.0), delta_range=(0.03, 0.08)) -> Fields:
    """Shear layer with a seeded perturbation amplitude delta and layer stiffness kappa."""
    rng = np.random.default_rng(seed)
    kappa = float(rng.uniform(*kappa_range))
    delta = float(rng.uniform(*delta_range))
    return double_shear_layer(L, u0, kappa=kappa, delta=delta)


CLOSURE_LAYERS = [(64, 32), (64, 64), (64, 64), (8, 64)]  # (outputs, inputs) per layer


def closure_initial_weights(seed: int, out_scale: float = 0.1) -> np.ndarray:
    """Seeded initial parameters of the closure network in its flat layout (W[out][in] then b[out] per
    layer): He-normal hidden weights, the output layer scaled by out_scale, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, (o, i) in enumerate(CLOSURE_LAYERS):
        w = rng.normal(0.0, np.sqrt(2.0 / i), size=(o, i))
        if k == len(CLOSURE_LAYERS) - 1:
            w *= out_scale
        parts += [w.ravel(), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)
