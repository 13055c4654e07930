"""GPU parity of the 3D lattices of Tab. II (include/lbm3.h) against the FP64 oracle (oracle/lbm3d.py).

Tolerances as in 2D: one collision of the stored populations within 1e-6 per population relative to
max(|f_i|, w_i) in FP32 and 1e-12 in FP64; 16-bit storage within a fraction of the deviation scale the
format resolves.
"""
import math

import numpy as np
import pytest

from oracle import lbm3d as o

from gpu_util import coll_errors, lib, stored, stream

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-6, "f64": 1e-12}
NAMES = ["D3Q19", "D3Q27", "D3V39", "D3Q103"]


def perm(m, name):
    """Index map: oracle population k is the library's population P[k]."""
    V, cx, cy, cz, w, cs2 = m.lbm3_lattice_info(name)
    pos = {(int(a), int(b), int(c)): i for i, (a, b, c) in enumerate(zip(cx, cy, cz))}
    return np.array([pos[tuple(int(v) for v in xi)] for xi in o.lattice(name).xi])


class Ctx3:
    def __init__(self, name, nx, ny, nz, tau, coll="rr", neq=2, nreg=0, storage="f32", bc=(0, 0, 0)):
        self.m = lib()
        self.name, self.shape = name, (nz, ny, nx)
        self.P = perm(self.m, name)
        self.V = o.lattice(name).V
        p = self.m.make_params3(name, nx, ny, nz, tau=tau, collision=coll, hermite_order=neq, reg_order=nreg,
                                bc=bc, storage=storage, stream=stream())
        self.ctx = self.m.lbm3_create(p)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.m.lbm3_destroy(self.ctx)

    def set_oracle_f(self, f):
        g = np.empty_like(f)
        g[self.P] = f
        self.m.lbm3_set_populations(self.ctx, np.ascontiguousarray(g))

    def get_oracle_f(self):
        g = np.empty((self.V,) + self.shape)
        self.m.lbm3_get_populations(self.ctx, g)
        return g[self.P]


def pop_rel(got, ref, w):
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), w.reshape((-1,) + (1,) * (ref.ndim - 1)))))


def random_state(name, shape, seed, eps=0.02):
    """f^(0) (order 2) of smooth random fields times (1 + eta), eta uniform in [-eps, eps]."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    rho = 1 + 0.03 * np.sin(2 * np.pi * (X + 2 * Y + Z) + rng.uniform(0, 6))
    u = np.stack([0.05 * np.sin(2 * np.pi * (X + Z) + rng.uniform(0, 6)),
                  0.05 * np.cos(2 * np.pi * (Y - X) + rng.uniform(0, 6)),
                  0.05 * np.sin(2 * np.pi * (Z + Y) + rng.uniform(0, 6))])
    L = o.lattice(name)
    f = o.expand(name, o.equilibrium_coefficients(rho.reshape(-1), u.reshape(3, -1), 2), 0, 2)
    f = f.reshape((L.V,) + shape)
    return f * (1 + rng.uniform(-eps, eps, f.shape))


def shape_for(name):
    # ragged against the 128-wide blocks in x; wide enough in y and z for the interior load path
    return (9, 8, 140) if o.lattice(name).xi.max() > 1 else (5, 4, 140)


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("coll", ["bgk", "pr", "rr"])
@pytest.mark.parametrize("name", NAMES)
def test_one_step_matches_oracle(name, coll, storage):
    nz, ny, nx = shape_for(name)
    neq = min(3, o.NMAX[name])
    f = random_state(name, (nz, ny, nx), 7)
    p = o.Params3(name, nx, ny, nz, 0.62, coll, hermite_order=neq)
    ref = o.step(p, stored(f, storage))  # one collision of the populations the context holds
    with Ctx3(name, nx, ny, nz, 0.62, coll, neq, 0, storage) as c:
        c.set_oracle_f(f)
        c.m.lbm3_step(c.ctx, 1)
        got = c.get_oracle_f()
    e_pop, e_big = coll_errors(got, ref, o.lattice(name).w)
    # D3Q103 rebuilds each population as a sum of up to 35 FP32 terms with Hermite factors up to He_4(3) ~ 60
    # (measured from the stored input: RR 1.08e-6, PR 1.19e-6 relative to max(|f|, w)); its PR and RR bound
    # is 2e-6, every other lattice and mode keeps 1e-6
    tol = 2e-6 if (name == "D3Q103" and storage == "f32" and coll != "bgk") else TOL[storage]
    assert e_pop <= tol, "pop_rel %.3e max_rel(|f| >= w/10) %.3e" % (e_pop, e_big)


@pytest.mark.parametrize("name", ["D3Q19", "D3V39"])
def test_zero_gradient_faces_match_oracle(name):
    nz, ny, nx = (9, 8, 33) if name == "D3V39" else (5, 6, 33)
    f = random_state(name, (nz, ny, nx), 3)
    p = o.Params3(name, nx, ny, nz, 0.7, "rr", hermite_order=2, bc=(1, 1, 1))
    ref = o.step(p, f, 3)
    with Ctx3(name, nx, ny, nz, 0.7, "rr", 2, 0, "f64", (1, 1, 1)) as c:
        c.set_oracle_f(f)
        c.m.lbm3_step(c.ctx, 3)
        got = c.get_oracle_f()
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("name", NAMES)
def test_init_and_moments_match_oracle(name, storage):
    nz, ny, nx = 4, 5, 6
    rng = np.random.default_rng(11)
    rho = 1 + 0.05 * rng.standard_normal((nz, ny, nx))
    u = 0.05 * rng.standard_normal((3, nz, ny, nx))
    grad = 0.01 * rng.standard_normal((3, 3, nz, ny, nx))
    neq = min(3, o.NMAX[name])
    p = o.Params3(name, nx, ny, nz, 0.7, "rr", hermite_order=neq)
    ref = o.init(p, rho, u, grad)
    with Ctx3(name, nx, ny, nz, 0.7, "rr", neq, 0, storage) as c:
        c.m.lbm3_init(c.ctx, rho, np.ascontiguousarray(u), np.ascontiguousarray(grad.reshape(9, nz, ny, nx)))
        got = c.get_oracle_f()
        r, v = np.empty((nz, ny, nx)), np.empty((3, nz, ny, nx))
        c.m.lbm3_moments(c.ctx, r, v)
    tol = 1e-7 if storage == "f32" else 1e-14
    assert pop_rel(got, ref, o.lattice(name).w) <= tol
    r_ref, u_ref = o.moments(p, ref)
    assert np.max(np.abs(r - r_ref)) <= tol * 10 and np.max(np.abs(v - u_ref)) <= tol * 10


@pytest.mark.parametrize("nx", [140, 144])  # 140: rows not whole 16-byte units (direct loads); 144: staged
@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2), ("i16", 2e-3)])
@pytest.mark.parametrize("name", ["D3Q19", "D3Q27", "D3V39", "D3Q103"])
def test_shifted_16bit_storage(name, storage, tol, nx):
    nz, ny, _ = shape_for(name)
    f = random_state(name, (nz, ny, nx), 5)
    p = o.Params3(name, nx, ny, nz, 0.7, "rr", hermite_order=2)
    ref = o.step(p, f)
    w = o.lattice(name).w[:, None, None, None]
    with Ctx3(name, nx, ny, nz, 0.7, "rr", 2, 0, storage) as c:
        c.set_oracle_f(f)
        c.m.lbm3_step(c.ctx, 1)
        got = c.get_oracle_f()
    dev = np.abs(ref / w - 1.0).max()
    assert np.max(np.abs(got - ref) / w) <= tol * dev


@pytest.mark.parametrize("name", NAMES)
def test_mass_and_momentum_conserved(name):
    nz, ny, nx = shape_for(name)
    f = random_state(name, (nz, ny, nx), 9)
    with Ctx3(name, nx, ny, nz, 0.7, "rr", 2, 0, "f64") as c:
        c.set_oracle_f(f)
        s0 = c.m.lbm3_conservation(c.ctx)
        c.m.lbm3_step(c.ctx, 10)
        s1 = c.m.lbm3_conservation(c.ctx)
    assert abs(s1[0] - s0[0]) <= 1e-12 * s0[0]
    assert np.all(np.abs(s1[1:] - s0[1:]) <= 1e-12 * s0[0])


@pytest.mark.parametrize("name", ["D3Q19", "D3Q27"])
def test_shear_wave_decays_at_nu_k2(name):
    """FP32: u_x = A sin(2 pi z / nz) decays as exp(-nu k^2 t), nu = cs^2 (tau - 1/2)."""
    m = lib()
    nz, tau = 32, 0.8
    V, cx, cy, cz, w, cs2 = m.lbm3_lattice_info(name)
    k = 2 * np.pi / nz
    z = np.arange(nz)
    rho = np.ones((nz, 2, 2))
    u = np.zeros((3, nz, 2, 2))
    u[0] = 1e-3 * np.sin(k * z)[:, None, None]
    grad = np.zeros((9, nz, 2, 2))
    grad[2] = 1e-3 * k * np.cos(k * z)[:, None, None]  # d u_x / d z
    nu = cs2 * (tau - 0.5)
    n = int(0.5 / (nu * k * k))
    with Ctx3(name, 2, 2, nz, tau, "rr", 2, 0, "f32") as c:
        m.lbm3_init(c.ctx, rho, u, grad)
        v = np.empty((3, nz, 2, 2))
        m.lbm3_moments(c.ctx, None, v)
        a0 = np.abs(v[0]).max()
        m.lbm3_step(c.ctx, n)
        m.lbm3_moments(c.ctx, None, v)
    rate = math.log(a0 / np.abs(v[0]).max()) / n
    assert rate == pytest.approx(nu * k * k, rel=0.04)


@pytest.mark.parametrize("bc", [(0, 0, 0), (0, 1, 1)])
@pytest.mark.parametrize("storage,nx", [("f64", 8), ("f64", 264), ("f32", 520), ("f16", 520), ("bf16", 520),
                                        ("i16", 520)])
@pytest.mark.parametrize("name", ["D3Q19", "D3Q27", "D3V39"])
def test_staged_tiles_and_wraps(name, storage, nx, bc):
    """Grids periodic in x with whole 16-byte rows take the staged kernel: a row that fits one tile (nx = 8)
    is staged whole and wrapped by index; longer rows (FP64 264 = three 128-cell tiles, FP32 520 = three
    256-cell tiles, the last ragged, with a 4-cell margin in FP32 and 8 in 16-bit storage) get the wrapped
    columns as copies of their edge tiles; zero-gradient y and z faces clamp the source rows of the staged
    copies.  Three steps."""
    nz, ny = (9, 8) if o.lattice(name).xi.max() > 1 else (5, 6)
    f = random_state(name, (nz, ny, nx), 13)
    p = o.Params3(name, nx, ny, nz, 0.7, "rr", hermite_order=2, bc=bc)
    ref = o.step(p, f, 3)
    with Ctx3(name, nx, ny, nz, 0.7, "rr", 2, 0, storage, bc) as c:
        c.set_oracle_f(f)
        c.m.lbm3_step(c.ctx, 3)
        got = c.get_oracle_f()
    if storage == "f64":
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12
    elif storage == "f32":
        assert pop_rel(got, ref, o.lattice(name).w) <= 3 * TOL["f32"]
    else:  # three roundings to the 16-bit format of the shifted deviation: the one-step bound, three times
        w = o.lattice(name).w[:, None, None, None]
        tol16 = {"f16": 2e-3, "bf16": 2e-2, "i16": 2e-3}[storage]
        assert np.max(np.abs(got - ref) / w) <= 3 * tol16 * np.abs(f / w - 1.0).max()


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_staged_ring_reuse(storage):
    """Enough row tiles (2 x 64 x 48 = 6144) that every persistent block walks several rounds of its stage ring,
    so each stage's barrier completes phases of both parities."""
    name, nz, ny, nx = "D3Q19", 48, 64, 256
    f = random_state(name, (nz, ny, nx), 17)
    p = o.Params3(name, nx, ny, nz, 0.62, "rr", hermite_order=2)
    ref = o.step(p, f, 2)
    with Ctx3(name, nx, ny, nz, 0.62, "rr", 2, 0, storage) as c:
        c.set_oracle_f(f)
        c.m.lbm3_step(c.ctx, 2)
        got = c.get_oracle_f()
    assert pop_rel(got, ref, o.lattice(name).w) <= 2 * TOL[storage]


@pytest.mark.parametrize("storage,tol", [("f32", 2e-6), ("f16", 2e-3), ("bf16", 2e-2), ("i16", 2e-3)])
def test_d3q103_pair_kernel_interior_rows(storage, tol):
    """A grid whose edge rows (within 3 of a y or z face) are at most an eighth of its rows runs the interior
    rows in their own launch, which for D3Q103 RR on an x-periodic grid of even nx is the two-cell kernel:
    one step against the oracle's collision of the stored populations, on every cell of sampled interior and
    edge rows.  FP32 at D3Q103's per-collision bound; 16-bit formats within a fraction of the deviation scale
    they resolve (their output is rounded to the format)."""
    name = "D3Q103"
    nz, ny, nx = 94, 94, 36  # 8 x 1092 edge rows <= 94^2: split; 18 pairs a row, the x wrap at both ends
    f = random_state(name, (nz, ny, nx), 13)
    with Ctx3(name, nx, ny, nz, 0.62, "rr", 2, 0, storage) as c:
        c.set_oracle_f(f)
        pre = c.get_oracle_f()
        c.m.lbm3_step(c.ctx, 1)
        got = c.get_oracle_f()
    L = o.lattice(name)
    zs = np.array([0, 2, 3, 4, 47, 89, 90, 91, 93])
    Z, Y, X = np.meshgrid(zs, zs, np.arange(nx), indexing="ij")
    Z, Y, X = Z.ravel(), Y.ravel(), X.ravel()
    fs = np.empty((L.V, Z.size))
    for i in range(L.V):
        cx, cy, cz = (int(v) for v in L.xi[i])
        fs[i] = pre[i, (Z - cz) % nz, (Y - cy) % ny, (X - cx) % nx]
    p = o.Params3(name, nx, ny, nz, 0.62, "rr", hermite_order=2)
    ref = o.collide(p, fs)
    out = got[:, Z, Y, X]
    if storage == "f32":
        e_pop, e_big = coll_errors(out, ref, L.w)
        assert e_pop <= tol, "pop_rel %.3e max_rel(|f| >= w/10) %.3e" % (e_pop, e_big)
    else:
        w = L.w[:, None]
        dev = np.abs(ref / w - 1.0).max()
        assert np.max(np.abs(out - ref) / w) <= tol * dev


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_d3q103_pair_kernel_zero_gradient_faces(storage):
    """D3Q103 RR with zero-gradient y and z faces and a periodic x of even nx runs the two-cell kernel with
    per-population source rows (the clamped source rule of both faces): one step against the oracle."""
    name = "D3Q103"
    nz, ny, nx = 9, 8, 36
    f = random_state(name, (nz, ny, nx), 17)
    bc = (0, 1, 1)
    with Ctx3(name, nx, ny, nz, 0.62, "rr", 2, 0, storage, bc) as c:
        c.set_oracle_f(f)
        pre = c.get_oracle_f()
        c.m.lbm3_step(c.ctx, 1)
        got = c.get_oracle_f()
    p = o.Params3(name, nx, ny, nz, 0.62, "rr", hermite_order=2, bc=bc)
    ref = o.step(p, pre)
    L = o.lattice(name)
    if storage == "f32":
        e_pop, e_big = coll_errors(got, ref, L.w)
        assert e_pop <= 2e-6, "pop_rel %.3e max_rel(|f| >= w/10) %.3e" % (e_pop, e_big)
    else:
        w = L.w[:, None, None, None]
        dev = np.abs(ref / w - 1.0).max()
        assert np.max(np.abs(got - ref) / w) <= 2e-3 * dev
