"""Batched sweep (lbm_batch_*): one graph-captured launch per step for many grids of both lattices.

Every instance of a batch is compared with the FP64 oracle after batched steps; the batched kernel
runs the same per-cell arithmetic as lbm_step, so its result must also be bit-identical to stepping
every instance on its own, with any launch shape the autotuner may pick.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl

from gpu_util import lib, perm, pop_rel, stored, stream

pytestmark = pytest.mark.gpu

SHAPES = [("D2Q9", 130, 70, 2e4), ("D2V17", 96, 64, 5e4), ("D2Q9", 300, 33, 1e5), ("D2V17", 257, 129, 3e4),
          ("D2Q9", 64, 64, 1e4), ("D2V17", 190, 41, 1e6)]


# with D2V37 (one cell per thread, 128-thread blocks): the three lattices of the benchmark's batched step
SHAPES37 = [("D2V37", 150, 33, 3e4), ("D2Q9", 96, 40, 1e4), ("D2V17", 130, 21, 5e4), ("D2V37", 64, 17, 1e5)]
NEQ = {"D2Q9": 2, "D2V17": 3, "D2V37": 4}


def params(m, storage, shapes=SHAPES):
    out = []
    for name, nx, ny, re in shapes:
        cs2 = orc.lattice(name).cs2
        u0, nu, _ = wl.shear_layer_params(nx, np.sqrt(cs2), 0.1, re)
        out.append(m.make_params(name, nx, ny, nu=nu, collision="rr", hermite_order=NEQ[name],
                                 storage=storage, stream=stream()))
    return out


def init_all(m, ctxs, shapes=SHAPES):
    for (name, nx, ny, re), c in zip(shapes, ctxs):
        cs2 = orc.lattice(name).cs2
        u0, _, _ = wl.shear_layer_params(nx, np.sqrt(cs2), 0.1, re)
        fl = wl.double_shear_layer(nx, u0, ny=ny)
        m.lbm_init(c, fl.rho, fl.ux, fl.uy, None, fl.grad_u)


def pops(m, c, name, nx, ny):
    V = orc.lattice(name).V
    f = np.empty((V, ny, nx))
    m.lbm_get_populations(c, f)
    return f


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batched_steps_equal_single_steps_bitwise(storage):
    m = lib()
    ps = params(m, storage)
    b = m.lbm_batch_create(ps)
    singles = [m.lbm_create(p) for p in ps]
    try:
        bc = [m.lbm_batch_context(b, i) for i in range(len(ps))]
        init_all(m, bc)
        init_all(m, singles)
        for n in (5, 2, 1):  # graph replays and a direct launch for the odd step
            m.lbm_batch_step(b, n)
            for c in singles:
                m.lbm_step(c, n)
        for (name, nx, ny, _), c0, c1 in zip(SHAPES, bc, singles):
            assert m.lbm_step_count(c0) == m.lbm_step_count(c1) == 8
            assert np.array_equal(pops(m, c0, name, nx, ny), pops(m, c1, name, nx, ny))
    finally:
        m.lbm_batch_destroy(b)
        for c in singles:
            m.lbm_destroy(c)


def test_autotuned_launch_keeps_results():
    m = lib()
    ps = params(m, "f16")
    b = m.lbm_batch_create(ps)
    singles = [m.lbm_create(p) for p in ps]
    try:
        ms = m.lbm_batch_autotune(b, 2)
        t, r, q = m.lbm_batch_get_launch(b)
        assert ms > 0 and t in (64, 128, 256) and r in (1, 2, 4, 8) and q in (0, 2, 4, 8)
        bc = [m.lbm_batch_context(b, i) for i in range(len(ps))]
        init_all(m, bc)
        init_all(m, singles)
        m.lbm_batch_step(b, 6)
        for c in singles:
            m.lbm_step(c, 6)
        for (name, nx, ny, _), c0, c1 in zip(SHAPES, bc, singles):
            assert np.array_equal(pops(m, c0, name, nx, ny), pops(m, c1, name, nx, ny))
    finally:
        m.lbm_batch_destroy(b)
        for c in singles:
            m.lbm_destroy(c)


def test_out_of_phase_instance_is_refused():
    m = lib()
    ps = params(m, "f32")[:2]
    b = m.lbm_batch_create(ps)
    try:
        c0 = m.lbm_batch_context(b, 0)
        m.lbm_step(c0, 1)
        with pytest.raises(m.LbmError) as e:
            m.lbm_batch_step(b, 2)
        assert e.value.code == m.EINVAL
    finally:
        m.lbm_batch_destroy(b)


@pytest.mark.parametrize("blocks_per_sm", [0, 2])
@pytest.mark.parametrize("storage,tol", [("f32", None), ("f16", 2e-3), ("bf16", 2e-2)])
def test_batched_steps_match_oracle(storage, tol, blocks_per_sm):
    """Every cell of every instance (D2Q9 and D2V17 mixed, ragged sizes, different Re) after three batched
    steps (a graph replay of two and a direct launch) against three oracle steps from the same
    initial populations: FP32 within 1e-6 per collision (pop_rel, three collisions), 16-bit storage
    relative to the deviation scale the format resolves; one block per item and a persistent grid."""
    m = lib()
    ps = params(m, storage)
    b = m.lbm_batch_create(ps)
    try:
        m.lbm_batch_set_launch(b, 128, 2, blocks_per_sm)
        refs, steps = [], 3
        for (name, nx, ny, re), i in zip(SHAPES, range(len(ps))):
            c = m.lbm_batch_context(b, i)
            Lt = orc.lattice(name)
            cs2 = Lt.cs2
            u0, _, _ = wl.shear_layer_params(nx, np.sqrt(cs2), 0.1, re)
            fl = wl.double_shear_layer(nx, u0, ny=ny)
            neq = {"D2Q9": 2, "D2V17": 3}[name]
            op = orc.params(name, nx, ny, m.lbm_tau(c), "rr", neq)
            f = orc.init(op, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
            f = f * (1.0 + wl.population_noise(Lt.V, nx, ny, 100 + i, 0.01))
            m.lbm_set_populations(c, np.ascontiguousarray(f[perm(name)]))
            refs.append((f, orc.step(op, stored(f, storage), steps)))
        m.lbm_batch_step(b, steps)
        for (name, nx, ny, _), i, (f0, ref) in zip(SHAPES, range(len(ps)), refs):
            Lt = orc.lattice(name)
            got = np.empty_like(ref)
            got[perm(name)] = pops(m, m.lbm_batch_context(b, i), name, nx, ny)
            if storage == "f32":
                assert pop_rel(got, ref, Lt.w) <= steps * 1e-6, (name, nx, ny)
            else:
                w = Lt.w[:, None, None]
                assert np.max(np.abs(got - ref) / w) <= steps * tol * np.abs(f0 / w - 1.0).max(), (name, nx, ny)
    finally:
        m.lbm_batch_destroy(b)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_with_d2v37_equals_single_steps_and_oracle(storage):
    """D2V37 instances (one cell per thread) batched with D2Q9 and D2V17 ones: bitwise equal to per-instance
    steps after 5 steps (graph replays and a direct launch), and every instance against three oracle
    steps from the same populations."""
    m = lib()
    ps = params(m, storage, SHAPES37)
    b = m.lbm_batch_create(ps)
    singles = [m.lbm_create(p) for p in ps]
    try:
        with pytest.raises(m.LbmError):
            m.lbm_batch_set_launch(b, 256, 1, 0)  # a batch holding D2V37 runs 128-thread blocks
        m.lbm_batch_set_launch(b, 128, 3, 0)
        bc = [m.lbm_batch_context(b, i) for i in range(len(ps))]
        init_all(m, bc, SHAPES37)
        init_all(m, singles, SHAPES37)
        m.lbm_batch_step(b, 5)
        for c in singles:
            m.lbm_step(c, 5)
        for (name, nx, ny, _), c0, c1 in zip(SHAPES37, bc, singles):
            assert np.array_equal(pops(m, c0, name, nx, ny), pops(m, c1, name, nx, ny)), name
        refs = []
        for (name, nx, ny, re), i in zip(SHAPES37, range(len(ps))):
            Lt = orc.lattice(name)
            op = orc.params(name, nx, ny, m.lbm_tau(bc[i]), "rr", NEQ[name])
            fl = wl.random_fields(nx, ny, 200 + i, u_scale=0.06)
            f = orc.init(op, fl.rho, fl.ux, fl.uy) * (1.0 + wl.population_noise(Lt.V, nx, ny, 300 + i, 0.01))
            m.lbm_set_populations(bc[i], np.ascontiguousarray(f[perm(name)]))
            refs.append((f, orc.step(op, stored(f, storage), 3)))
        m.lbm_batch_step(b, 3)
        for (name, nx, ny, _), c, (f0, ref) in zip(SHAPES37, bc, refs):
            Lt = orc.lattice(name)
            got = np.empty_like(ref)
            got[perm(name)] = pops(m, c, name, nx, ny)
            if storage == "f32":
                assert pop_rel(got, ref, Lt.w) <= 3e-6, name
            else:
                w = Lt.w[:, None, None]
                assert np.max(np.abs(got - ref) / w) <= 3 * 2e-3 * np.abs(f0 / w - 1.0).max(), name
    finally:
        m.lbm_batch_destroy(b)
        for c in singles:
            m.lbm_destroy(c)
