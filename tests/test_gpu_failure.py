"""Failure path of the staged step kernels, exercised without a GPU fault.

The staged kernels copy population rows into shared memory asynchronously and wait for the copies
with a time limit.  The testing hook (lbm_test_inject_copy_fault / lbm3_test_inject_copy_fault) makes
one thread block's producer announce its last tile's copies without issuing them and shortens the
limit to a few milliseconds, so that block's compute warps give up: the kernel returns, the context
reports LBM_ETIMEOUT on the host, and the device stays usable (a fresh context steps correctly).  No
copy is in flight when the block ends and every wait is bounded, so nothing faults or hangs."""
import numpy as np
import pytest

from oracle import lbm3d as o3
from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl

from gpu_util import Ctx, lib, stream

pytestmark = pytest.mark.gpu


def shear_state(name, nx, ny):
    Lt = orc.lattice(name)
    u0, nu, _ = wl.shear_layer_params(nx, np.sqrt(Lt.cs2), 0.1, 3e4)
    fl = wl.double_shear_layer(nx, u0, ny=ny)
    tau = orc.tau_from_nu(Lt.cs2, nu)
    op = orc.params(name, nx, ny, tau, "rr", Lt.nmax)
    return Lt, tau, op, orc.init(op, fl.rho, fl.ux, fl.uy, None, fl.grad_u)


@pytest.mark.parametrize("name,storage", [("D2Q9", "f16"), ("D2V17", "bf16")])
def test_staged_2d_copy_wait_timeout_is_reported(name, storage):
    import torch
    m = lib()
    nx, ny = 1024, 32  # x-periodic rows of whole 16-byte units: the staged pair kernel
    Lt, tau, op, f = shear_state(name, nx, ny)
    with Ctx(name, nx, ny, tau, "rr", Lt.nmax, 0, storage) as c:
        c.set_oracle_f(f)
        m.lbm_test_inject_copy_fault(c.ctx, 0, 0.002)
        c.step(1)
        torch.cuda.synchronize()  # the kernel returned
        with pytest.raises(m.LbmError) as e:
            m.lbm_conservation(c.ctx)
        assert e.value.code == m.ETIMEOUT
        with pytest.raises(m.LbmError) as e:
            m.lbm_diagnostics(c.ctx)
        assert e.value.code == m.ETIMEOUT
    # the device is still usable: a fresh context steps and matches the oracle
    with Ctx(name, nx, ny, tau, "rr", Lt.nmax, 0, storage) as c:
        c.set_oracle_f(f)
        c.step(1)
        got = c.get_oracle_f()
        m.lbm_conservation(c.ctx)
    ref = orc.step(op, f)
    w = Lt.w[:, None, None]
    tol = 2e-3 if storage == "f16" else 2e-2
    assert np.max(np.abs(got - ref) / w) <= tol * np.abs(f / w - 1.0).max()


def test_staged_2d_short_limit_without_fault_completes():
    """The hook off (block -1) with a shortened limit of 0.5 s: every wait completes, no status."""
    m = lib()
    name, nx, ny = "D2Q9", 1024, 32
    Lt, tau, op, f = shear_state(name, nx, ny)
    with Ctx(name, nx, ny, tau, "rr", Lt.nmax, 0, "f16") as c:
        c.set_oracle_f(f)
        m.lbm_test_inject_copy_fault(c.ctx, -1, 0.5)
        c.step(3)
        m.lbm_conservation(c.ctx)


def test_fault_hook_rejects_bad_arguments():
    m = lib()
    with Ctx("D2Q9", 64, 8, 0.6, "rr", 2, 0, "f16") as c:
        for block, wait in ((-2, 0.1), (0, 0.0), (0, 11.0), (0, -1.0)):
            with pytest.raises(m.LbmError) as e:
                m.lbm_test_inject_copy_fault(c.ctx, block, wait)
            assert e.value.code == m.EINVAL


def test_staged_3d_copy_wait_timeout_is_reported():
    import torch
    m = lib()
    name, nx, ny, nz, tau = "D3Q19", 64, 8, 8, 0.6
    V, cx, cy, cz, w, cs2 = m.lbm3_lattice_info(name)
    rho, u, grad = wl.taylor_green_3d_box(nx, ny, nz, 0.1 * np.sqrt(cs2))
    op = o3.Params3(name, nx, ny, nz, tau, "rr", hermite_order=2)
    p = m.make_params3(name, nx, ny, nz, tau=tau, collision="rr", hermite_order=2, storage="f32", stream=stream())
    c = m.lbm3_create(p)
    try:
        m.lbm3_init(c, rho, u, grad)
        m.lbm3_test_inject_copy_fault(c, 0, 0.002)
        m.lbm3_step(c, 1)
        torch.cuda.synchronize()
        with pytest.raises(m.LbmError) as e:
            m.lbm3_conservation(c)
        assert e.value.code == m.ETIMEOUT
    finally:
        m.lbm3_destroy(c)
    c = m.lbm3_create(p)
    try:
        m.lbm3_init(c, rho, u, grad)
        m.lbm3_step(c, 2)
        r3, u3 = np.empty((nz, ny, nx)), np.empty((3, nz, ny, nx))
        m.lbm3_moments(c, r3, u3)
        m.lbm3_conservation(c)
    finally:
        m.lbm3_destroy(c)
    r_o, u_o = o3.moments(op, o3.step(op, o3.init(op, rho, u, grad), 2))
    assert np.linalg.norm(u3 - u_o) / np.linalg.norm(u_o) <= 1e-5
    assert np.linalg.norm(r3 - r_o) / np.linalg.norm(r_o) <= 1e-6
