"""Learned closure (lbm_closure_*): tensor-core forward and backward against the FP64 reference network,
training, the feature / box-filter kernels against their definitions, and the closure step against the
plain RR step."""
import numpy as np
import pytest

from oracle import mlp
from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl

from gpu_util import Ctx, lib, pop_rel

pytestmark = pytest.mark.gpu


def torch_mod():
    import torch
    torch.cuda.set_device(0)
    return torch


def as_bf16_tensor(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).cuda().contiguous()


def sample(n, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, mlp.NI))
    x[:, :27] = rng.normal(size=(n, 27))
    y = np.zeros((n, mlp.NO))
    y[:, :3] = rng.normal(size=(n, 3)) * 0.3
    return x, y


def test_forward_matches_reference():
    torch, m = torch_mod(), lib()
    w = wl.closure_initial_weights(3, out_scale=1.0)
    x, _ = sample(1000, 4)
    cl = m.lbm_closure_create()
    try:
        m.lbm_closure_set_weights(cl, w)
        xt = as_bf16_tensor(torch, x)
        y = torch.zeros((1000, mlp.NO), dtype=torch.float32, device="cuda")
        m.lbm_closure_forward(cl, xt, 1000, y)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.float64)
    finally:
        m.lbm_closure_destroy(cl)
    ref, _ = mlp.forward(mlp.bf16_round(w), mlp.bf16_round(x))
    # BF16 activations between layers: a few parts in 1e3 of the output scale
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-2


def test_gradients_match_reference():
    torch, m = torch_mod(), lib()
    w = wl.closure_initial_weights(5, out_scale=1.0)
    x, y = sample(256, 6)
    cl = m.lbm_closure_create()
    try:
        m.lbm_closure_set_weights(cl, w)
        g, loss = m.lbm_closure_gradients(cl, as_bf16_tensor(torch, x), torch.tensor(y, dtype=torch.float32).cuda(),
                                          256)
    finally:
        m.lbm_closure_destroy(cl)
    ref_loss, ref_g = mlp.loss_and_grad(mlp.bf16_round(w), mlp.bf16_round(x), y)
    assert abs(loss - ref_loss) / ref_loss < 2e-2
    gp, rp = mlp.unpack(g.astype(np.float64)), mlp.unpack(ref_g)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        assert np.linalg.norm(gp[name] - rp[name]) / np.linalg.norm(rp[name]) < 5e-2, name


def test_training_reduces_loss_on_a_teacher_network():
    torch, m = torch_mod(), lib()
    n = 8192
    x, _ = sample(n, 7)
    teacher = wl.closure_initial_weights(8, out_scale=1.0)
    y, _ = mlp.forward(mlp.bf16_round(teacher), mlp.bf16_round(x))
    y[:, 3:] = 0.0
    cl = m.lbm_closure_create()
    try:
        m.lbm_closure_set_weights(cl, wl.closure_initial_weights(9))
        xt, yt = as_bf16_tensor(torch, x), torch.tensor(y, dtype=torch.float32).cuda()
        first = m.lbm_closure_train_step(cl, xt, yt, n, 1e-3)
        for _ in range(600):
            last = m.lbm_closure_train_step(cl, xt, yt, n, 1e-3)
    finally:
        m.lbm_closure_destroy(cl)
    assert last < 0.2 * first


def test_features_and_coarsening_match_definitions():
    torch, m = torch_mod(), lib()
    nx, ny, r, u0 = 48, 32, 8, 0.05
    fl = wl.random_fields(nx, ny, 11, u_scale=0.05)
    t = lambda a: torch.tensor(a, dtype=torch.float64).cuda()
    rho, ux, uy = t(fl.rho), t(fl.ux), t(fl.uy)
    cx, cy = nx // r, ny // r
    rc, uxc, uyc = (torch.zeros((cy, cx), dtype=torch.float64, device="cuda") for _ in range(3))
    y = torch.zeros((cx * cy, mlp.NO), dtype=torch.float32, device="cuda")
    m.lbm_closure_coarsen(rho, ux, uy, nx, ny, r, u0, rc, uxc, uyc, y)
    feat = torch.zeros((nx * ny, mlp.NI), dtype=torch.bfloat16, device="cuda")
    m.lbm_closure_features(rho, ux, uy, nx, ny, u0, feat)
    torch.cuda.synchronize()
    box = lambda a: a.reshape(cy, r, cx, r).mean(axis=(1, 3))
    mb = box(fl.rho)
    ub, vb = box(fl.rho * fl.ux) / mb, box(fl.rho * fl.uy) / mb
    assert np.allclose(rc.cpu().numpy(), mb, rtol=1e-13) and np.allclose(uxc.cpu().numpy(), ub, rtol=1e-12)
    tau = np.stack([box(fl.rho * fl.ux * fl.ux) - mb * ub * ub, box(fl.rho * fl.ux * fl.uy) - mb * ub * vb,
                    box(fl.rho * fl.uy * fl.uy) - mb * vb * vb], -1).reshape(-1, 3) / u0 ** 2
    assert np.allclose(y.cpu().numpy()[:, :3], tau, rtol=1e-5, atol=1e-7)
    f = feat.float().cpu().numpy()
    ref = np.zeros((ny, nx, 27))
    k = 0
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            sh = lambda a: np.roll(np.roll(a, -dy, 0), -dx, 1)
            ref[..., k] = (sh(fl.rho) - 1) / u0
            ref[..., k + 1] = sh(fl.ux) / u0
            ref[..., k + 2] = sh(fl.uy) / u0
            k += 3
    assert np.allclose(f[:, :27], mlp.bf16_round(ref.reshape(-1, 27)), rtol=0, atol=0)
    assert np.all(f[:, 27:] == 0)


def test_closure_step_with_zero_network_is_the_rr_step():
    """With all parameters zero the closure adds nothing: the step is the plain RR step (oracle parity)."""
    torch, m = torch_mod(), lib()
    name, nx, ny, tau = "D2Q9", 96, 40, 0.6
    Lt = orc.lattice(name)
    fl = wl.random_fields(nx, ny, 12, u_scale=0.06)
    op = orc.params(name, nx, ny, tau, "rr", 2)
    f = orc.init(op, fl.rho, fl.ux, fl.uy) * (1.0 + wl.population_noise(Lt.V, nx, ny, 13, 0.02))
    ref = orc.step(op, f, 3)
    cl = m.lbm_closure_create()
    try:
        with Ctx(name, nx, ny, tau, "rr", 2, 0, "f32") as c:
            c.set_oracle_f(f)
            m.lbm_step_closure(c.ctx, cl, 0.05, 3)
            got = c.get_oracle_f()
    finally:
        m.lbm_closure_destroy(cl)
    assert pop_rel(got, ref, Lt.w) <= 3e-6


def test_trained_closure_beats_plain_rr_on_the_coarse_grid():
    """Train on box-filtered (x8) 512^2 RR shear layers (Re 3e4, 4 seeds of kappa and delta), then run the
    64^2 coarse grid from the filtered initial state with and without the closure: the closure lowers the
    vorticity-spectrum error against the filtered fine run, averaged over the snapshots."""
    torch_mod()
    from paper_1704_04413_gb300 import closure_pipeline as cp
    data = cp.generate(512, 8, 3e4, seeds=range(4), convective_times=1.0)
    assert all(data.fine_finite)
    cl, losses, _ = cp.train(data, epochs=20)
    try:
        var = float(data.y[:, :3].var(dim=0).sum().item())
        assert losses[-1] < 0.1 * var  # explains most of the filtered subgrid stress
        res = cp.compare(data, cl)
    finally:
        lib().lbm_closure_destroy(cl)
    plain = np.mean([r["spectrum_err"] for r in res["plain"]])
    closure = np.mean([r["spectrum_err"] for r in res["closure"]])
    assert closure < plain


@pytest.mark.parametrize("bc_x", ["periodic", "zero_gradient"])
def test_fused_closure_step_equals_the_composed_stages(bc_x):
    """lbm_step_closure (moments, then features + network + collision fused per 32 x 4 tile) against
    lbm_moments + lbm_closure_features + lbm_closure_forward + lbm_closure_apply, bit for bit, on a grid
    that is ragged in both directions, over three steps with a network whose corrections are not small."""
    torch, m = torch_mod(), lib()
    nx, ny, u0 = 80, 50, 0.05
    fl = wl.random_fields(nx, ny, seed=21, u_scale=0.04)
    bc = m.PERIODIC if bc_x == "periodic" else m.ZERO_GRADIENT
    ps = m.make_params("D2Q9", nx, ny, tau=0.6, collision="rr", hermite_order=2, storage="f32", bc_x=bc)
    c1, c2 = m.lbm_create(ps), m.lbm_create(ps)
    cl = m.lbm_closure_create()
    try:
        m.lbm_closure_set_weights(cl, wl.closure_initial_weights(13, out_scale=1.0))
        for c in (c1, c2):
            m.lbm_init(c, fl.rho, fl.ux, fl.uy)
        n = nx * ny
        r, u, v = (torch.zeros((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3))
        x = torch.zeros((n, mlp.NI), dtype=torch.bfloat16, device="cuda")
        y = torch.zeros((n, mlp.NO), dtype=torch.float32, device="cuda")
        for _ in range(3):
            m.lbm_step_closure(c1, cl, u0, 1)
            m.lbm_moments(c2, r, u, v)
            m.lbm_closure_features(r, u, v, nx, ny, u0, x, None)
            m.lbm_closure_forward(cl, x, n, y, None)
            assert float(y[:, :3].abs().max()) > 1e-2  # the correction is active
            m.lbm_closure_apply(c2, y, u0)
        f1, f2 = np.empty((9, ny, nx)), np.empty((9, ny, nx))
        m.lbm_get_populations(c1, f1)
        m.lbm_get_populations(c2, f2)
        assert np.array_equal(f1, f2)
    finally:
        m.lbm_closure_destroy(cl)
        m.lbm_destroy(c1)
        m.lbm_destroy(c2)
