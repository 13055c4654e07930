"""Learned closure (lbm_closure_*): tensor-core forward and backward against the FP64 reference network,
training, the feature / box-filter kernels against their definitions, and the closure step against the
plain RR step."""
import numpy as np
import pytest

from oracle import mlp
from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl

import closure_bounds as cb
from gpu_util import Ctx, assert_coll, lib, pop_rel, stored

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
    """Every output of the tensor-core forward within the rounding bound of its BF16 activations
    (probabilistic, lam = 6) plus the worst case of the hardware tanh and FP32 accumulation, against the
    FP64 network on the same BF16 weight matrices, FP32 biases and BF16 inputs; and within the
    worst-case first-order bound."""
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
    ref, bound = cb.forward_bound_probabilistic(w, x)
    _, worst = cb.forward_bound(w, x)
    err = np.abs(got - ref)
    assert np.all(err <= 1.25 * bound), "max err / bound %.3f" % np.max(err / bound)
    assert np.all(err <= 1.25 * worst)


def test_gradients_match_reference():
    """Loss and every gradient entry of the tensor-core backward against the FP64 reference on the same
    parameters, within 8 standard deviations of the error the kernels' BF16 roundings and hardware tanh
    put on that entry (estimated by 64 draws of a random-rounding model of the same computation), plus a
    floor of 1e-6 of the largest entry for entries with no rounding in their path."""
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
    ref_loss, ref_g, _ = cb.gradient_bound(w, x, y)
    s_loss, s_g = cb.gradient_spread(w, x, y)
    assert abs(loss - ref_loss) <= 8 * s_loss + 1e-6 * ref_loss, (loss, ref_loss, s_loss)
    err = np.abs(g.astype(np.float64) - ref_g)
    tol = 8 * s_g + 1e-6 * np.abs(ref_g).max()
    assert np.all(err <= tol), "max err / tol %.3f at %d" % (np.max(err / tol), int(np.argmax(err / tol)))


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


def closure_state(nx, ny, seed, neq=4):
    name = "D2Q9"
    Lt = orc.lattice(name)
    fl = wl.random_fields(nx, ny, seed, u_scale=0.06)
    op = orc.params(name, nx, ny, 0.7, "bgk", neq)
    return orc.init(op, fl.rho, fl.ux, fl.uy) * (1.0 + wl.population_noise(Lt.V, nx, ny, seed + 1, 0.02))


@pytest.mark.parametrize("neq,nreg", [(2, 0), (4, 0), (2, 2)])
def test_closure_apply_matches_oracle(neq, nreg):
    """lbm_closure_apply with a given correction field y (components 0..2 = (xx, xy, yy) / u0^2) against the
    oracle's RR collision with Delta a1^(2) = u0^2 y / (1 - 1/tau) added before the recursion, cell by cell
    at the FP32 per-collision bound, on a grid ragged against the tiles with a zero-gradient x edge."""
    torch, m = torch_mod(), lib()
    name, nx, ny, tau, u0 = "D2Q9", 150, 19, 0.58, 0.05
    Lt = orc.lattice(name)
    f = closure_state(nx, ny, 31, neq)
    yv = np.random.default_rng(32).normal(size=(nx * ny, mlp.NO)).astype(np.float32)
    op = orc.params(name, nx, ny, tau, "rr", neq, nreg, bc_x=1)
    ref = orc.step_delta(op, stored(f, "f32"), orc.closure_delta(yv, u0, tau, nx, ny))
    assert np.abs(ref - orc.step(op, stored(f, "f32"))).max() > 1e-4 * Lt.w.min()  # the correction matters
    with Ctx(name, nx, ny, tau, "rr", neq, nreg, "f32", bcx=1) as c:
        c.set_oracle_f(f)
        m.lbm_closure_apply(c.ctx, torch.tensor(yv).cuda(), u0)
        got = c.get_oracle_f()
    assert_coll(got, ref, Lt.w, 1e-6)


def test_closure_step_with_a_nonzero_network_matches_oracle():
    """lbm_step_closure, one step with a non-zero network: the oracle collides each cell with the
    correction the network predicts from that cell's features (the GPU's forward of the GPU's features,
    themselves checked against their definition and the reference network above); cell by cell at the
    FP32 per-collision bound."""
    torch, m = torch_mod(), lib()
    name, nx, ny, tau, u0 = "D2Q9", 96, 40, 0.6, 0.05
    Lt = orc.lattice(name)
    f = closure_state(nx, ny, 41)
    n = nx * ny
    op = orc.params(name, nx, ny, tau, "rr", 4)
    cl = m.lbm_closure_create()
    try:
        m.lbm_closure_set_weights(cl, wl.closure_initial_weights(13, out_scale=1.0))
        with Ctx(name, nx, ny, tau, "rr", 4, 0, "f32") as c:
            c.set_oracle_f(f)
            r, u, v = (torch.zeros((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3))
            x = torch.zeros((n, mlp.NI), dtype=torch.bfloat16, device="cuda")
            y = torch.zeros((n, mlp.NO), dtype=torch.float32, device="cuda")
            m.lbm_moments(c.ctx, r, u, v)
            m.lbm_closure_features(r, u, v, nx, ny, u0, x, None)
            m.lbm_closure_forward(cl, x, n, y, None)
            yv = y.cpu().numpy()
            assert np.abs(yv[:, :3]).max() > 1e-2  # the correction is active
            m.lbm_step_closure(c.ctx, cl, u0, 1)
            got = c.get_oracle_f()
    finally:
        m.lbm_closure_destroy(cl)
    ref = orc.step_delta(op, stored(f, "f32"), orc.closure_delta(yv, u0, tau, nx, ny))
    assert_coll(got, ref, Lt.w, 1e-6)
