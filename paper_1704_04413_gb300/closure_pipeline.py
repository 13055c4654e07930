"""Learned-closure workflow on top of the C ABI: training data from filtered fine RR runs, training,
and the coarse-grid comparison against plain RR.

Every computation is a library kernel (fine and coarse steps, moments, box filter, features, MLP
forward/backward, Adam); PyTorch only provides device buffers and random permutations of sample
indices.  The vorticity spectra of the comparison are measurements taken on the host.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lbm
from . import workloads as wl


@dataclass
class ClosureData:
    x: object            # [N, 32] BF16 features (CUDA tensor)
    y: object            # [N, 8] FP32 targets (CUDA tensor)
    truth: dict          # coarse-step index -> filtered (rho, ux, uy) of the first training seed (host)
    u0: float
    nu_coarse: float
    coarse: int
    factor: int
    fine_finite: list = field(default_factory=list)
    seconds: float = 0.0
    held_out: dict = field(default_factory=dict)  # seed -> truth dict of fine runs kept out of training


def _vorticity(u, v):
    def d(g, a):
        return (-np.roll(g, -2, a) + 8 * np.roll(g, -1, a) - 8 * np.roll(g, 1, a) + np.roll(g, 2, a)) / 12.0
    return d(v, 1) - d(u, 0)


def vorticity_spectrum(u, v):
    """Shell-summed |FFT(omega)|^2 for integer wavenumber shells 0 .. n/2 - 1."""
    w = _vorticity(u, v)
    n = w.shape[0]
    W = np.abs(np.fft.fft2(w)) ** 2
    k = np.fft.fftfreq(n) * n
    K = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2).astype(int)
    return np.bincount(K.ravel(), W.ravel())[: n // 2]


def spectrum_error(u, v, u_ref, v_ref):
    """RMS over shells 1 .. n/2-1 of log(E / E_ref)."""
    e, r = vorticity_spectrum(u, v)[1:], vorticity_spectrum(u_ref, v_ref)[1:]
    return float(np.sqrt(np.mean((np.log(e + 1e-30) - np.log(r + 1e-30)) ** 2)))


def generate(fine: int, factor: int, reynolds: float, seeds, convective_times: float = 1.0, snapshots: int = 16,
             mach: float = 0.1, stream=None, held_out=()) -> ClosureData:
    """Fine D2Q9 RR shear layers (seeded kappa, delta), box-filtered by `factor` every few coarse steps.
    The runs of `seeds` give the training samples; those of `held_out` give only evaluation truths."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    coarse = fine // factor
    _, _, _, _, cs2 = lbm.lbm_lattice_info("D2Q9")
    u0, nu_f, steps_tc = wl.shear_layer_params(fine, np.sqrt(cs2), mach, reynolds)
    _, nu_c, _ = wl.shear_layer_params(coarse, np.sqrt(cs2), mach, reynolds)
    total = int(round(convective_times * steps_tc)) // factor * factor
    every = max(factor, (total // snapshots) // factor * factor)
    dev = lambda n: torch.zeros((n, n), dtype=torch.float64, device="cuda")
    X, Y, truth, finite, held = [], [], {}, [], {}
    seeds = list(seeds)
    for k, seed in enumerate(seeds + list(held_out)):
        train = k < len(seeds)
        fl = wl.perturbed_shear_layer(fine, u0, seed)
        ctx = lbm.lbm_create(lbm.make_params("D2Q9", fine, fine, nu=nu_f, collision="rr", hermite_order=2,
                                             storage="f32", stream=st))
        try:
            lbm.lbm_init(ctx, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
            rho, ux, uy = dev(fine), dev(fine), dev(fine)
            for s in range(0, total + 1, every):
                if s:
                    lbm.lbm_step(ctx, every)
                lbm.lbm_moments(ctx, rho, ux, uy)
                rc, uc, vc = dev(coarse), dev(coarse), dev(coarse)
                y = torch.zeros((coarse * coarse, lbm.CLOSURE_OUT), dtype=torch.float32, device="cuda")
                lbm.lbm_closure_coarsen(rho, ux, uy, fine, fine, factor, u0, rc, uc, vc, y, st)
                x = torch.zeros((coarse * coarse, lbm.CLOSURE_IN), dtype=torch.bfloat16, device="cuda")
                lbm.lbm_closure_features(rc, uc, vc, coarse, coarse, u0, x, st)
                if train:
                    X.append(x)
                    Y.append(y)
                fields = (rc.cpu().numpy(), uc.cpu().numpy(), vc.cpu().numpy())
                if k == 0:
                    truth[s // factor] = fields
                if not train:
                    held.setdefault(seed, {})[s // factor] = fields
            finite.append(bool(torch.isfinite(rho).all().item()))
        finally:
            lbm.lbm_destroy(ctx)
    torch.cuda.synchronize()
    return ClosureData(torch.cat(X), torch.cat(Y), truth, u0, nu_c, coarse, factor, finite, time.perf_counter() - t0,
                       held)


def train(data: ClosureData, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
    """Adam on shuffled minibatches; returns (closure handle, per-epoch mean losses, seconds).
    Minibatches are gathered and trained on the current PyTorch stream."""
    import torch
    st = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    cl = lbm.lbm_closure_create()
    lbm.lbm_closure_set_weights(cl, wl.closure_initial_weights(seed))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = data.x.shape[0]
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        el = []
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            el.append(lbm.lbm_closure_train_step(cl, data.x[idx].contiguous(), data.y[idx].contiguous(), batch, lr,
                                                   st))
        losses.append(float(np.mean(el)))
    torch.cuda.synchronize()
    return cl, losses, time.perf_counter() - t0


def compare(data: ClosureData, cl, stream=None, truth=None):
    """Coarse runs from the filtered initial state: plain RR and RR with the closure, each snapshot's
    vorticity-spectrum error and vorticity relative L2 error against the filtered fine run (`truth`, default
    the first training seed's)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    n = data.coarse
    truth = truth if truth is not None else data.truth
    r0, u0f, v0f = truth[0]
    gx = lambda a: (np.roll(a, -1, 1) - np.roll(a, 1, 1)) / 2.0
    gy = lambda a: (np.roll(a, -1, 0) - np.roll(a, 1, 0)) / 2.0
    grad = np.ascontiguousarray(np.stack([gx(u0f), gy(u0f), gx(v0f), gy(v0f)]))
    out = {}
    for mode in ("plain", "closure"):
        c = lbm.lbm_create(lbm.make_params("D2Q9", n, n, nu=data.nu_coarse, collision="rr", hermite_order=2,
                                           storage="f32", stream=st))
        try:
            lbm.lbm_init(c, np.ascontiguousarray(r0), np.ascontiguousarray(u0f), np.ascontiguousarray(v0f), None, grad)
            done, rows = 0, []
            for s in sorted(truth)[1:]:
                if mode == "plain":
                    lbm.lbm_step(c, s - done)
                else:
                    lbm.lbm_step_closure(c, cl, data.u0, s - done)
                done = s
                rr, uu, vv = (np.empty((n, n)) for _ in range(3))
                lbm.lbm_moments(c, rr, uu, vv)
                _, ut, vt = truth[s]
                wt, wc = _vorticity(ut, vt), _vorticity(uu, vv)
                rows.append({"coarse_step": s, "spectrum_err": spectrum_error(uu, vv, ut, vt),
                             "vorticity_rel_l2": float(np.linalg.norm(wc - wt) / np.linalg.norm(wt))})
            out[mode] = rows
        finally:
            lbm.lbm_destroy(c)
    return out
