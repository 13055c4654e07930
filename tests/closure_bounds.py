"""Element-wise error bounds of the closure network's tensor-core kernels (test helper).

The kernels run the network of oracle/mlp.py with BF16 weight matrices, FP32 biases, BF16 inputs and
activations, FP32 accumulation and the hardware tanh in GELU.  Their result differs from the FP64
reference evaluated on the same BF16 weights and inputs by the rounding the kernels add on the way.
These functions bound that difference per output / per gradient entry, to first order, by carrying an
absolute error bound alongside every intermediate of the FP64 reference:
  * a BF16 rounding of a value v adds at most U |v|, U = 2^-8 (8-bit significand, round to nearest);
  * an FP32 dot product of K terms adds at most K 2^-24 sum |terms| (taken as 2^-16 sum |terms|, K <= 64 and
    any accumulation order of the tensor cores or the atomics);
  * the hardware tanh has a relative error below 2^-10.99 (PTX ISA), taken as 2^-10 absolute on |tanh| <= 1,
    which moves GELU(z) = z (1 + tanh) / 2 by at most |z| 2^-11 and GELU'(z) by (1/2 + |z| k (1 + 3 c z^2)) 2^-10;
  * an error dz of a pre-activation moves GELU by at most (|GELU'(z)| + G2 dz) dz, G2 = max |GELU''|, and
    GELU' by G2 dz.
Second-order terms (products of two bounds) are dropped; the tests compare against the bound times 1.25.

forward_bound_probabilistic gives the tighter bound of probabilistic rounding-error analysis (Higham &
Mary, SIAM J. Sci. Comput. 41, 2019): to first order the output error is sum_k J_k e_k over the rounding
events k (J_k its derivative with respect to the rounded value), and if the rounding errors e_k are
independent, mean zero and bounded by a_k, Hoeffding's inequality gives
|sum_k J_k e_k| <= lam sqrt(sum_k J_k^2 a_k^2) with probability at least 1 - 2 exp(-lam^2 / 2).  The tanh
errors are not random and enter with their worst case sum |J| a.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

U = 2.0 ** -8
ACC = 2.0 ** -16
TANH = 2.0 ** -10
_K, _C = np.sqrt(2.0 / np.pi), 0.044715


def _gelu2_max():
    z = np.linspace(-12, 12, 200001)
    t = np.tanh(_K * (z + _C * z ** 3))
    dt = (1 - t * t) * _K * (1 + 3 * _C * z * z)
    # d/dz of gelu'(z) = 0.5 (1 + t) + 0.5 z dt
    d2t = -2 * t * dt * _K * (1 + 3 * _C * z * z) + (1 - t * t) * _K * 6 * _C * z
    return float(np.max(np.abs(0.5 * dt + 0.5 * dt + 0.5 * z * d2t)))


G2 = _gelu2_max()


def reference_params(w):
    """The parameters the kernels use: weight matrices rounded to BF16, biases in FP32."""
    p = mlp.unpack(np.asarray(w, dtype=np.float32).astype(np.float64))
    for k in ("W1", "W2", "W3", "W4"):
        p[k] = mlp.bf16_round(p[k])
    return p


def _forward(p, x):
    h, dh = mlp.bf16_round(x), np.zeros_like(np.asarray(x, dtype=np.float64))
    layers = []
    for l in (1, 2, 3):
        W, b = p["W%d" % l], p["b%d" % l]
        z = h @ W.T + b
        dz = dh @ np.abs(W).T + ACC * (np.abs(h) @ np.abs(W).T + np.abs(b))
        g = mlp.gelu(z)
        dg = (np.abs(mlp.gelu_grad(z)) + G2 * dz) * dz + np.abs(z) * TANH / 2
        layers.append((h, dh, z, dz))
        h, dh = g, dg + U * (np.abs(g) + dg)
    W, b = p["W4"], p["b4"]
    out = h @ W.T + b
    dout = dh @ np.abs(W).T + ACC * (np.abs(h) @ np.abs(W).T + np.abs(b))
    return out, dout, layers, (h, dh)


def forward_bound(w, x):
    """(reference output, bound on |kernel output - reference output|), both [n][OUT]."""
    out, dout, _, _ = _forward(reference_params(w), x)
    return out, dout


def gradient_bound(w, x, y, n_used=3):
    """(reference loss, reference gradient, bound on the gradient error) for the mean squared error of the
    first n_used outputs; gradients in the flat parameter layout."""
    p = reference_params(w)
    n = x.shape[0]
    out, dout, layers, (h3, dh3) = _forward(p, x)
    used = np.zeros_like(out)
    used[:, :n_used] = 1.0
    diff = (out - np.asarray(y, dtype=np.float64)) * used
    loss = float((diff ** 2).sum() / n)
    G = 2.0 * diff / n
    dG = 2.0 * dout * used / n
    dG = dG + U * (np.abs(G) + dG)
    g, bnd = {}, {}
    g["W4"] = G.T @ h3
    bnd["W4"] = np.abs(G).T @ dh3 + dG.T @ np.abs(h3) + ACC * (np.abs(G).T @ np.abs(h3))
    g["b4"] = G.sum(0)
    bnd["b4"] = dG.sum(0) + ACC * np.abs(G).sum(0)
    W = p["W4"]
    up = G @ W
    dup = dG @ np.abs(W) + ACC * (np.abs(G) @ np.abs(W))
    for l in (3, 2, 1):
        hin, dhin, z, dz = layers[l - 1]
        gp = mlp.gelu_grad(z)
        D = up * gp
        dgp = G2 * dz + (0.5 + np.abs(z) * _K * (1 + 3 * _C * z * z)) * TANH
        dD = np.abs(gp) * dup + np.abs(up) * dgp
        dD = dD + U * (np.abs(D) + dD)
        g["W%d" % l] = D.T @ hin
        bnd["W%d" % l] = np.abs(D).T @ dhin + dD.T @ np.abs(hin) + ACC * (np.abs(D).T @ np.abs(hin))
        g["b%d" % l] = D.sum(0)
        bnd["b%d" % l] = dD.sum(0) + ACC * np.abs(D).sum(0)
        W = p["W%d" % l]
        up = D @ W
        dup = dD @ np.abs(W) + ACC * (np.abs(D) @ np.abs(W))
    return loss, mlp.pack(g), mlp.pack(bnd)


def forward_bound_probabilistic(w, x, lam=6.0):
    """(reference output, bound) with the BF16 activation roundings combined by Hoeffding's inequality at
    `lam` (failure probability per output at most 2 exp(-lam^2 / 2)) and the tanh and FP32 accumulation
    errors at their worst case."""
    p = reference_params(w)
    out, _, layers, (h3, _) = _forward(p, x)
    n = x.shape[0]
    # Jacobians of the outputs with respect to h1, h2, h3 (per sample), from the output layer down
    z = [layers[l][2] for l in range(3)]
    J3 = np.broadcast_to(p["W4"], (n,) + p["W4"].shape)                     # [n][OUT][H]
    J2 = np.einsum("noh,nh,hk->nok", J3, mlp.gelu_grad(z[2]), p["W3"])
    J1 = np.einsum("noh,nh,hk->nok", J2, mlp.gelu_grad(z[1]), p["W2"])
    hs = [mlp.gelu(z[0]), mlp.gelu(z[1]), mlp.gelu(z[2])]
    var = np.zeros_like(out)
    worst = np.zeros_like(out)
    for J, h, zz in ((J1, hs[0], z[0]), (J2, hs[1], z[1]), (J3, hs[2], z[2])):
        var += np.einsum("nok,nk->no", J * J, (U * np.abs(h)) ** 2)
        worst += np.einsum("nok,nk->no", np.abs(J), np.abs(zz) * TANH / 2)
    acc = ACC * (np.abs(h3) @ np.abs(p["W4"]).T + np.abs(p["b4"]))
    return out, lam * np.sqrt(var) + worst + acc


def _emulate_gradient(p, x, y, rng, n_used=3):
    """The kernels' loss gradient with every BF16 rounding replaced by a random relative error uniform in
    [-U, U] and every tanh by a random relative error uniform in [-2^-11, 2^-11] (FP64 otherwise)."""
    n = x.shape[0]

    def rnd(v):
        return v * (1.0 + U * rng.uniform(-1.0, 1.0, v.shape))

    def th(z):
        return np.tanh(_K * (z + _C * z ** 3)) * (1.0 + TANH / 2 * rng.uniform(-1.0, 1.0, z.shape))

    h, zs = [mlp.bf16_round(x)], []
    for l in (1, 2, 3):
        z = h[-1] @ p["W%d" % l].T + p["b%d" % l]
        zs.append(z)
        h.append(rnd(0.5 * z * (1.0 + th(z))))
    out = h[3] @ p["W4"].T + p["b4"]
    d = np.zeros_like(out)
    d[:, :n_used] = out[:, :n_used] - np.asarray(y, dtype=np.float64)[:, :n_used]
    loss = float((d ** 2).sum() / n)
    G = rnd(2.0 * d / n)
    g = {"W4": G.T @ h[3], "b4": G.sum(0)}
    up = G @ p["W4"]
    for l in (3, 2, 1):
        z = zs[l - 1]
        t = th(z)
        D = rnd(up * (0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _K * (1.0 + 3 * _C * z * z)))
        g["W%d" % l], g["b%d" % l] = D.T @ h[l - 1], D.sum(0)
        up = D @ p["W%d" % l]
    return loss, mlp.pack(g)


def gradient_spread(w, x, y, runs=64, seed=0):
    """(spread of the loss, per-entry spread of the gradient): standard deviations over `runs` draws of the
    random rounding model of _emulate_gradient, the scale of the error the kernels' BF16 roundings and
    hardware tanh put on each value."""
    p = reference_params(w)
    rng = np.random.default_rng(seed)
    runs_ = [_emulate_gradient(p, x, y, rng) for _ in range(runs)]
    losses = np.array([r[0] for r in runs_])
    gs = np.stack([r[1] for r in runs_])
    return float(losses.std(ddof=1)), gs.std(axis=0, ddof=1)
