"""FP64 reference of the learned closure network (test infrastructure only).

Plain numpy forward and backward of x -> 64 -> 64 -> 64 -> out with the tanh form of GELU
(Hendrycks & Gimpel) on the hidden layers, loss = mean over samples of the squared error summed over
the first `n_used` outputs.  Parameters use the flat layout of lbm_closure_set_weights:
W1[64][32] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[8][64] b4[8].

Pinned by finite differences of the loss (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

NI, NH, NO = 32, 64, 8
SHAPES = [("W1", (NH, NI)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
          ("W4", (NO, NH)), ("b4", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(w):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(w[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def pack(p):
    return np.concatenate([p[name].ravel() for name, _ in SHAPES])


_K = np.sqrt(2.0 / np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_K * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_K * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _K * (1.0 + 3 * 0.044715 * z * z)


def forward(w, x):
    p = unpack(w)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l in (1, 2, 3):
        z = h @ p["W%d" % l].T + p["b%d" % l]
        cache.append((h, z))
        h = gelu(z)
    out = h @ p["W4"].T + p["b4"]
    return out, (cache, h)


def loss_and_grad(w, x, y, n_used=3):
    p = unpack(w)
    out, (cache, h3) = forward(w, x)
    n = x.shape[0]
    diff = np.zeros_like(out)
    diff[:, :n_used] = out[:, :n_used] - np.asarray(y, dtype=np.float64)[:, :n_used]
    loss = float((diff ** 2).sum() / n)
    g = {}
    dout = 2.0 * diff / n
    g["W4"] = dout.T @ h3
    g["b4"] = dout.sum(0)
    dh = dout @ p["W4"]
    for l in (3, 2, 1):
        hin, z = cache[l - 1]
        dz = dh * gelu_grad(z)
        g["W%d" % l] = dz.T @ hin
        g["b%d" % l] = dz.sum(0)
        dh = dz @ p["W%d" % l]
    return loss, pack(g)


def bf16_round(a):
    """Round float values to bfloat16 (nearest even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    rnd = ((bits >> 16) & 1) + 0x7FFF
    out = ((bits + rnd) >> 16) << 16
    return out.astype(np.uint32).view(np.float32).astype(np.float64)
