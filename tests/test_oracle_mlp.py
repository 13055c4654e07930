"""Pins of the FP64 reference network of the learned closure (oracle/mlp.py): backward against central
finite differences of the loss, GELU against torch's tanh-approximate GELU, BF16 rounding against
torch's bfloat16 conversion."""
import numpy as np
import pytest

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.normal(size=mlp.NPARAM) * 0.2
    x = rng.normal(size=(7, mlp.NI))
    y = rng.normal(size=(7, mlp.NO))
    loss, g = mlp.loss_and_grad(w, x, y)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, x, y)[0] - mlp.loss_and_grad(wm, x, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))
    # outputs beyond the first 3 carry no loss
    p = mlp.unpack(g)
    assert np.all(p["W4"][3:] == 0) and np.all(p["b4"][3:] == 0)


def test_gelu_matches_torch_tanh_gelu():
    torch = pytest.importorskip("torch")
    z = np.linspace(-6, 6, 101)
    ref = torch.nn.functional.gelu(torch.tensor(z), approximate="tanh").numpy()
    assert np.max(np.abs(mlp.gelu(z) - ref)) < 1e-12
    # derivative by central differences
    h = 1e-6
    assert np.max(np.abs(mlp.gelu_grad(z) - (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h))) < 1e-8


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(1).normal(size=1000) * 10.0 ** np.random.default_rng(2).uniform(-5, 5, 1000)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(v), ref)
