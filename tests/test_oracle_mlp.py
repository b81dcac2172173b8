"""Pins of the oracle's surrogate MLP (8 -> 256 -> 256 -> 4, tanh-form GELU):
gradients against central finite differences of the loss, Adam against
torch.optim.Adam on the CPU, GELU against its definition's limits and its
published distance to the erf form."""
import math

import numpy as np
import pytest

import oracle as O


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in O.MLP_SHAPES.items():
        fan_in = shp[1] if len(shp) == 2 else 16
        p[k] = rng.normal(0, scale / math.sqrt(fan_in) * 3, shp)
    return p


def test_gelu_definition():
    assert O.gelu(0.0) == 0.0
    assert abs(O.gelu(10.0) - 10.0) < 1e-12 and abs(O.gelu(-10.0)) < 1e-12
    for x in np.linspace(-5, 5, 101):
        exact = 0.5 * x * (1 + math.erf(x / math.sqrt(2)))
        assert abs(O.gelu(x) - exact) < 2e-3   # tanh form vs erf form (Hendrycks & Gimpel)
        assert abs(O.gelu(x) - O.gelu(-x) - x) < 1e-12  # gelu(x) - gelu(-x) = x


def test_backward_matches_finite_differences():
    p = _params(1)
    rng = np.random.default_rng(2)
    x = rng.random((5, 8))
    t = rng.normal(0, 1, (5, 4))
    loss, g = O.mlp_backward(p, x, t)
    y = O.mlp_forward(p, x)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-12
    h = 1e-6
    for k in O.MLP_ORDER:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = np.mean((O.mlp_forward(p, x) - t) ** 2)
            flat[idx] = old - h
            lm = np.mean((O.mlp_forward(p, x) - t) ** 2)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    w = rng.normal(0, 1, 50)
    m, v = np.zeros(50), np.zeros(50)
    tw = torch.tensor(w.copy(), requires_grad=True)
    opt = torch.optim.Adam([tw], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = rng.normal(0, 1, 50)
        O.adam(w, g, m, v, 1e-3, 0.9, 0.999, 1e-8, step)
        opt.zero_grad()
        tw.grad = torch.tensor(g)
        opt.step()
        assert np.allclose(w, tw.detach().numpy(), rtol=0, atol=1e-12)
