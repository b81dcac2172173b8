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


def test_forward_matches_torch_fp64():
    """The forward pass against an independent fp64 restatement: torch's
    linear layers and its tanh-form GELU on the CPU (a library, not the
    oracle's own code).  A dropped bias, a GELU taken before the wrong
    layer or a transposed weight changes the outputs by O(1)."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    p = _params(11, scale=1.0)
    x = np.random.default_rng(12).random((37, 8))
    t = {k: torch.tensor(v, dtype=torch.float64) for k, v in p.items()}
    h1 = F.gelu(F.linear(torch.tensor(x), t["W1"], t["b1"]), approximate="tanh")
    h2 = F.gelu(F.linear(h1, t["W2"], t["b2"]), approximate="tanh")
    ref = F.linear(h2, t["W3"], t["b3"]).numpy()
    y = O.mlp_forward(p, x)
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12), np.abs(y - ref).max()


def _gelu_hand(z):
    return 0.5 * z * (1.0 + math.tanh(math.sqrt(2.0 / math.pi) * (z + 0.044715 * z ** 3)))


def test_forward_hand_worked_two_unit_network():
    """Hand-worked case: one path through hidden unit 3 of layer 1 and unit 5
    of layer 2 into output 1, every other weight zero.
        z1 = 0.5 x0 - 2 x7 + 0.25,  h1 = gelu(z1)
        z2 = 1.5 h1 - 0.75,         h2 = gelu(z2)
        y1 = -2 h2 + 0.125;  y0 = 0.5 gelu(b2[9]) with b2[9] = 1; y2 = y3 = b3
    Output 0 exercises layer 2's bias and GELU with no layer-1 input; output 1
    the whole chain."""
    p = {k: np.zeros(shp) for k, shp in O.MLP_SHAPES.items()}
    p["W1"][3, 0], p["W1"][3, 7], p["b1"][3] = 0.5, -2.0, 0.25
    p["W2"][5, 3], p["b2"][5] = 1.5, -0.75
    p["b2"][9] = 1.0
    p["W3"][1, 5], p["b3"][1] = -2.0, 0.125
    p["W3"][0, 9] = 0.5
    p["b3"][2], p["b3"][3] = -3.0, 7.0
    for x0, x7 in ((0.2, 0.9), (1.0, 0.0), (0.0, 0.4)):
        x = np.zeros((1, 8))
        x[0, 0], x[0, 7] = x0, x7
        h1 = _gelu_hand(0.5 * x0 - 2.0 * x7 + 0.25)
        h2 = _gelu_hand(1.5 * h1 - 0.75)
        want = [0.5 * _gelu_hand(1.0), -2.0 * h2 + 0.125, -3.0, 7.0]
        y = O.mlp_forward(p, x)[0]
        assert np.allclose(y, want, rtol=0, atol=1e-14), (y, want)
