"""Pins of the FP64 MLP oracle: finite differences, closed forms, Adam's first
step, and bfloat16 rounding against torch."""
import numpy as np
import pytest

from oracle import mlp


def fd_grad(f, p, h=1e-6):
    g = np.zeros_like(p)
    for i in range(p.size):
        a, b = p.copy(), p.copy()
        a[i] += h
        b[i] -= h
        g[i] = (f(a) - f(b)) / (2 * h)
    return g


@pytest.mark.parametrize("seed", [0, 1])
def test_param_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    d, w, B = 6, 5, 7
    p = mlp.init_params(d, w, rng)
    p += 0.1 * rng.normal(size=p.size)          # non-zero biases too
    x = rng.normal(size=(B, d))
    t = rng.normal(size=B)
    loss, g, _ = mlp.backward(p, x, t, d, w)
    fd = fd_grad(lambda q: mlp.backward(q, x, t, d, w)[0], p)
    assert np.max(np.abs(g - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_input_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    d, w, B = 5, 4, 3
    p = mlp.init_params(d, w, rng) + 0.05
    x = rng.normal(size=(B, d))
    _, _, dx = mlp.backward(p, x, None, d, w)
    for b in range(B):
        f = lambda xb: mlp.forward(p, np.vstack([x[:b], xb[None], x[b + 1:]]), d, w)[0][b]
        assert np.allclose(dx[b], fd_grad(f, x[b].copy()), atol=1e-8)


def test_zero_hidden_weights_closed_form():
    """W2 = 0, b2 = 0 makes H2 = SiLU(0) = 0, so y = b3 everywhere; with
    SiLU'(0) = 1/2: dW1 = db1 = dw3 = dx = 0, db2 = w3/2 sum(dy),
    dW2 = (w3/2) (x) (H1^T dy), db3 = sum(dy)."""
    rng = np.random.default_rng(5)
    d, w, B = 8, 6, 10
    p = mlp.init_params(d, w, rng)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, d, w)
    o = w * d + w
    p[o:o + w * w] = 0.0
    p[-1] = 0.7
    x = rng.normal(size=(B, d))
    t = rng.normal(size=B)
    y, _ = mlp.forward(p, x, d, w)
    assert np.allclose(y, 0.7)
    loss, g, dx = mlp.backward(p, x, t, d, w)
    dy = 2 * (0.7 - t) / B
    h1 = mlp.silu(x @ W1.T + b1)
    dW1, db1, dW2, db2, dw3, db3 = mlp.unpack(g, d, w)
    assert np.allclose(dW1, 0) and np.allclose(db1, 0) and np.allclose(dw3, 0)
    assert np.allclose(dx, 0.0)
    assert np.allclose(db2, 0.5 * w3 * dy.sum())
    assert np.allclose(dW2, np.outer(0.5 * w3, h1.T @ dy))
    assert np.isclose(db3[0], dy.sum())


def test_adam_first_step_has_size_lr():
    rng = np.random.default_rng(1)
    p = rng.normal(size=50)
    g = rng.normal(size=50) * 10
    newp, m, v = mlp.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    assert np.allclose(np.abs(newp - p), 1e-3, rtol=1e-6)
    assert np.all(np.sign(p - newp) == np.sign(g))


def test_silu_gradient():
    z = np.linspace(-6, 6, 25)
    h = 1e-6
    assert np.allclose(mlp.silu_grad(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-9)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    a = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-5, 5, 1000),
                        [0.0, 1.0, -2.5, 1.00390625, 1.01171875]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), ref)
