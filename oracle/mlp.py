"""FP64 reference of the MLP surrogate of E(theta) (oracle side; test
infrastructure only).

Architecture: x (d_in) -> Linear(d_in, w) -> SiLU -> Linear(w, w) -> SiLU ->
Linear(w, 1). Loss: mean squared error. Optimiser: Adam with bias correction.
The paper has no learned component; this network is the surrogate that
proposes optimiser steps for the VQE loop of Sec. V.B, checked by the MPS.

Flat parameter order: W1 (w x d_in, row-major), b1 (w), W2 (w x w), b2 (w),
w3 (w), b3 (1).

With ``quantize=True`` the operands of the four GEMMs of a training step are
rounded to bfloat16 (round to nearest even) at the same points as the GPU
kernels: x, W1, H1 = SiLU(Z1), W2, dZ2, dZ1. Everything else stays FP64.

Pins (``tests/test_oracle_mlp.py``): gradients against central finite
differences, a closed form with zero hidden weights, Adam's first step of
size lr, and bf16 rounding against torch's conversion.
"""
import numpy as np


def n_params(d_in, w):
    return w * d_in + w + w * w + w + w + 1


def init_params(d_in, w, rng):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    p = []
    p.append(rng.uniform(-1, 1, (w, d_in)) / np.sqrt(d_in))
    p.append(np.zeros(w))
    p.append(rng.uniform(-1, 1, (w, w)) / np.sqrt(w))
    p.append(np.zeros(w))
    p.append(rng.uniform(-1, 1, w) / np.sqrt(w))
    p.append(np.zeros(1))
    return np.concatenate([a.ravel() for a in p])


def unpack(params, d_in, w):
    o = 0
    out = []
    for shape in ((w, d_in), (w,), (w, w), (w,), (w,), (1,)):
        k = int(np.prod(shape))
        out.append(np.asarray(params[o:o + k], dtype=np.float64).reshape(shape))
        o += k
    return out


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, d_in, w, quantize=False):
    q = bf16_round if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(params, d_in, w)
    x = np.asarray(x, dtype=np.float64)
    z1 = q(x) @ q(W1).T + b1
    h1 = silu(z1)
    z2 = q(h1) @ q(W2).T + b2
    h2 = silu(z2)
    y = h2 @ w3 + b3[0]
    return y, (x, z1, h1, z2, h2)


def backward(params, x, target, d_in, w, quantize=False):
    """Returns (loss, grad_params, grad_x). With target None the loss is the
    sum of outputs (so grad_x is dy/dx row by row) and loss is y."""
    q = bf16_round if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(params, d_in, w)
    y, (x, z1, h1, z2, h2) = forward(params, x, d_in, w, quantize)
    B = x.shape[0]
    if target is None:
        loss = y
        dy = np.ones(B)
    else:
        r = y - np.asarray(target, dtype=np.float64)
        loss = float(np.mean(r * r))
        dy = 2.0 * r / B
    dw3 = h2.T @ dy
    db3 = np.array([dy.sum()])
    dz2 = (dy[:, None] * w3[None, :]) * silu_grad(z2)
    dW2 = q(dz2).T @ q(h1)
    db2 = dz2.sum(axis=0)
    dh1 = q(dz2) @ q(W2)
    dz1 = dh1 * silu_grad(z1)
    dW1 = q(dz1).T @ q(x)
    db1 = dz1.sum(axis=0)
    dx = q(dz1) @ q(W1)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])
    return loss, grad, dx


def adam_step(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1). Returns new (params, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
