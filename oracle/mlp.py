"""CPU oracle for the rank-bracket network (fp64 numpy). TEST INFRASTRUCTURE ONLY.

Network: x (41) -> relu(x W1 + b1) (64) -> relu(h1 W2 + b2) (64) -> o = h2 W3 + b3 (2),
mu = o[0], s = clamp(o[1], -8, 2). Loss per row: 0.5 (y - mu)^2 exp(-2 s) + s (the negative
log-likelihood of y under N(mu, e^s) up to a constant); the batch loss is the mean.
The parameter vector layout: W1[41][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2].
The gradient below is derived by hand from these formulas (chain rule layer by layer).
parity pinned by central finite differences and closed forms (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

F, H = 41, 64
SIZES = [("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, 2)), ("b3", (2,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def bf16_values(bits: np.ndarray) -> np.ndarray:
    """bf16 bit patterns -> their exact values as float64."""
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def forward(p: np.ndarray, x: np.ndarray):
    w = unpack(np.asarray(p, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ w["W1"] + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"] + w["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ w["W3"] + w["b3"]
    return o, (x, z1, h1, z2, h2)


def loss_and_grad(p: np.ndarray, x: np.ndarray, y: np.ndarray):
    w = unpack(np.asarray(p, dtype=np.float64))
    o, (x, z1, h1, z2, h2) = forward(p, x)
    n = x.shape[0]
    mu, s_raw = o[:, 0], o[:, 1]
    s = np.clip(s_raw, -8.0, 2.0)
    e = np.asarray(y, dtype=np.float64) - mu
    inv = np.exp(-2.0 * s)
    loss = np.mean(0.5 * e * e * inv + s)
    d_o = np.zeros_like(o)
    d_o[:, 0] = -e * inv / n
    inside = (s_raw > -8.0) & (s_raw < 2.0)
    d_o[:, 1] = np.where(inside, (1.0 - e * e * inv) / n, 0.0)
    g = {}
    g["W3"] = h2.T @ d_o
    g["b3"] = d_o.sum(axis=0)
    d_h2 = d_o @ w["W3"].T
    d_z2 = d_h2 * (z2 > 0)
    g["W2"] = h1.T @ d_z2
    g["b2"] = d_z2.sum(axis=0)
    d_h1 = d_z2 @ w["W2"].T
    d_z1 = d_h1 * (z1 > 0)
    g["W1"] = x.T @ d_z1
    g["b1"] = d_z1.sum(axis=0)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return float(loss), flat


def loss_only(p, x, y) -> float:
    o, _ = forward(p, x)
    mu = o[:, 0]
    s = np.clip(o[:, 1], -8.0, 2.0)
    e = np.asarray(y, dtype=np.float64) - mu
    return float(np.mean(0.5 * e * e * np.exp(-2.0 * s) + s))
