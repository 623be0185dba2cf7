"""Warm-start MLP in float64 -- TEST INFRASTRUCTURE ONLY.

No counterpart in the paper.  y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with the
periodic angle loss L = sum mask * 2 (1 - cos(y - t)) / sum mask.  With
``bf16=True`` every GEMM operand is rounded to bfloat16 (round to nearest even)
at the points where the CUDA kernels round; sums are exact float64.  With
``bf16=False`` the network is smooth, which lets finite differences pin the
backward formulas.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round float64/float32 values to bfloat16 (nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def _r(a, on):
    return bf16(a) if on else np.asarray(a, dtype=np.float64)


def forward(x, w1, b1, w2, b2, w3, b3, bf=True):
    z1 = _r(x, bf) @ _r(w1, bf) + b1
    z2 = _r(np.maximum(z1, 0), bf) @ _r(w2, bf) + b2
    y = _r(np.maximum(z2, 0), bf) @ _r(w3, bf) + b3
    return z1, z2, y


def loss_and_dy(y, t, mask):
    ms = mask.sum()
    inv = 1.0 / ms if ms > 0 else 0.0
    loss = float((mask * 2 * (1 - np.cos(y - t))).sum() * inv)
    dy = mask * 2 * np.sin(y - t) * inv
    return loss, dy


def backward(x, w1, w2, w3, z1, z2, dy, bf=True):
    """Gradients (gw1, gb1, gw2, gb2, gw3, gb3) given dL/dy."""
    a2 = np.maximum(z2, 0)
    a1 = np.maximum(z1, 0)
    gw3 = _r(a2, bf).T @ _r(dy, bf)
    gb3 = dy.sum(0)
    dz2 = (_r(dy, bf) @ _r(w3, bf).T) * (z2 > 0)
    gw2 = _r(a1, bf).T @ _r(dz2, bf)
    gb2 = dz2.sum(0)
    dz1 = (_r(dz2, bf) @ _r(w2, bf).T) * (z1 > 0)
    gw1 = _r(x, bf).T @ _r(dz1, bf)
    gb1 = dz1.sum(0)
    return gw1, gb1, gw2, gb2, gw3, gb3


def init(F, H, O, seed=0):
    """He-style initialisation (float32 master weights)."""
    rng = np.random.default_rng(seed)
    w1 = (rng.standard_normal((F, H)) * np.sqrt(2.0 / F)).astype(np.float32)
    w2 = (rng.standard_normal((H, H)) * np.sqrt(2.0 / H)).astype(np.float32)
    w3 = (rng.standard_normal((H, O)) * np.sqrt(1.0 / H)).astype(np.float32)
    return dict(w1=w1, b1=np.zeros(H, np.float32), w2=w2, b2=np.zeros(H, np.float32),
                w3=w3, b3=np.zeros(O, np.float32))
