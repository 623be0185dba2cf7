"""Adam update (Kingma & Ba 2015), the optimiser the paper's training listings
use (``optax.adam``, Sec. III.D and the Rydberg example).  TEST INFRASTRUCTURE ONLY.

m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
theta <- theta - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps),  t = 1, 2, ...
"""
from __future__ import annotations

import numpy as np


def adam_step(theta, m, v, g, t, lr=2e-2, b1=0.9, b2=0.999, eps=1e-8):
    """One step at iteration t (1-based).  Returns new (theta, m, v)."""
    theta = np.asarray(theta, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
