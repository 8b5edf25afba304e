"""Training-side steps around the rasterizer in plain FP64 numpy -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may use this module (see the package docstring); it shares no code with the
CUDA path. ODGS trains with the 3DGS recipe (App. A.1): the optimised variables are log-scales,
opacity logits and unnormalised quaternions, activated before rasterisation, and Adam updates
them.

  * activations: s = exp(log s), o = sigmoid(logit) = 1 / (1 + exp(-logit)); the rasterizer
    normalises the quaternion itself;
  * chain rule: dL/dlog s = dL/ds * s, dL/dlogit = dL/do * o (1 - o);
  * Adam (Kingma & Ba 2015, Algorithm 1) with bias correction at step t >= 1:
        m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
        p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def activate(log_scales, logits):
    s = np.exp(np.asarray(log_scales, dtype=np.float64))
    o = 1.0 / (1.0 + np.exp(-np.asarray(logits, dtype=np.float64)))
    return s, o


def chain(log_scales, logits, d_scales, d_opacity):
    """Gradients w.r.t. the raw variables from the gradients w.r.t. the activated ones."""
    s, o = activate(log_scales, logits)
    return np.asarray(d_scales, dtype=np.float64) * s, np.asarray(d_opacity, dtype=np.float64) * o * (1.0 - o)


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step at step count t (1-based); returns new (p, m, v) in FP64. lr may be an array
    broadcast against p (per-element learning rates)."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - np.asarray(lr, dtype=np.float64) * mh / (np.sqrt(vh) + eps), m, v
