"""ERP photometric loss (L1 + D-SSIM) in plain float64 PyTorch on the CPU -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may use this module (see the package docstring); it shares no code with the
CUDA path. ODGS trains with the 3DGS loss (App. A.1 keeps 3DGS's hyper-parameters):
    L = (1 - lambda) L1 + lambda (1 - SSIM),   lambda = 0.2,
SSIM (Wang et al. 2004) with an 11 x 11 Gaussian window of sigma 1.5 and C1 = 0.01^2,
C2 = 0.03^2, on [3, H, W] images, averaged over channels and pixels.

Readings for ERP images (the paper is silent):
  * the mean over pixels may be weighted by the solid angle of each pixel row, proportional to
    cos(theta_j) with theta_j the elevation of row j's centre (Eq. 4: theta = pi (1/2 - (j + 1/2) / H));
  * the window wraps around the longitude seam (the ERP image is periodic in u) and is
    zero-padded above the first and below the last row.
The gradient is PyTorch's autograd of this forward (the L1 term's derivative at I = T is 0).
"""
from __future__ import annotations

import numpy as np

LAMBDA = 0.2
WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window_1d():
    """Normalised 11-tap Gaussian (FP64 numpy)."""
    k = np.arange(WINDOW) - WINDOW // 2
    g = np.exp(-(k * k) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def row_weights(H):
    """cos(theta_j) of the row centres (Eq. 4's elevation)."""
    theta = np.pi * (0.5 - (np.arange(H) + 0.5) / H)
    return np.cos(theta)


def _blur(t, g, wrap_u):
    """Separable 11-tap correlation of [C, H, W] (torch, FP64): u wrapped or zero-padded, v zero-padded."""
    import torch
    import torch.nn.functional as F
    r = WINDOW // 2
    C, H, W = t.shape
    x = t[:, None]  # [C, 1, H, W]
    if wrap_u:
        x = torch.cat([x[..., W - r:], x, x[..., :r]], dim=-1)
    else:
        x = F.pad(x, (r, r, 0, 0))
    x = F.pad(x, (0, 0, r, r))
    gk = torch.tensor(g, dtype=t.dtype)
    x = F.conv2d(x, gk.view(1, 1, 1, WINDOW))
    x = F.conv2d(x, gk.view(1, 1, WINDOW, 1))
    return x[:, 0]


def ssim_map(img, tgt, wrap_u=True):
    """Per-pixel, per-channel SSIM map of two [3, H, W] torch tensors (FP64)."""
    g = window_1d()
    mx = _blur(img, g, wrap_u)
    my = _blur(tgt, g, wrap_u)
    sxx = _blur(img * img, g, wrap_u) - mx * mx
    syy = _blur(tgt * tgt, g, wrap_u) - my * my
    sxy = _blur(img * tgt, g, wrap_u) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def loss_and_grad(img, tgt, lam=LAMBDA, area_weight=True, wrap_u=True):
    """(loss, dL/dimg) for numpy [3, H, W] arrays, in FP64."""
    import torch
    x = torch.tensor(np.asarray(img, dtype=np.float64), requires_grad=True)
    y = torch.tensor(np.asarray(tgt, dtype=np.float64))
    H = x.shape[1]
    w = torch.tensor(row_weights(H) if area_weight else np.ones(H), dtype=torch.float64)[None, :, None]
    wsum = 3.0 * x.shape[2] * w.sum()
    l1 = (w * (x - y).abs()).sum() / wsum
    ssim = (w * ssim_map(x, y, wrap_u)).sum() / wsum
    loss = (1.0 - lam) * l1 + lam * (1.0 - ssim)
    loss.backward()
    return float(loss.detach()), x.grad.numpy().copy()
