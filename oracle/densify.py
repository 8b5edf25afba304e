"""Densification of ODGS (Sec. 3.3, App. A.1) in plain numpy -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may use this module (see the package docstring). It restates the method; it
shares no code with the CUDA path.

ODGS keeps the 3DGS densification loop and changes one thing: the gradient threshold of a
Gaussian depends on its elevation theta_mu seen from the camera,
    tau_mu = tau_min + (1 - cos theta_mu) (tau_max - tau_min),  tau_min = 2e-5, tau_max = 1e-4,
so that Gaussians near the poles, which the ERP projection stretches, are densified less.

Readings (the paper is silent on them):
  * statistics per Gaussian over the views in which it was visible (survived culling):
    the sum of || (dL/du * W/2, dL/dv * H/2) || (the ERP-mean gradient in the [-1, 1] image
    coordinates in which 3DGS states its threshold), the sum of 1 - cos theta_mu, and the count;
    the Gaussian is densified when the mean gradient reaches tau_mu taken at the mean of
    1 - cos theta_mu over those views;
  * densified Gaussians are cloned when their largest scale is at most percent_dense x the
    scene extent (App. A.1: percent_dense = 1e-3), split into two otherwise; a split child is
    placed at mu + R(q) (s * z) with z ~ N(0, I) (passed in) and has the scales s / 1.6;
  * Gaussians with opacity below min_opacity (or, when max_scale > 0, a scale above it) are
    removed together with their clones or children;
  * output order: kept and cloned originals in index order, then the clones, then the first
    children of the split Gaussians, then their second children.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import oracle as O

TAU_MIN = 2e-5   # App. A.1, densify_grad_threshold_min
TAU_MAX = 1e-4   # App. A.1, densify_grad_threshold_max
PERCENT_DENSE = 1e-3  # App. A.1

KEEP, CLONE, SPLIT, PRUNE = 0, 1, 2, 4


@dataclass
class DensifyParams:
    tau_min: float = TAU_MIN
    tau_max: float = TAU_MAX
    percent_dense: float = PERCENT_DENSE
    scene_extent: float = 1.0
    min_opacity: float = 0.005
    max_scale: float = 0.0
    raw_params: bool = False  # scales are log-scales, opacity logits


def tau(one_minus_cos):
    """Sec. 3.3: the elevation-dependent gradient threshold (FP64)."""
    return TAU_MIN + np.asarray(one_minus_cos, dtype=np.float64) * (TAU_MAX - TAU_MIN)


def stats(p: O.Params, views, st: O.Settings, dLdC, pix=None):
    """Sums over the views of (gradient norm, 1 - cos theta, visible count) per Gaussian.

    dLdC[v] is the loss gradient w.r.t. view v's image ([3, H, W], or [npix, 3] for the pixels
    pix[v]). Returns float64, float64, int64 arrays of length n.
    """
    n = p.n
    grad = np.zeros(n)
    elev = np.zeros(n)
    count = np.zeros(n, dtype=np.int64)
    for k, v in enumerate(views):
        pj = O.project(p, v, st)
        visible = pj[:, O.PJ_VALID] > 0
        g = O.backward(p, v, st, dLdC[k], pix=None if pix is None else pix[k], want_g2=True)["screen"]
        gu = g[:, 0] * (v.width / 2.0)
        gv = g[:, 1] * (v.height / 2.0)
        norm = np.sqrt(gu * gu + gv * gv)
        grad += np.where(visible, norm, 0.0)
        elev += np.where(visible, 1.0 - np.cos(pj[:, O.PJ_THETA]), 0.0)
        count += visible
    return grad, elev, count


def select(grad, elev, count, scales, opacity, prm: DensifyParams):
    """Action per Gaussian from float32 statistics, decided in float32 (the kernel's precision):
    mean gradient g / c and mean 1 - cos theta e / c, each one rounded division; tau as one
    rounded product and one rounded sum; ties at the threshold densify."""
    f = np.float32
    grad = np.asarray(grad, dtype=f)
    elev = np.asarray(elev, dtype=f)
    count = np.asarray(count, dtype=np.uint32)
    seen = count > 0
    c = np.where(seen, count, 1).astype(f)
    gmean = np.where(seen, grad / c, f(0))
    emean = np.where(seen, elev / c, f(0))
    t = f(prm.tau_min) + emean * (f(prm.tau_max) - f(prm.tau_min))
    hot = seen & (gmean >= t)
    smax = np.max(np.asarray(scales, dtype=f), axis=1)
    op = np.asarray(opacity, dtype=f)
    if prm.raw_params:
        # thresholds mapped into log-scale / logit space once, in double, then rounded to float
        pd, ext, mo = (float(f(x)) for x in (prm.percent_dense, prm.scene_extent, prm.min_opacity))
        big_thr = f(np.log(pd * ext))
        op_thr = f(np.log(mo / (1.0 - mo))) if mo > 0 else f(-np.inf)
        max_thr = f(np.log(float(f(prm.max_scale)))) if prm.max_scale > 0 else f(np.inf)
    else:
        big_thr = f(prm.percent_dense) * f(prm.scene_extent)
        op_thr = f(prm.min_opacity)
        max_thr = f(prm.max_scale) if prm.max_scale > 0 else f(np.inf)
    big = smax > big_thr
    prune = (op < op_thr) | (smax > max_thr)
    act = np.where(hot, np.where(big, SPLIT, CLONE), KEEP)
    return np.where(prune, PRUNE, act).astype(np.uint8)


def _rotation(q):
    """Rotation matrices of the normalised quaternions (w, x, y, z), FP64."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def apply(means, scales, quats, opacity, sh, action, noise, raw_params=False):
    """New parameter arrays (FP64) after cloning, splitting and pruning; noise is [n, 2, 3].
    With raw_params the scales are log-scales: children get log s - ln 1.6."""
    action = np.asarray(action)
    keep = (action == KEEP) | (action == CLONE)
    clone = action == CLONE
    split = action == SPLIT
    arrays = [np.asarray(a, dtype=np.float64) for a in (means, scales, quats, opacity, sh)]
    out = [np.concatenate([a[keep], a[clone], a[split], a[split]]) for a in arrays]
    if split.any():
        R = _rotation(arrays[2][split])
        s = np.exp(arrays[1][split]) if raw_params else arrays[1][split]
        mu = arrays[0][split]
        kids = []
        for c in range(2):
            z = np.asarray(noise, dtype=np.float64)[split, c]
            kids.append(mu + np.einsum("nij,nj->ni", R, s * z))
        nk, nc, ns = int(keep.sum()), int(clone.sum()), int(split.sum())
        out[0][nk + nc:nk + nc + ns] = kids[0]
        out[0][nk + nc + ns:] = kids[1]
        out[1][nk + nc:] = out[1][nk + nc:] - np.log(1.6) if raw_params else out[1][nk + nc:] / 1.6
    return out
