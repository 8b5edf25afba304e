"""Shared helpers for the parity tests: run the CUDA path and the oracle on the same scene."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

F32 = lambda x: float(np.float32(x))  # noqa: E731  (settings are float32 on the device)

# Image tolerance and decision bands (see the oracle's blend_pixel margins).
IMG_TOL = 1e-4
EPS_SKIP = 2e-5
EPS_TERM = 1e-4
EPS_CLAMP = 2e-5
GRAD_TOL = 1e-3
# element-wise gradient band: |g - g_ref| <= GRAD_BAND * (|g_ref| + GRAD_FLOOR * max|g_ref|), per
# tensor, for every element (no fraction may fall outside)
GRAD_BAND = 1e-3
GRAD_FLOOR = 1e-3
GRAD_NAMES = ("means", "scales", "quats", "opacity", "sh")


def oracle_settings(rs, deg=None):
    return O.Settings(sh_degree=rs.sh_degree if deg is None else deg, dilation=F32(rs.cov_dilation),
                      r_near=F32(rs.r_near), r_far=F32(rs.r_far), bg=tuple(F32(b) for b in rs.bg))


def to_torch(scene, device="cuda", requires_grad=False):
    import torch
    ts = [torch.tensor(a, device=device, requires_grad=requires_grad)
          for a in (scene.means, scene.scales, scene.quats, scene.opacity, scene.sh)]
    return ts


def gpu_render(scene, rs, views=None, rast=None, want_T=True):
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    views = scene.views if views is None else views
    rast = rast or Rasterizer()
    m, s, q, o, sh = to_torch(scene)
    imgs, Ts = rast.forward(m, s, q, o, sh, views, rs, want_T=want_T)
    torch.cuda.synchronize()
    assert rast.status() == 0, f"device status {rast.status()}"
    out = [im.cpu().numpy().astype(np.float64) for im in imgs]
    Tn = [t.cpu().numpy().astype(np.float64) for t in Ts] if want_T else None
    return out, Tn, rast


def compare_image(gpu, ref, margins, tol=IMG_TOL, max_amb_frac=2e-3):
    """Max-abs over non-ambiguous pixels; returns (max_err, ambiguous fraction)."""
    amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM)
    if gpu.ndim == 3:  # [3, H, W]
        err = np.abs(gpu - ref).max(axis=0)
    else:  # [npix, 3]
        err = np.abs(gpu - ref).max(axis=1)
    ok = ~amb
    max_err = float(err[ok].max()) if ok.any() else 0.0
    frac = float(amb.mean())
    assert frac <= max_amb_frac, f"ambiguous pixel fraction {frac}"
    assert max_err <= tol, f"max abs error {max_err} (worst at {np.unravel_index(np.argmax(np.where(ok, err, 0)), err.shape)})"
    return max_err, frac


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def assert_grads_close(gpu, ref, names=GRAD_NAMES, tol=GRAD_TOL):
    """Gradient parity per parameter tensor: relative L2 error <= tol and every element within
    GRAD_BAND * (|g_ref| + GRAD_FLOOR * max|g_ref|). The message names the worst element."""
    for k in names:
        g = np.asarray(gpu[k], np.float64).ravel()
        r = np.asarray(ref[k], np.float64).ravel()
        e = rel_l2(g, r)
        assert e <= tol, f"{k}: relative L2 error {e:.3e}"
        if r.size == 0:
            continue
        lim = GRAD_BAND * (np.abs(r) + GRAD_FLOOR * np.abs(r).max())
        d = np.abs(g - r)
        bad = d > lim
        if bad.any():
            i = int(np.argmax(np.where(lim > 0, d / np.where(lim > 0, lim, 1.0), np.inf * (d > 0))))
            raise AssertionError(
                f"{k}: {int(bad.sum())} of {bad.size} elements outside the element-wise band; worst index {i}: "
                f"gpu {g[i]:.9e} ref {r[i]:.9e} |d| {d[i]:.3e} > band {lim[i]:.3e} (max|ref| {np.abs(r).max():.3e})")
