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


# rounding-error bound of a float32 evaluation of a sum of per-pixel contributions, in units of the
# sum of their absolute values: about 20-30 roundings per contribution (the blend's transmittance
# recovery and arithmetic, the summation tree), with a factor 2 of margin
SUM_BOUND = 64.0 * 2.0 ** -24


def assert_grads_close(gpu, ref, names=GRAD_NAMES, tol=GRAD_TOL, slack=None, what=""):
    """Gradient parity per parameter tensor: relative L2 error <= tol and every element within
    GRAD_BAND * (|g_ref| + GRAD_FLOOR * max|g_ref|), plus slack[k] (per element) when given. The
    message names the worst element."""
    for k in names:
        g = np.asarray(gpu[k], np.float64).ravel()
        r = np.asarray(ref[k], np.float64).ravel()
        e = rel_l2(g, r)
        assert e <= tol, f"{what}{k}: relative L2 error {e:.3e}"
        if r.size == 0:
            continue
        lim = GRAD_BAND * (np.abs(r) + GRAD_FLOOR * np.abs(r).max())
        if slack is not None:
            lim = lim + np.asarray(slack[k], np.float64).ravel()
        d = np.abs(g - r)
        bad = d > lim
        if bad.any():
            i = int(np.argmax(np.where(lim > 0, d / np.where(lim > 0, lim, 1.0), np.inf * (d > 0))))
            raise AssertionError(
                f"{what}{k}: {int(bad.sum())} of {bad.size} elements outside the element-wise band; worst index {i}: "
                f"gpu {g[i]:.9e} ref {r[i]:.9e} |d| {d[i]:.3e} > band {lim[i]:.3e} (max|ref| {np.abs(r).max():.3e})")


def slice_params(pj):
    """The conic of the oracle's projection records [n, PJ_NFIELDS] in slice form (a, beta, gamma):
    a dx^2 + 2 b dx dy + c dy^2 = a (dx - beta dy)^2 + gamma dy^2, i.e. beta = -b / a and
    gamma = c - b^2 / a (FP64; zeros where the Gaussian is culled)."""
    a, b, c = (pj[:, O.PJ_CONIC + i] for i in range(3))
    ok = a > 0
    sa = np.where(ok, a, 1.0)
    return np.where(ok, a, 0.0), np.where(ok, -b / sa, 0.0), np.where(ok, c - b * b / sa, 0.0)


def screen_xy_to_slice(g2, pj):
    """Screen-space gradients [n, 9] with the conic in image-axis entries (a, b, c; b the single
    off-diagonal variable) -> the same with the conic in slice form (a, beta, gamma): since the
    entries are (a, -a beta, gamma + a beta^2), dL/da = dL/da' - beta dL/db' + beta^2 dL/dc',
    dL/dbeta = -a dL/db' + 2 a beta dL/dc', dL/dgamma = dL/dc'."""
    a, beta, _ = slice_params(pj)
    out = np.array(g2, dtype=np.float64, copy=True)
    da, db, dc = g2[:, 2], g2[:, 3], g2[:, 4]
    out[:, 2] = da - beta * db + beta * beta * dc
    out[:, 3] = -a * db + 2.0 * a * beta * dc
    out[:, 4] = dc
    return out


def screen_slice_to_xy(g2, pj):
    """Inverse of screen_xy_to_slice (FP64)."""
    a, beta, _ = slice_params(pj)
    sa = np.where(a > 0, a, 1.0)
    out = np.array(g2, dtype=np.float64, copy=True)
    ga, gb, gg = g2[:, 2], g2[:, 3], g2[:, 4]
    out[:, 4] = gg
    out[:, 3] = np.where(a > 0, 2.0 * beta * gg - gb / sa, 0.0)
    out[:, 2] = np.where(a > 0, ga + beta * beta * gg - beta * gb / sa, 0.0)
    return out


def screen_abs_xy_to_slice(g2abs, pj):
    """Bounds of the absolute per-pixel contribution sums of the slice-form conic gradients from
    those of the image-axis entries (triangle inequality on the linear map of screen_xy_to_slice)."""
    a, beta, _ = slice_params(pj)
    out = np.array(g2abs, dtype=np.float64, copy=True)
    aa, ab, ac = g2abs[:, 2], g2abs[:, 3], g2abs[:, 4]
    out[:, 2] = aa + np.abs(beta) * ab + beta * beta * ac
    out[:, 3] = np.abs(a) * ab + 2.0 * np.abs(a * beta) * ac
    out[:, 4] = ac
    return out
