"""Densification of ODGS (Sec. 3.3, App. A.1) on the device.

The backward preprocess adds, per Gaussian and per view in which it was visible, the norm of its
ERP-mean gradient (in 3DGS's [-1, 1] image units), 1 - cos(elevation) and 1 to three running
sums (``DensifyStats``, passed to ``Rasterizer.backward(..., densify=stats)``). ``select`` turns
them into KEEP / CLONE / SPLIT / PRUNE with the threshold
    tau = tau_min + (1 - cos theta) (tau_max - tau_min),
and ``apply`` builds the new parameter arrays (kept, then clones, then the split children).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L

KEEP, CLONE, SPLIT, PRUNE = 0, 1, 2, 4


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _stream(device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


@dataclass
class DensifyParams:
    tau_min: float = 2e-5       # App. A.1
    tau_max: float = 1e-4       # App. A.1
    percent_dense: float = 1e-3  # App. A.1
    scene_extent: float = 1.0
    min_opacity: float = 0.005
    max_scale: float = 0.0
    raw_params: bool = False  # scales are log-scales and opacity logits

    def to_c(self) -> L.DensifyParams:
        return L.DensifyParams(self.tau_min, self.tau_max, self.percent_dense, self.scene_extent, self.min_opacity,
                               self.max_scale, int(bool(self.raw_params)))


class DensifyStats:
    """Running sums of the densification statistics of n Gaussians (float32, float32, int32)."""

    def __init__(self, n: int, device=None):
        device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.grad = torch.zeros(n, dtype=torch.float32, device=device)
        self.elev = torch.zeros(n, dtype=torch.float32, device=device)
        self.count = torch.zeros(n, dtype=torch.int32, device=device)

    def reset(self):
        self.grad.zero_()
        self.elev.zero_()
        self.count.zero_()


def select(stats: DensifyStats, scales: torch.Tensor, opacity: torch.Tensor,
           params: DensifyParams = None) -> torch.Tensor:
    """One action byte per Gaussian (KEEP, CLONE, SPLIT or PRUNE)."""
    params = params or DensifyParams()
    n = stats.grad.numel()
    dev = stats.grad.device
    for t in (scales, opacity):
        if t.dtype != torch.float32 or not t.is_contiguous() or t.device != dev:
            raise ValueError("scales and opacity must be contiguous float32 tensors on the statistics' device")
    if scales.shape != (n, 3) or opacity.numel() != n:
        raise ValueError("scales [n, 3] and opacity [n] must match the statistics")
    action = torch.empty(n, dtype=torch.uint8, device=dev)
    lib = L.load()
    prm = params.to_c()
    L.check(lib.odgs_densify_select(_ptr(stats.grad), _ptr(stats.elev), _ptr(stats.count), _ptr(scales),
                                    _ptr(opacity), int(n), C.byref(prm), _ptr(action), _stream(dev)),
            "odgs_densify_select")
    return action


def apply(means, scales, quats, opacity, sh, action, noise=None, generator=None, raw_params=False):
    """Densified (means, scales, quats, opacity, sh). noise: [n, 2, 3] standard normal draws for
    the split children (drawn with ``generator`` when None). raw_params: scales are log-scales.
    Synchronizes once to read the count."""
    n = means.shape[0]
    dev = means.device
    if noise is None:
        noise = torch.randn((n, 2, 3), device=dev, dtype=torch.float32, generator=generator)
    ins = [means, scales, quats, opacity, sh, noise]
    for t in ins:
        if t.dtype != torch.float32 or not t.is_contiguous() or t.device != dev:
            raise ValueError("parameters and noise must be contiguous float32 tensors on one device")
    if action.dtype != torch.uint8 or action.numel() != n:
        raise ValueError("action must be a uint8 tensor of n elements")
    k = sh.shape[1]
    cap = 2 * n
    out = [torch.empty((cap,) + tuple(t.shape[1:]), dtype=torch.float32, device=dev)
           for t in (means, scales, quats, opacity, sh)]
    lib = L.load()
    nbytes = C.c_size_t()
    L.check(lib.odgs_densify_scratch_size(int(n), C.byref(nbytes)), "odgs_densify_scratch_size")
    scratch = torch.empty(max(int(nbytes.value), 16), dtype=torch.uint8, device=dev)
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    g = L.Gaussians(_ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity), _ptr(sh), int(n))
    o = L.ParamsOut(*[_ptr(t) for t in out])
    L.check(lib.odgs_densify_apply(C.byref(g), int(k), int(bool(raw_params)), _ptr(action), _ptr(noise), C.byref(o),
                                   int(cap),
                                   _ptr(n_out), _ptr(scratch), C.c_size_t(scratch.numel()), _stream(dev)),
            "odgs_densify_apply")
    m = int(n_out.item())
    if m > cap:  # cannot happen: every Gaussian yields at most two outputs
        raise RuntimeError(f"odgs_densify_apply: {m} outputs for capacity {cap}")
    return [t[:m] for t in out]
