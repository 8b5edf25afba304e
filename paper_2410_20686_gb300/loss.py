"""Fused L1 + D-SSIM loss of 3DGS training on ERP images (forward and gradient on the device).

    L = sum over views of (1 - lambda) L1 + lambda (1 - SSIM),   lambda = 0.2,

SSIM with an 11 x 11 Gaussian window (sigma 1.5); both terms are means over each view's
3 x W x H values, weighted per row by cos(theta) (the row's solid angle) when area_weight, with
the window wrapping around the longitude seam when wrap_u. ``l1_dssim`` has the signature of a
``GraphedFrame`` loss function: (images, targets) -> (loss, [dL/dimage]).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def l1_dssim(images, targets, lam: float = 0.2, area_weight: bool = True, wrap_u: bool = True, want_grad: bool = True):
    dev = images[0].device
    lib = L.load()
    need = 16
    for im in images:
        n = C.c_size_t()
        L.check(lib.odgs_loss_scratch_size(int(im.shape[2]), int(im.shape[1]), C.byref(n)), "odgs_loss_scratch_size")
        need = max(need, int(n.value))
    scratch = torch.empty(need, dtype=torch.uint8, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)  # the first view writes it, the others add
    grads = []
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for k, (im, tg) in enumerate(zip(images, targets)):
        for t in (im, tg):
            if t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != 3 or t.shape[0] != 3 or t.device != dev:
                raise ValueError("images and targets must be contiguous float32 [3, H, W] tensors on one device")
        if im.shape != tg.shape:
            raise ValueError("image and target shapes differ")
        g = torch.empty_like(im) if want_grad else None
        prm = L.LossParams(float(lam), int(bool(area_weight)), int(bool(wrap_u)), int(k > 0))
        L.check(lib.odgs_loss_l1_dssim(_ptr(im), _ptr(tg), int(im.shape[2]), int(im.shape[1]), C.byref(prm), _ptr(g),
                                       _ptr(loss), _ptr(scratch), C.c_size_t(scratch.numel()), stream),
                "odgs_loss_l1_dssim")
        grads.append(g)
    return loss[0], grads
