"""Fused Adam over the five Gaussian parameter tensors (one kernel launch per step).

The learning rates default to the 3DGS recipe that ODGS trains with (App. A.1): positions
1.6e-4 x scene extent (the caller may decay it per step), SH DC 2.5e-3 and higher-order SH
2.5e-3 / 20, opacity 0.05, scaling 5e-3, rotation 1e-3; betas (0.9, 0.999), eps 1e-15. With
``RenderSettings(raw_params=True)`` the tensors are the raw variables 3DGS optimises
(log-scales, opacity logits, unnormalised quaternions) and the rasterizer's gradients are w.r.t.
them.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L

NAMES = ("means", "scales", "quats", "opacity", "sh")


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


class GaussianAdam:
    def __init__(self, params, scene_extent: float = 1.0, lr=None, betas=(0.9, 0.999), eps: float = 1e-15):
        self.params = list(params)
        for t in self.params:
            if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
                raise ValueError("parameters must be contiguous float32 CUDA tensors")
        self.lr = dict(means=1.6e-4 * scene_extent, sh_dc=2.5e-3, sh_rest=2.5e-3 / 20.0, opacity=0.05,
                       scales=5e-3, quats=1e-3)
        if lr:
            self.lr.update(lr)
        self.betas, self.eps = betas, eps
        self.m = [torch.zeros_like(t) for t in self.params]
        self.v = [torch.zeros_like(t) for t in self.params]
        self.t = 0

    def step(self, grads):
        """One Adam step with grads (dict by parameter name, or a list in NAMES order)."""
        g = [grads[k] for k in NAMES] if isinstance(grads, dict) else list(grads)
        self.t += 1
        groups = (L.AdamGroup * 5)()
        for k, (name, p, gr, m, v) in enumerate(zip(NAMES, self.params, g, self.m, self.v)):
            if gr.shape != p.shape or gr.dtype != torch.float32 or not gr.is_contiguous():
                raise ValueError(f"gradient of {name} must be a contiguous float32 tensor shaped like it")
            if name == "sh":  # [n, K, 3]: the first 3 floats of every row are the DC coefficients
                row, head, lr, lr_tail = 3 * p.shape[1], 3, self.lr["sh_dc"], self.lr["sh_rest"]
            else:
                row, head, lr, lr_tail = 1, 1, self.lr[name], self.lr[name]
            groups[k] = L.AdamGroup(_ptr(p).value, _ptr(gr).value, _ptr(m).value, _ptr(v).value, p.numel(),
                                    lr, lr_tail, row, head)
        prm = L.AdamParams(self.betas[0], self.betas[1], self.eps, self.t)
        stream = C.c_void_p(torch.cuda.current_stream(self.params[0].device).cuda_stream)
        L.check(L.load().odgs_adam_step(groups, 5, C.byref(prm), stream), "odgs_adam_step")
