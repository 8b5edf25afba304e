"""PyTorch-facing wrapper of the ODGS C ABI: device buffers, streams and autograd.

Every step of the rasterizer runs in the CUDA library (``libodgs.so``); this module only
allocates the caller-owned workspace / pair buffer as torch tensors, passes pointers and the
current stream, and exposes the forward and backward passes as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L


@dataclass
class RenderSettings:
    sh_degree: int = 3
    tile_w: int = 16
    tile_h: int = 16
    batch: int = 128  # forward staging batch (the backward stages at most 64)
    cov_dilation: float = 0.3
    r_near: float = 0.2
    r_far: float = 1e4
    bg: tuple = (0.0, 0.0, 0.0)
    recompute_lists: bool = False
    grad_accumulate: bool = False
    pixels_per_thread: int = 0      # forward blend (0: automatic, 2 where it fits)
    raw_params: bool = False  # scales are log-scales and opacity logits (activated by the kernels)
    pixels_per_thread_bwd: int = 0  # backward blend (0: automatic, 4 where it fits)
    checked: bool = False  # flag (ODGS_DEV_NONFINITE) and cull non-finite parameters / gradients
    full_lists: bool = False  # keep whole tile lists (default: cut after the tile saturates; same results)

    def c_struct(self, sh_coeffs: int) -> L.Settings:
        s = L.Settings()
        s.sh_degree, s.sh_coeffs = int(self.sh_degree), int(sh_coeffs)
        s.tile_w, s.tile_h, s.batch = int(self.tile_w), int(self.tile_h), int(self.batch)
        s.cov_dilation, s.r_near, s.r_far = float(self.cov_dilation), float(self.r_near), float(self.r_far)
        s.bg[:] = [float(b) for b in self.bg]
        s.recompute_lists = int(bool(self.recompute_lists))
        s.grad_accumulate = int(bool(self.grad_accumulate))
        s.pixels_per_thread = int(self.pixels_per_thread)
        s.raw_params = int(bool(self.raw_params))
        s.pixels_per_thread_bwd = int(self.pixels_per_thread_bwd)
        s.checked = int(bool(self.checked))
        s.full_lists = int(bool(self.full_lists))
        return s


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _views_array(views):
    arr = (L.View * len(views))()
    for i, v in enumerate(views):
        if isinstance(v, L.View):
            arr[i] = v
        else:
            arr[i] = L.make_view(v.width, v.height, v.R_wc, v.t_wc, getattr(v, "model", 0), getattr(v, "fx", 0.0),
                                 getattr(v, "fy", 0.0), getattr(v, "cx", 0.0), getattr(v, "cy", 0.0))
    return arr


class PairPool:
    """A pair buffer shared by several rasterizers whose tile lists need not coexist (with
    ``recompute_lists`` each backward pass rebuilds its lists), so a frame split into view groups
    needs pair memory for its largest group only."""

    def __init__(self, device=None):
        self.device = device
        self.tensor = None
        self.capacity = 0

    def reserve(self, lib, capacity: int, device):
        need = C.c_size_t()
        L.check(lib.odgs_pair_buffer_size(int(capacity), C.byref(need)), "odgs_pair_buffer_size")
        if self.tensor is None or self.tensor.numel() < need.value:
            self.tensor = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=device)
        self.capacity = max(self.capacity, int(capacity))


class Rasterizer:
    """One frame of state (a C ``odgs_ctx``) plus its device buffers.

    ``capacity_mode``: "query" reads the pair count back after the preprocess (one stream
    synchronisation) and grows the pair buffer when needed; "fixed" never synchronises and uses
    the pair buffer as sized so far (``reserve_pairs``), which CUDA-graph capture requires.
    """

    def __init__(self, device=None, capacity_mode: str = "query", headroom: float = 1.25, pairs: PairPool = None):
        self.lib = L.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            h = C.c_void_p()
            L.check(self.lib.odgs_create(C.byref(h)), "odgs_create")
        self.ctx = h
        self.capacity_mode = capacity_mode
        self.headroom = headroom
        self.ws = None
        self.pool = pairs if pairs is not None else PairPool(self.device)
        self.frame = 0
        self.n_views = 0
        self._keep = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None) and self.ctx.value:
                self.lib.odgs_destroy(self.ctx)
                self.ctx = C.c_void_p(0)
        except Exception:
            pass

    # ---------------------------------------------------------------- buffers
    def _ensure_workspace(self, n, views_c, nv, st_c):
        need = C.c_size_t()
        L.check(self.lib.odgs_workspace_size(int(n), views_c, nv, C.byref(st_c), C.byref(need)), "odgs_workspace_size")
        if self.ws is None or self.ws.numel() < need.value:
            self.ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=self.device)
        return int(need.value)

    def reserve_pairs(self, capacity: int):
        self.pool.reserve(self.lib, capacity, self.device)

    @property
    def capacity(self) -> int:
        return self.pool.capacity

    @property
    def pairs(self):
        return self.pool.tensor

    # ---------------------------------------------------------------- passes
    def preprocess(self, means, scales, quats, opacity, sh, views, settings: RenderSettings):
        means, scales, quats, opacity, sh = (t.contiguous() for t in (means, scales, quats, opacity, sh))
        for t in (means, scales, quats, opacity, sh):
            if not t.is_cuda or t.dtype != torch.float32:
                raise TypeError("Gaussian parameters must be float32 CUDA tensors")
        n = means.shape[0]
        sh_coeffs = sh.shape[1] if sh.dim() == 3 else 1
        st_c = settings.c_struct(sh_coeffs)
        views_c = _views_array(views)
        nv = len(views)
        self._ensure_workspace(n, views_c, nv, st_c)
        g = L.Gaussians(_ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity), _ptr(sh), int(n))
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_preprocess(self.ctx, C.byref(g), views_c, nv, C.byref(st_c), _ptr(self.ws),
                                         self.ws.numel(), stream), "odgs_preprocess")
        # the library keeps raw pointers until the backward pass
        self._keep = (means, scales, quats, opacity, sh)
        self._views_c = views_c
        self.n_views = nv
        self.views = list(views)
        self.settings = settings
        self.frame += 1
        return self._keep

    def query_pairs(self) -> int:
        p = C.c_size_t()
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        st = self.lib.odgs_query_pairs(self.ctx, C.byref(p), stream)
        # capacity and non-finite inputs are reported by status() and do not stop the frame
        if st not in (L.ODGS_OK, L.ODGS_ERR_CAPACITY, L.ODGS_ERR_NONFINITE):
            L.check(st, "odgs_query_pairs")
        return int(p.value)

    def bin_sort(self):
        if self.capacity_mode == "query":
            p = self.query_pairs()
            if p > self.capacity or self.pairs is None:
                self.reserve_pairs(max(int(p * self.headroom) + 1024, 1024))
        elif self.pairs is None:
            raise RuntimeError("fixed capacity mode: call reserve_pairs() first")
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_bin_sort(self.ctx, _ptr(self.pairs), self.capacity, stream), "odgs_bin_sort")

    def render_fwd(self, images=None, want_T=True):
        views = self.views
        if images is None:
            images = [torch.empty((3, v.height, v.width), dtype=torch.float32, device=self.device) for v in views]
        Ts = [torch.empty((v.height, v.width), dtype=torch.float32, device=self.device) for v in views] if want_T else None
        img_arr = (C.c_void_p * len(views))(*[im.data_ptr() for im in images])
        T_arr = (C.c_void_p * len(views))(*[t.data_ptr() for t in Ts]) if want_T else None
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_render_fwd(self.ctx, img_arr, T_arr, stream), "odgs_render_fwd")
        return images, Ts

    def render_bwd(self, grad_images):
        """Reverse blend: per-(view, Gaussian) screen-space gradients into the workspace."""
        gi = [g.contiguous() for g in grad_images]
        arr = (C.c_void_p * len(gi))(*[g.data_ptr() for g in gi])
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_render_bwd(self.ctx, arr, stream), "odgs_render_bwd")
        self._gi_keep = gi

    def preprocess_bwd(self, grads=None, densify=None):
        """Chain rule to the five parameter gradients (written, or added when grad_accumulate).
        densify: optional object with float32 ``grad``, ``elev`` and int32 ``count`` tensors [n]
        to which the frame's densification statistics are added (Sec. 3.3)."""
        means, scales, quats, opacity, sh = self._keep
        if grads is None:
            grads = dict(means=torch.empty_like(means), scales=torch.empty_like(scales),
                         quats=torch.empty_like(quats), opacity=torch.empty_like(opacity), sh=torch.empty_like(sh))
        gc = L.Grads(_ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"]), _ptr(grads["opacity"]),
                     _ptr(grads["sh"]))
        if densify is not None:
            n = means.shape[0]
            for name, dt in (("grad", torch.float32), ("elev", torch.float32), ("count", torch.int32)):
                t = getattr(densify, name)
                if t.dtype != dt or t.numel() != n or not t.is_contiguous() or t.device != means.device:
                    raise ValueError(f"densify.{name} must be a contiguous {dt} tensor of {n} elements on {means.device}")
            gc.densify_grad, gc.densify_elev, gc.densify_count = (_ptr(densify.grad), _ptr(densify.elev),
                                                                  _ptr(densify.count))
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_preprocess_bwd(self.ctx, C.byref(gc), stream), "odgs_preprocess_bwd")
        return grads

    def backward(self, grad_images, grads=None, densify=None):
        self.render_bwd(grad_images)
        return self.preprocess_bwd(grads, densify)

    def stats(self) -> dict:
        s = L.Stats()
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_frame_stats(self.ctx, C.byref(s), stream), "odgs_frame_stats")
        return dict(pairs=int(s.pairs), pairs_sorted=int(s.pairs_sorted), evals_fwd=int(s.evals_fwd),
                    evals_bwd=int(s.evals_bwd), blended=int(s.blended), entries_tile=int(s.entries_tile),
                    visible=int(s.visible), status=int(s.status))

    def status(self) -> int:
        bits = C.c_uint32()
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_get_status(self.ctx, C.byref(bits), stream), "odgs_get_status")
        return int(bits.value)

    def set_wait_limit(self, reads: int):
        """Bound of the sorts' look-back waits from the next bin_sort (0: give up at once)."""
        L.check(self.lib.odgs_set_wait_limit(self.ctx, int(reads)), "odgs_set_wait_limit")

    def debug_lists(self) -> dict:
        """Copies of the frame's depth order, tile-sorted pairs and tile ranges (uint32 tensors;
        synchronises the stream once to read the number of sorted pairs)."""
        n_items = int(self._keep[0].shape[0]) * self.n_views
        s = self.settings
        n_tiles = sum((v.width // s.tile_w) * ((v.height + s.tile_h - 1) // s.tile_h) for v in self.views)
        n_pairs = self.stats()["pairs_sorted"]
        u32 = dict(dtype=torch.int32, device=self.device)
        out = dict(depth_keys=torch.empty(n_items, **u32), depth_items=torch.empty(n_items, **u32),
                   pair_tiles=torch.empty(n_pairs, **u32), pair_items=torch.empty(n_pairs, **u32),
                   ranges=torch.empty((n_tiles, 2), **u32))
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_debug_lists(self.ctx, _ptr(out["depth_keys"]), _ptr(out["depth_items"]), n_items,
                                          _ptr(out["pair_tiles"]), _ptr(out["pair_items"]), n_pairs,
                                          _ptr(out["ranges"]), n_tiles, stream), "odgs_debug_lists")
        torch.cuda.current_stream(self.device).synchronize()
        return {k: v.cpu().numpy().view(np.uint32) for k, v in out.items()}

    def debug_screen_grads(self):
        """The last backward blend's per-(view, Gaussian) screen-space gradients, [views * n, 9]
        float32 (dL/du, dL/dv, dL/da, dL/db, dL/dc, dL/do, dL/dr, dL/dg, dL/db)."""
        n_items = int(self._keep[0].shape[0]) * self.n_views
        out = torch.empty((n_items, 12), dtype=torch.float32, device=self.device)
        stream = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        L.check(self.lib.odgs_debug_screen_grads(self.ctx, _ptr(out), n_items, stream), "odgs_debug_screen_grads")
        return out[:, :9].cpu().numpy()

    def launch_count(self) -> int:
        return int(self.lib.odgs_last_launch_count(self.ctx))

    def forward(self, means, scales, quats, opacity, sh, views, settings: RenderSettings, want_T=True):
        self.preprocess(means, scales, quats, opacity, sh, views, settings)
        self.bin_sort()
        return self.render_fwd(want_T=want_T)


class ODGSRender(torch.autograd.Function):
    """Differentiable ERP rendering of one frame (any number of views).

    forward(rasterizer, settings, views, means, scales, quats, opacity, sh) -> images (one
    [3, H, W] tensor per view). backward returns gradients for the five parameter tensors.
    """

    @staticmethod
    def forward(ctx, rast: Rasterizer, settings: RenderSettings, views, means, scales, quats, opacity, sh):
        images, _ = rast.forward(means, scales, quats, opacity, sh, views, settings, want_T=False)
        ctx.rast = rast
        ctx.frame = rast.frame
        ctx.save_for_backward(means, scales, quats, opacity, sh)
        return tuple(images)

    @staticmethod
    def backward(ctx, *grad_images):
        rast: Rasterizer = ctx.rast
        if rast.frame != ctx.frame:
            raise RuntimeError("ODGSRender: the rasterizer rendered another frame before this backward pass; "
                               "use one Rasterizer per pending frame")
        views = rast.views
        gi = [g if g is not None else torch.zeros((3, v.height, v.width), device=rast.device)
              for g, v in zip(grad_images, views)]
        g = rast.backward(gi)
        return None, None, None, g["means"], g["scales"], g["quats"], g["opacity"], g["sh"]


def render(means, scales, quats, opacity, sh, views, settings: RenderSettings = None, rasterizer: Rasterizer = None):
    """Render ``views`` of the Gaussians; differentiable w.r.t. the five parameter tensors."""
    settings = settings or RenderSettings()
    rast = rasterizer or Rasterizer(means.device)
    return ODGSRender.apply(rast, settings, list(views), means, scales, quats, opacity, sh)


def measure_peaks(device=None) -> dict:
    """FP32 FMA (TFLOP/s) and exp2f (G/s) throughput of the current device, by odgs_measure_peaks."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    lib = L.load()
    p = L.Peaks()
    with torch.cuda.device(dev):
        stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        L.check(lib.odgs_measure_peaks(C.byref(p), stream), "odgs_measure_peaks")
    return {"ffma_tflops": float(p.ffma_tflops), "ex2_gops": float(p.ex2_gops), "sms": int(p.sms)}
