"""One fwd+bwd frame over many ERP views, captured once into a CUDA graph and replayed.

A frame renders all its views in one persistent launch per blend direction (global (view, tile)
work queue), sorts all views' items together, and sums every view's gradient into one set of
parameter-gradient buffers. ``GraphedFrame`` sizes the caller-owned buffers with one eager run,
switches the rasterizer to fixed pair capacity (no host synchronisation), and captures

    preprocess -> bin_sort -> render_fwd -> loss (torch) -> render_bwd -> preprocess_bwd

into a ``torch.cuda.CUDAGraph``. ``replay()`` then re-runs the frame on whatever the parameter
tensors hold at that time (same shapes, same device addresses).
"""
from __future__ import annotations

import torch

from .rasterizer import Rasterizer, RenderSettings

_GRAD_NAMES = ("means", "scales", "quats", "opacity", "sh")


def l1_grad(images, targets):
    """sum_v mean |I_v - T_v| and its gradient w.r.t. each image, sign(I - T) / (3 W H), by the
    fused loss kernel (L1 term alone, unweighted)."""
    from .loss import l1_dssim
    return l1_dssim(images, targets, lam=0.0, area_weight=False, wrap_u=True)


class GraphedFrame:
    """Fixed-shape fwd+bwd frame of ``views`` replayed from a CUDA graph.

    params: [means, scales, quats, opacity, sh] device tensors (read at every replay).
    targets: one [3, H, W] device tensor per view. Gradients land in ``self.grads``; the loss of
    the last replay in ``self.loss``.
    """

    def __init__(self, params, views, targets, settings: RenderSettings = None, headroom: float = 1.3,
                 loss_fn=l1_grad):
        self.params = list(params)
        self.views = list(views)
        self.targets = list(targets)
        self.settings = settings or RenderSettings()
        self.loss_fn = loss_fn
        dev = self.params[0].device
        self.rast = Rasterizer(dev, capacity_mode="query", headroom=headroom)
        self.grads = {k: torch.empty_like(t) for k, t in zip(_GRAD_NAMES, self.params)}
        # eager run: sizes the workspace and the pair buffer, loads every kernel
        self._step()
        torch.cuda.synchronize(dev)
        st = self.rast.status()
        if st != 0:
            raise RuntimeError(f"device status {st} during the sizing run")
        self.rast.capacity_mode = "fixed"
        self.launches = self.rast.launch_count()
        # warm up on a side stream, then capture
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            self._step()
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.loss = self._step()

    def _step(self):
        r = self.rast
        r.preprocess(*self.params, self.views, self.settings)
        r.bin_sort()
        images, _ = r.render_fwd(want_T=False)
        loss, gi = self.loss_fn(images, self.targets)
        r.render_bwd(gi)
        r.preprocess_bwd(self.grads)
        self.images = images
        return loss

    def replay(self):
        self.graph.replay()
        return self.loss

    def status(self) -> int:
        """Device status bits of the last replay (synchronises)."""
        return self.rast.status()


class GroupedFrame:
    """One fwd+bwd frame whose views are rendered in groups that share one pair buffer.

    Each group's tile lists are rebuilt in its backward pass (``recompute_lists``), so the pair
    buffer only has to hold the largest group's lists, not the whole frame's. Gradients of all
    groups are summed into ``self.grads``. Runs eagerly (no graph).
    """

    def __init__(self, params, views, targets, settings: RenderSettings = None, group_size: int = 1,
                 headroom: float = 1.3, loss_fn=l1_grad):
        from dataclasses import replace
        from .rasterizer import PairPool
        self.params = list(params)
        self.views = list(views)
        self.targets = list(targets)
        base = settings or RenderSettings()
        self.loss_fn = loss_fn
        dev = self.params[0].device
        self.groups = [self.views[i:i + group_size] for i in range(0, len(self.views), group_size)]
        self.settings = [replace(base, recompute_lists=True, grad_accumulate=(i > 0)) for i in range(len(self.groups))]
        self.pool = PairPool(dev)
        self.rasts = [Rasterizer(dev, capacity_mode="fixed", pairs=self.pool) for _ in self.groups]
        self.grads = {k: torch.empty_like(t) for k, t in zip(_GRAD_NAMES, self.params)}
        # size the shared pair buffer for the largest group (one synchronising query per group)
        need = 0
        for r, vs, st in zip(self.rasts, self.groups, self.settings):
            r.preprocess(*self.params, vs, st)
            need = max(need, r.query_pairs())
        for r in self.rasts:
            r.reserve_pairs(int(need * headroom) + 1024)

    def step(self):
        images = []
        for r, vs, st in zip(self.rasts, self.groups, self.settings):
            imgs, _ = r.forward(*self.params, vs, st, want_T=False)
            images += imgs
        loss, gi = self.loss_fn(images, self.targets)
        k = 0
        for r, vs in zip(self.rasts, self.groups):
            r.backward(gi[k:k + len(vs)], self.grads)
            k += len(vs)
        self.images = images
        return loss

    def status(self) -> int:
        bits = 0
        for r in self.rasts:
            bits |= r.status()
        return bits

    def pair_buffer_bytes(self) -> int:
        return int(self.pool.tensor.numel()) if self.pool.tensor is not None else 0
