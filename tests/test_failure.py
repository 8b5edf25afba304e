"""Failure reporting without a GPU fault.

1. A frame with more (tile, Gaussian) pairs than the pair buffer holds: the device clips the
   emission at the capacity, sets ODGS_DEV_CAPACITY in the status word, and every later kernel
   works on the clipped lists (nothing is written out of bounds); the host learns of it from the
   status, and a following frame with enough capacity is exact again.
2. A sort whose bounded look-back wait runs out (the bound set to 0 reads, so that it gives up at
   once rather than after a hang): ODGS_DEV_TIMEOUT, finite results, and recovery."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import compare_image, oracle_settings, to_torch

pytestmark = pytest.mark.gpu


def test_pair_capacity_overflow_is_reported_and_the_next_frame_recovers():
    import torch
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = S.random_scene(2000, 256, 128, seed=41, sh_degree=1, radius=(1.0, 5.0))
    rs = RenderSettings(sh_degree=1, full_lists=True)  # every pair of the footprints is emitted
    params = to_torch(sc)
    probe = Rasterizer()
    probe.forward(*params, sc.views, rs, want_T=False)
    needed = probe.stats()["pairs"]
    cap = needed // 4  # a quarter of what the frame needs
    rast = Rasterizer(capacity_mode="fixed")
    rast.reserve_pairs(cap)
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    g = rast.backward([torch.ones_like(imgs[0])])
    torch.cuda.synchronize()
    assert rast.status() & L.DEV_CAPACITY
    assert rast.stats()["pairs"] == needed and rast.stats()["pairs_sorted"] == cap
    assert torch.isfinite(imgs[0]).all() and all(torch.isfinite(t).all() for t in g.values())
    # the same rasterizer with enough room: the status clears and the image is the oracle's
    rast.reserve_pairs(needed + 1024)
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    torch.cuda.synchronize()
    assert rast.status() == 0
    p = O.Params.of(sc)
    col, _, _, margins = O.render(p, sc.views[0], oracle_settings(rs))
    compare_image(imgs[0].cpu().numpy().astype(np.float64), col, margins)


def test_query_mode_grows_the_pair_buffer_instead():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = S.random_scene(2000, 256, 128, seed=42, sh_degree=1, radius=(1.0, 5.0))
    rast = Rasterizer(capacity_mode="query")
    rast.reserve_pairs(1024)
    rast.forward(*to_torch(sc), sc.views, RenderSettings(sh_degree=1), want_T=False)
    torch.cuda.synchronize()
    assert rast.status() == 0 and rast.capacity >= rast.stats()["pairs"]


def test_sort_that_gives_up_is_reported_and_the_next_frame_recovers():
    """A look-back wait bound of 0 makes every sort CTA after the first give up at once (no GPU
    fault, no hang): the frame reports ODGS_ERR_TIMEOUT, its images and gradients are finite (every
    index read after the sort is bounded), and the next frame at the default bound is exact."""
    import ctypes as C

    import torch
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = S.random_scene(6000, 256, 128, seed=44, sh_degree=1, radius=(1.0, 5.0))  # 3 depth-sort tiles
    rs = RenderSettings(sh_degree=1)
    params = to_torch(sc)
    rast = Rasterizer()
    rast.reserve_pairs(4 << 20)
    rast.set_wait_limit(0)
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    g = rast.backward([torch.ones_like(imgs[0])])
    torch.cuda.synchronize()
    assert rast.status() & L.DEV_TIMEOUT
    pairs = C.c_size_t()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert rast.lib.odgs_query_pairs(rast.ctx, C.byref(pairs), stream) == L.ODGS_ERR_TIMEOUT
    assert torch.isfinite(imgs[0]).all() and all(torch.isfinite(t).all() for t in g.values())
    rast.set_wait_limit(1 << 22)
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    torch.cuda.synchronize()
    assert rast.status() == 0
    p = O.Params.of(sc)
    col, _, _, margins = O.render(p, sc.views[0], oracle_settings(rs))
    compare_image(imgs[0].cpu().numpy().astype(np.float64), col, margins)
