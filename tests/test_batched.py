"""Many-view frames: one persistent launch per blend direction, CUDA-graph replay, gradients of
all views summed into one buffer; and the autotuner."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import compare_image, oracle_settings, rel_l2

NAMES = ("means", "scales", "quats", "opacity", "sh")


def test_autotune_candidates_pass_the_library_validation():
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300 import autotune as A
    from paper_2410_20686_gb300 import build as B
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    B.build()
    lib = L.load()
    widths = [512, 1024, 2048]
    views = (L.View * 3)(*[L.make_view(w, w // 2, np.eye(3), np.zeros(3)) for w in widths])
    cands = A.candidates(widths, tiles=((16, 16), (16, 8), (32, 8), (8, 8), (32, 16), (16, 32), (8, 4), (32, 32)),
                         ppts=(1, 2, 4))
    assert len(cands) > 20
    for tw, th, b, pf, pb in cands:
        st = RenderSettings(tile_w=tw, tile_h=th, batch=b, pixels_per_thread=pf, pixels_per_thread_bwd=pb).c_struct(16)
        out = C.c_size_t()
        assert lib.odgs_workspace_size(1000, views, 3, C.byref(st), C.byref(out)) == 0, (tw, th, b, pf, pb)
    # and a shape the tuner rejects is rejected by the library too
    st = RenderSettings(tile_w=32, tile_h=32, pixels_per_thread=1).c_struct(16)
    assert not A.valid(32, 32, 1, widths)
    assert lib.odgs_workspace_size(1000, views, 3, C.byref(st), C.byref(C.c_size_t())) == -1


def _scene():
    sizes = [(128, 64), (128, 64), (256, 128), (64, 32)]
    views = [S.yaw_view(w, h, (0.3 * i - 0.4, 0.05 * i, 0.1), 1.1 * i - 1.5) for i, (w, h) in enumerate(sizes)]
    return S.random_scene(3000, 128, 64, seed=301, sh_degree=3, views=views, log_scale=(-2.6, 0.5))


@pytest.mark.gpu
def test_graphed_frame_matches_eager_and_oracle():
    import torch
    from paper_2410_20686_gb300.graph import GraphedFrame
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = _scene()
    rs = RenderSettings(sh_degree=3)
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    targets = [torch.tensor(t, device="cuda") for t in S.target_images(sc, 3)]
    gf = GraphedFrame(params, sc.views, targets, rs)
    gf.replay()
    torch.cuda.synchronize()
    assert gf.status() == 0
    g1 = {k: v.clone() for k, v in gf.grads.items()}
    imgs1 = [im.clone() for im in gf.images]
    # eager reference through the same library
    rast = Rasterizer()
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    gi = [torch.sign(im - tg) / im.numel() for im, tg in zip(imgs, targets)]
    ge = rast.backward(gi)
    for a, b in zip(imgs1, imgs):
        assert torch.equal(a, b)
    for k in NAMES:
        assert rel_l2(g1[k].cpu().numpy(), ge[k].cpu().numpy()) < 1e-6, k
    # replaying after the parameters change renders the new parameters
    with torch.no_grad():
        params[0].add_(0.01)
    gf.replay()
    torch.cuda.synchronize()
    imgs2, _ = rast.forward(*params, sc.views, rs, want_T=False)
    for a, b in zip(gf.images, imgs2):
        assert torch.equal(a, b)
    # and the images agree with the oracle view by view
    with torch.no_grad():
        params[0].sub_(0.01)
    gf.replay()
    torch.cuda.synchronize()
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    for v, im in zip(sc.views, gf.images):
        ref, _, _, margins = O.render(p, v, st)
        compare_image(im.cpu().numpy().astype(np.float64), ref, margins)


@pytest.mark.gpu
def test_autotune_picks_and_caches(tmp_path):
    import torch
    from paper_2410_20686_gb300 import autotune as A
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    sc = S.random_scene(2000, 256, 128, seed=303, sh_degree=1)
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    cache = str(tmp_path / "tune.json")
    cands = [(16, 16, 64, 4, 4), (16, 8, 32, 2, 4), (32, 8, 64, 4, 2), (16, 16, 64, 2, 4)]
    rs = A.autotune(params, sc.views, RenderSettings(sh_degree=1), cache_path=cache, iters=2, cands=cands)
    assert (rs.tile_w, rs.tile_h, rs.batch, rs.pixels_per_thread, rs.pixels_per_thread_bwd) in cands
    again = A.autotune(params, sc.views, RenderSettings(sh_degree=1), cache_path=cache, cands=[(8, 8, 32, 2, 2)])
    assert (again.tile_w, again.tile_h) == (rs.tile_w, rs.tile_h)  # served from the cache


@pytest.mark.gpu
@pytest.mark.parametrize("group", [1, 2])
def test_grouped_frame_with_recomputed_lists_matches_one_frame(group):
    import torch
    from paper_2410_20686_gb300.graph import GroupedFrame, l1_grad
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = _scene()
    rs = RenderSettings(sh_degree=3)
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    targets = [torch.tensor(t, device="cuda") for t in S.target_images(sc, 3)]
    gfr = GroupedFrame(params, sc.views, targets, rs, group_size=group)
    gfr.step()
    torch.cuda.synchronize()
    assert gfr.status() == 0
    rast = Rasterizer()
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    _, gi = l1_grad(imgs, targets)
    ge = rast.backward(gi)
    for a, b in zip(gfr.images, imgs):
        assert torch.equal(a, b)
    for k in NAMES:
        assert rel_l2(gfr.grads[k].cpu().numpy(), ge[k].cpu().numpy()) < 1e-6, k
    # the shared pair buffer holds one group's lists, not the frame's
    assert gfr.pair_buffer_bytes() < rast.pairs.numel()
