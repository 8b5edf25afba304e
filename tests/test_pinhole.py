"""Pinhole (perspective) views through the same sort and blend kernels: parity with the oracle's
pinhole model, cube faces and mixed ERP / pinhole frames, tile invariance, and the tangent-point
agreement with the ERP model (P2)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import EPS_CLAMP, EPS_SKIP, EPS_TERM, assert_grads_close, compare_image, oracle_settings, to_torch

pytestmark = pytest.mark.gpu
NAMES = ("means", "scales", "quats", "opacity", "sh")


def _rs(**kw):
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    return RenderSettings(**kw)


def _scene_with(views, n=1500, seed=31):
    sc = S.random_scene(n, 64, 32, seed=seed, sh_degree=3, radius=(1.0, 6.0), log_scale=(-3.2, 0.5))
    sc.views = list(views)
    return sc


def _posed_pinhole():
    R = Rotation.from_euler("xyz", [0.15, -0.4, 0.1]).as_matrix().astype(np.float32)
    return S.pinhole_view(256, 192, 160.0, 150.0, 130.0, 90.0, R, [0.1, -0.05, 0.2])


def test_pinhole_forward_and_backward_match_the_oracle():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sc = _scene_with([_posed_pinhole()])
    rs = _rs(sh_degree=3)
    v = sc.views[0]
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    col, _, _, margins = O.render(p, v, st)
    rast = Rasterizer()
    params = to_torch(sc)
    out, _ = rast.forward(*params, [v], rs, want_T=False)
    compare_image(out[0].cpu().numpy().astype(np.float64), col, margins)
    amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
    w = np.random.default_rng(4).normal(size=(3, v.height, v.width)) * (~amb)[None]
    g = rast.backward([torch.tensor(w, dtype=torch.float32, device="cuda")])
    torch.cuda.synchronize()
    assert rast.status() == 0
    ref = O.backward(p, v, st, w)
    assert_grads_close({k: g[k].cpu().numpy().astype(np.float64) for k in NAMES}, ref, NAMES)


def test_cubemap_faces_in_one_frame():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sc = _scene_with(S.cubemap_views(96, center=(0.05, -0.02, 0.03)), n=2000, seed=32)
    rs = _rs(sh_degree=3)
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    rast = Rasterizer()
    imgs, _ = rast.forward(*to_torch(sc), sc.views, rs, want_T=False)
    torch.cuda.synchronize()
    assert rast.status() == 0
    for v, im in zip(sc.views, imgs):
        col, _, _, margins = O.render(p, v, st)
        compare_image(im.cpu().numpy().astype(np.float64), col, margins)


def test_mixed_erp_and_pinhole_views_in_one_frame():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    views = [S.View.identity(256, 128), _posed_pinhole(), S.yaw_view(128, 64, (0.0, 0.1, 0.0), 0.7)]
    sc = _scene_with(views, n=1200, seed=33)
    rs = _rs(sh_degree=3)
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    rast = Rasterizer()
    imgs, _ = rast.forward(*to_torch(sc), sc.views, rs, want_T=False)
    ws = []
    for v, im in zip(sc.views, imgs):
        col, _, _, margins = O.render(p, v, st)
        compare_image(im.cpu().numpy().astype(np.float64), col, margins)
        amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
        ws.append(np.random.default_rng(v.width).normal(size=(3, v.height, v.width)) * (~amb)[None])
    g = rast.backward([torch.tensor(w, dtype=torch.float32, device="cuda") for w in ws])
    torch.cuda.synchronize()
    ref = None
    for v, w in zip(sc.views, ws):
        r = O.backward(p, v, st, w)
        ref = r if ref is None else {k: ref[k] + r[k] for k in NAMES}
    assert_grads_close({k: g[k].cpu().numpy().astype(np.float64) for k in NAMES}, ref, NAMES)


def test_pinhole_images_do_not_depend_on_the_tiling():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sc = _scene_with([_posed_pinhole()])
    base = None
    for tw, th, b in [(16, 16, 64), (32, 8, 32), (8, 16, 128)]:
        rast = Rasterizer()
        imgs, _ = rast.forward(*to_torch(sc), sc.views, _rs(sh_degree=3, tile_w=tw, tile_h=th, batch=b), want_T=False)
        torch.cuda.synchronize()
        im = imgs[0].cpu().numpy()
        if base is None:
            base = im
        else:
            np.testing.assert_array_equal(im, base)


def test_p2_erp_and_pinhole_agree_at_the_tangent_point_on_the_gpu():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    W, H = 256, 128
    rgb = np.array([0.8, 0.3, 0.55], np.float32)
    sc = S.Scene(np.array([[0.0, 0.0, 2.0]], np.float32), np.full((1, 3), 0.02, np.float32),
                 np.array([[0.9, 0.1, -0.3, 0.2]], np.float32), np.array([0.85], np.float32),
                 ((rgb - 0.5) * 2 * np.sqrt(np.pi)).reshape(1, 1, 3).astype(np.float32), 0)
    rs = _rs(sh_degree=0)
    erp, _ = Rasterizer().forward(*to_torch(sc), [S.View.identity(W, H)], rs, want_T=False)
    pin, _ = Rasterizer().forward(*to_torch(sc), [S.pinhole_view(W, H, W / (2 * np.pi), H / np.pi)], rs,
                                  want_T=False)
    torch.cuda.synchronize()
    np.testing.assert_allclose(pin[0].cpu().numpy(), erp[0].cpu().numpy(), atol=1e-5)
    assert float((erp[0] > 0).sum()) > 12
