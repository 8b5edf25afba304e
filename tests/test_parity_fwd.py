"""GPU forward parity: the CUDA rasterizer (through the C ABI) against the FP64 oracle.

Images must agree within 1e-4 max-abs per channel on every pixel whose discrete decisions
(alpha >= 1/255, T >= 1e-4) are not within rounding of their thresholds; such ambiguous pixels
are counted and bounded.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import compare_image, gpu_render, oracle_settings

pytestmark = pytest.mark.gpu


def _rs(**kw):
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    return RenderSettings(**kw)


def _check_full(scene, rs, views=None):
    views = scene.views if views is None else views
    imgs, Ts, _ = gpu_render(scene, rs, views)
    p = O.Params.of(scene)
    st = oracle_settings(rs)
    out = []
    for v, im, T in zip(views, imgs, Ts):
        ref, Tref, nc, margins = O.render(p, v, st)
        out.append(compare_image(im, ref, margins))
        amb = O.ambiguous(margins, 2e-5, 1e-4)
        assert np.abs(T - Tref)[~amb].max() <= 1e-4
    return out


def test_config0_full_image():
    sc = S.config0()
    err, frac = _check_full(sc, _rs(sh_degree=0))[0]
    assert err < 1e-5


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_random_scene_ragged_tiles_and_pose(deg):
    view = S.yaw_view(208, 100, center=(0.3, -0.2, 0.1), yaw=0.7)
    sc = S.random_scene(3000, 208, 100, seed=10 + deg, sh_degree=deg, views=[view])
    _check_full(sc, _rs(sh_degree=deg, bg=(0.2, 0.5, 0.1)))


def test_general_rotation_pose():
    from scipy.spatial.transform import Rotation
    R = Rotation.from_euler("xyz", [0.4, -1.1, 0.25]).as_matrix()
    c = np.array([0.5, 0.3, -0.4])
    view = S.View(320, 160, R.astype(np.float32), (-R @ c).astype(np.float32))
    sc = S.random_scene(2500, 320, 160, seed=21, sh_degree=3, views=[view])
    _check_full(sc, _rs(sh_degree=3))


def test_multiple_views_in_one_launch():
    views = [S.View.identity(128, 64), S.yaw_view(256, 128, (0.2, 0, 0), 2.0), S.yaw_view(64, 40, (0, 0.1, 0), -1.0)]
    sc = S.random_scene(1500, 128, 64, seed=31, sh_degree=2, views=views)
    _check_full(sc, _rs(sh_degree=2))


def test_seam_and_pole_stress():
    """Gaussians on the +-180 deg seam and within a few degrees of both poles, including
    pole-stretched ones wider than half the image (seam split inside a tile)."""
    rng = np.random.default_rng(5)
    n = 600
    W, H = 256, 128
    r = rng.uniform(1.0, 4.0, n)
    phi = np.where(rng.uniform(size=n) < 0.5, np.pi - rng.uniform(0, 0.05, n), -np.pi + rng.uniform(0, 0.05, n))
    theta = rng.uniform(-0.3, 0.3, n)
    k = n // 3
    theta[:k] = np.sign(rng.normal(size=k)) * (np.pi / 2 - rng.uniform(0.001, 0.08, k))
    phi[:k] = rng.uniform(-np.pi, np.pi, k)
    t = np.stack([r * np.cos(theta) * np.sin(phi), -r * np.sin(theta), r * np.cos(theta) * np.cos(phi)], 1)
    sc = S.random_scene(n, W, H, seed=41, sh_degree=1)
    sc.means[:] = t.astype(np.float32)
    sc.scales[:] = np.exp(rng.normal(-2.5, 0.4, size=(n, 3))).astype(np.float32)
    _check_full(sc, _rs(sh_degree=1))


def test_huge_gaussian_covers_all_columns():
    sc = S.random_scene(50, 128, 64, seed=51, sh_degree=0)
    sc.means[0] = [0.1, -0.25, 0.05]
    sc.scales[0] = [0.3, 0.2, 0.25]
    sc.opacity[0] = 0.9
    _check_full(sc, _rs(sh_degree=0))


def test_empty_scene_and_all_culled_give_background():
    from paper_2410_20686_gb300.scenes import Scene
    bg = (0.25, 0.5, 0.75)
    empty = Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                  np.zeros((0,), np.float32), np.zeros((0, 1, 3), np.float32), 0, [S.View.identity(64, 32)])
    imgs, Ts, _ = gpu_render(empty, _rs(sh_degree=0, bg=bg))
    assert np.allclose(imgs[0], np.asarray(bg, np.float32)[:, None, None]) and np.all(Ts[0] == 1.0)
    far = S.random_scene(100, 64, 32, seed=3, sh_degree=0, radius=(2e4, 3e4))
    imgs, Ts, _ = gpu_render(far, _rs(sh_degree=0, bg=bg))
    assert np.allclose(imgs[0], np.asarray(bg, np.float32)[:, None, None])


def test_tiling_and_batch_are_invisible_bitwise():
    """P8: per-pixel results do not depend on the tile shape or the batch size."""
    view = S.yaw_view(256, 120, (0.1, 0.0, -0.1), 0.3)
    sc = S.random_scene(4000, 256, 120, seed=61, sh_degree=3, views=[view], log_scale=(-2.8, 0.6))
    base, bT, _ = gpu_render(sc, _rs(sh_degree=3))
    for tw, th, b in [(8, 8, 32), (32, 8, 64), (16, 32, 256), (8, 16, 17), (32, 32, 128), (16, 16, 1)]:
        imgs, Ts, _ = gpu_render(sc, _rs(sh_degree=3, tile_w=tw, tile_h=th, batch=b))
        assert np.array_equal(imgs[0], base[0]), (tw, th, b)
        assert np.array_equal(Ts[0], bT[0]), (tw, th, b)


def test_yaw_quarter_turn_rolls_the_image():
    """P4 on the GPU: a yaw of exactly 90 deg (rotation entries 0 and +-1) moves every Gaussian
    by W/4 columns; the image rolls accordingly."""
    W, H = 256, 128
    sc = S.random_scene(2000, W, H, seed=71, sh_degree=2)
    R_cw = np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], np.float32)  # yaw = +90 deg
    base, _, _ = gpu_render(sc, _rs(sh_degree=2))
    rot, _, _ = gpu_render(sc, _rs(sh_degree=2), views=[S.View(W, H, R_cw.T.copy(), np.zeros(3, np.float32))])
    assert np.abs(rot[0] - np.roll(base[0], -W // 4, axis=2)).max() < 1e-5


def test_config1_sampled_pixels():
    sc = S.config1()
    rs = _rs(sh_degree=3)
    imgs, _, _ = gpu_render(sc, rs)
    v = sc.views[0]
    pix = S.sample_pixels(v.width, v.height, 2048, S.stress_tiles(v.width, v.height), seed=1)
    col, T, nc, margins = O.render(O.Params.of(sc), v, oracle_settings(rs), pix=pix)
    gpu = imgs[0].reshape(3, -1)[:, pix].T
    compare_image(gpu, col, margins)


@pytest.mark.slow
def test_config2_sampled_pixels():
    sc = S.config2()
    rs = _rs(sh_degree=3)
    imgs, _, _ = gpu_render(sc, rs)
    v = sc.views[0]
    pix = S.sample_pixels(v.width, v.height, 1024, S.stress_tiles(v.width, v.height)[:4], seed=2)
    col, T, nc, margins = O.render(O.Params.of(sc), v, oracle_settings(rs), pix=pix)
    gpu = imgs[0].reshape(3, -1)[:, pix].T
    compare_image(gpu, col, margins)


def test_largest_view_16384x8192():
    """The largest supported view: pixel anchors up to 16383 in their 16-bit fields and 524,288
    tiles. Sampled pixels: random ones, the seam and pole tiles, and the tiles holding the first
    Gaussians' centres."""
    sc = S.random_scene(5000, 16384, 8192, seed=23, sh_degree=1, radius=(0.5, 3.0), log_scale=(-3.0, 0.5))
    rs = _rs(sh_degree=1)
    imgs, _, _ = gpu_render(sc, rs, want_T=False)
    v = sc.views[0]
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    pj = O.project(p, v, st)
    vis = pj[:, O.PJ_VALID] > 0
    centres = [(int(u) // 16, int(w) // 16) for u, w in pj[vis][:12, [O.PJ_U, O.PJ_V]]]
    pix = S.sample_pixels(v.width, v.height, 4096, S.stress_tiles(v.width, v.height) + centres, seed=24)
    col, T, nc, margins = O.render(p, v, st, pix=pix)
    gpu = imgs[0].reshape(3, -1)[:, pix].T
    compare_image(gpu, col, margins)
    assert (nc > 0).sum() > 1000  # the sample reaches many covered pixels, not only background
