"""Tile lists cut at saturated tiles (the default; full_lists = 0).

A tile's list ends after the depth bucket in which a lower bound of its Gaussians' coverage (alpha
at the tile's corner pixels, summed as -log2(1 - alpha) in depth order) proves that every pixel
of the tile has stopped: the blend of Eq. 3 never reaches the entries after it. Checked against
the whole lists of the same frame (full_lists = 1), which tests/test_lists_exact.py checks against
the oracle: images and final T bit for bit, gradients up to the order of the atomic sums, every
cut list a prefix of the whole one, and the cut actually taken on part of the tiles. The scenes
put near, large, nearly opaque Gaussians over one side of the sphere (some across the longitude
seam) in front of many small ones, so that tiles saturate on that side and not on the other.
"""
import numpy as np
import pytest

from paper_2410_20686_gb300 import scenes as S
from tests.helpers import rel_l2, to_torch

pytestmark = pytest.mark.gpu
NAMES = ("means", "scales", "quats", "opacity", "sh")


def _scene(n_near, n_far, width, height, seed, views=None):
    sc = S.random_scene(n_near + n_far, width, height, seed=seed, sh_degree=1, radius=(3.0, 8.0),
                        log_scale=(-2.6, 0.4), views=views)
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_near, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[:, 0] = np.abs(d[:, 0])  # x > 0: the right half of an identity-pose ERP view
    d[: n_near // 8, 2] = -np.abs(d[: n_near // 8, 2])  # an eighth towards -z: across the seam
    sc.means[:n_near] = (d * rng.uniform(1.0, 1.6, (n_near, 1))).astype(np.float32)
    sc.scales[:n_near] = np.exp(rng.normal(-0.8, 0.2, (n_near, 3))).astype(np.float32)
    sc.opacity[:n_near] = 0.97
    return sc


def _run(sc, rs, weights, lists_after_backward=False):
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    rast = Rasterizer()
    imgs, Ts = rast.forward(*to_torch(sc), sc.views, rs, want_T=True)
    lists = None if lists_after_backward else rast.debug_lists()
    stats = rast.stats()
    g = rast.backward([torch.tensor(w, dtype=torch.float32, device="cuda") for w in weights])
    torch.cuda.synchronize()
    assert rast.status() == 0
    if lists_after_backward:
        lists = rast.debug_lists()
    return ([i.cpu().numpy() for i in imgs], [t.cpu().numpy() for t in Ts], lists, stats,
            {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()})


def _compare(sc, **kw):
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    rng = np.random.default_rng(11)
    weights = [rng.normal(size=(3, v.height, v.width)) for v in sc.views]
    full = _run(sc, RenderSettings(sh_degree=1, full_lists=True, **kw), weights)
    cut = _run(sc, RenderSettings(sh_degree=1, **kw), weights)
    for a, b in zip(full[0] + full[1], cut[0] + cut[1]):
        assert np.array_equal(a, b), np.abs(a - b).max()
    fl, cl = full[2], cut[2]
    assert cut[3]["pairs"] == full[3]["pairs"] and cut[3]["pairs_sorted"] < 0.8 * full[3]["pairs_sorted"]
    fr, cr = fl["ranges"].astype(np.int64), cl["ranges"].astype(np.int64)
    flen, clen = fr[:, 1] - fr[:, 0], cr[:, 1] - cr[:, 0]
    assert (clen <= flen).all() and clen.sum() == cut[3]["pairs_sorted"]
    for t in np.nonzero(flen)[0]:
        a, b = fr[t, 0], cr[t, 0]
        assert np.array_equal(cl["pair_items"][b:b + clen[t]], fl["pair_items"][a:a + clen[t]]), t
        assert (cl["pair_tiles"][b:b + clen[t]] == t).all()
    # the cut is taken on part of the tiles only
    assert (clen < flen).sum() > 0 and ((clen == flen) & (flen > 0)).sum() > 0
    for k in NAMES:
        assert rel_l2(cut[4][k], full[4][k]) < 1e-6, k
    return full, cut


def test_cut_lists_give_the_whole_lists_results_erp():
    _compare(_scene(1200, 8000, 256, 128, seed=5))


def test_cut_lists_give_the_whole_lists_results_multiview_with_pinhole():
    views = [S.View.identity(512, 256), S.yaw_view(256, 128, (0.1, -0.05, 0.2), 2.4),
             S.pinhole_view(240, 160, 150.0, 150.0, 119.5, 80.0, R_wc=np.asarray(S.yaw_view(8, 4, (0, 0, 0), -1.2).R_wc),
                            t_wc=np.zeros(3, np.float32))]
    _compare(_scene(1500, 12000, 512, 256, seed=7, views=views))


def test_cut_lists_other_tile_shape_and_rebuilt_lists():
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    sc = _scene(1000, 6000, 256, 128, seed=9)
    _, cut = _compare(sc, tile_w=32, tile_h=8)
    # the lists rebuilt for the backward pass are the same cut lists, and so are the gradients
    weights = [np.random.default_rng(11).normal(size=(3, v.height, v.width)) for v in sc.views]
    rs = RenderSettings(sh_degree=1, tile_w=32, tile_h=8, recompute_lists=True)
    _, _, again, _, g = _run(sc, rs, weights, lists_after_backward=True)
    for k in cut[2]:
        assert np.array_equal(cut[2][k], again[k]), k
    for k in NAMES:
        assert rel_l2(g[k], cut[4][k]) < 1e-6, k


def test_cut_lists_ragged_rows_and_a_tile_height_of_six():
    # tiles of 16 x 6 pixels (a tile height that is no power of two) on a 256 x 130 view, whose
    # last tile row has 4 pixel rows: the coverage bound takes the tile's last pixel row, not a
    # row past the image
    _compare(_scene(1200, 8000, 256, 130, seed=13), tile_w=16, tile_h=6)


def test_cut_lists_on_the_1m_gaussian_frame():
    # the bench's frame, whose polar tiles saturate after a few hundred of their ~10K entries:
    # images and T bit for bit, gradients up to the order of the atomic sums, and the cut lists
    # prefixes of the whole ones on the pole and seam tiles and 64 random tiles
    sc = S.config2()
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    rng = np.random.default_rng(21)
    weights = [rng.normal(size=(3, v.height, v.width)) for v in sc.views]
    full = _run(sc, RenderSettings(sh_degree=3, full_lists=True), weights)
    cut = _run(sc, RenderSettings(sh_degree=3), weights)
    for a, b in zip(full[0] + full[1], cut[0] + cut[1]):
        assert np.array_equal(a, b), np.abs(a - b).max()
    assert cut[3]["pairs_sorted"] < 0.5 * full[3]["pairs_sorted"]
    fr, cr = full[2]["ranges"].astype(np.int64), cut[2]["ranges"].astype(np.int64)
    v = sc.views[0]
    tiles_x = v.width // 16
    check = [ty * tiles_x + tx for tx, ty in S.stress_tiles(v.width, v.height)]
    check += list(rng.choice(len(fr), 64, replace=False))
    for t in check:
        n = cr[t, 1] - cr[t, 0]
        assert n <= fr[t, 1] - fr[t, 0]
        assert np.array_equal(cut[2]["pair_items"][cr[t, 0]:cr[t, 1]], full[2]["pair_items"][fr[t, 0]:fr[t, 0] + n]), t
    for k in NAMES:
        assert rel_l2(cut[4][k], full[4][k]) < 1e-6, k
