"""Bit-exact checks of the integer work of the binning (depth keys, depth order, per-tile lists and
their ranges) against the oracle.

The paper fixes the blend order as sorting by depth (Sec. 3.1, the order of Eq. 3); the reading
of the depth is the radial distance |t| in IEEE single precision with a fixed operation order
(t_z for pinhole views), ties broken by item index. The library exposes its lists through
odgs_debug_lists. For every checked frame:
  - every depth key of a listed item equals the oracle's float32 key bit for bit, and the sorted
    (key, item) sequence is strictly increasing and a permutation of all items;
  - the pair list is sorted by tile, each tile's run is strictly ordered by (key, item), the
    ranges are exactly the runs (a searchsorted over the tile ids), and the run lengths add up
    to the pair count;
  - every tile lists every Gaussian that the oracle's projection gives alpha >= 1/255 at one of the
    tile's pixel centres (brute force over the pixels, with a margin of 1e-5 on the Mahalanobis
    bound so that float32 rounding cannot decide it), and no tile lists a Gaussian whose ellipse
    alpha = 1/255 (inflated by the binning's 1e-4 and a further 1e-3) misses the rectangle spanned
    by the tile's pixel centres.
These checks take the whole lists (full_lists); the lists cut at saturated tiles are prefixes of
them, checked in tests/test_truncated_lists.py.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import oracle_settings, to_torch

pytestmark = pytest.mark.gpu

NO_KEY = 0xFFFFFFFF


def _rs(**kw):
    # the whole lists: the truncated ones are checked against them (tests/test_truncated_lists.py)
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    kw.setdefault("full_lists", True)
    return RenderSettings(**kw)


def _camera_points(view, rng, n, kind):
    """World points whose camera-space direction lies near the seam or a pole of ``view``."""
    r = rng.uniform(1.0, 4.0, n)
    if kind == "seam":
        phi = np.pi - rng.uniform(-np.radians(5.0), np.radians(5.0), n)
        theta = rng.uniform(-1.0, 1.0, n)
    else:
        phi = rng.uniform(-np.pi, np.pi, n)
        theta = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0) * rng.uniform(np.radians(80.0), np.radians(89.9), n)
    t = np.stack([r * np.cos(theta) * np.sin(phi), -r * np.sin(theta), r * np.cos(theta) * np.cos(phi)], 1)
    R = np.asarray(view.R_wc, np.float64)
    return ((t - np.asarray(view.t_wc, np.float64)) @ R).astype(np.float32)  # R^T (t - t_wc)


def _scene(n=3000, seed=5):
    v0 = S.yaw_view(256, 128, (0.2, -0.1, 0.3), 0.9)
    v1 = S.yaw_view(128, 64, (-0.4, 0.2, 0.1), -2.3)
    v2 = S.pinhole_view(96, 64, 70.0, 70.0, R_wc=np.asarray(v0.R_wc), t_wc=np.asarray(v0.t_wc))
    sc = S.random_scene(n, 256, 128, seed=seed, sh_degree=1, radius=(0.8, 5.0), log_scale=(-3.0, 0.6),
                        views=[v0, v1, v2])
    rng = np.random.default_rng(seed)
    k = n // 5
    sc.means[:k] = _camera_points(v0, rng, k, "seam")
    sc.means[k:2 * k] = _camera_points(v0, rng, k, "pole")
    return sc


def _conic_bounds(pj):
    a, b, c = pj[:, O.PJ_CONIC], pj[:, O.PJ_CONIC + 1], pj[:, O.PJ_CONIC + 2]
    o = pj[:, O.PJ_OPAC]
    with np.errstate(divide="ignore", invalid="ignore"):
        Q = np.where(255.0 * o > 1.0, 2.0 * np.log(255.0 * o), -1.0)
        det = a * c - b * b
        eu = np.sqrt(np.maximum(Q, 0.0) * c / det)
        ev = np.sqrt(np.maximum(Q, 0.0) * a / det)
    ok = (pj[:, O.PJ_VALID] > 0) & (Q > 0) & (det > 0)
    return a, b, c, Q, eu, ev, ok


def _tile_rect(view, tw, th, t):
    tiles_x = view.width // tw
    tx, ty = t % tiles_x, t // tiles_x
    x0, x1 = tx * tw, tx * tw + tw - 1
    y0, y1 = ty * th, min(ty * th + th, view.height) - 1
    return x0, x1, y0, y1


def _required_items(pj, view, tw, th, t):
    """Items with alpha >= 1/255 (by a clear margin) at some pixel centre of local tile t."""
    a, b, c, Q, eu, ev, ok = _conic_bounds(pj)
    x0, x1, y0, y1 = _tile_rect(view, tw, th, t)
    u, v = pj[:, O.PJ_U], pj[:, O.PJ_V]
    W = view.width
    erp = view.model == 0
    # candidates: bounding box (seam-shifted for ERP) meets the tile's pixel centres
    cand = ok & (v + ev >= y0 + 0.5) & (v - ev <= y1 + 0.5)
    hx = np.zeros_like(cand)
    for sh in ((-W, 0, W) if erp else (0,)):
        hx |= (u + sh + eu >= x0 + 0.5) & (u + sh - eu <= x1 + 0.5)
    cand &= hx
    idx = np.nonzero(cand)[0]
    if idx.size == 0:
        return set()
    ys, xs = np.meshgrid(np.arange(y0, y1 + 1) + 0.5, np.arange(x0, x1 + 1) + 0.5, indexing="ij")
    dx = xs.ravel()[None, :] - u[idx, None]
    if erp:
        dx = dx - W * np.floor(dx / W + 0.5)
    dy = ys.ravel()[None, :] - v[idx, None]
    q = a[idx, None] * dx * dx + 2.0 * b[idx, None] * dx * dy + c[idx, None] * dy * dy
    inside = (q <= (Q[idx, None] * (1.0 - 1e-5) - 1e-6)).any(axis=1)
    return set(idx[inside].tolist())


def _rect_min_q(a, b, c, u, v, xl, xh, yl, yh):
    """Minimum of a dx^2 + 2 b dx dy + c dy^2 over the rectangle [xl, xh] x [yl, yh] (vectorised)."""
    dxl, dxh, dyl, dyh = xl - u, xh - u, yl - v, yh - v
    inside = (dxl <= 0) & (dxh >= 0) & (dyl <= 0) & (dyh >= 0)
    best = np.full(np.shape(u), np.inf)
    for dxe in (dxl, dxh):  # vertical edges: minimise over dy
        dy = np.clip(-b * dxe / c, dyl, dyh)
        best = np.minimum(best, a * dxe * dxe + 2 * b * dxe * dy + c * dy * dy)
    for dye in (dyl, dyh):  # horizontal edges: minimise over dx
        dx = np.clip(-b * dye / a, dxl, dxh)
        best = np.minimum(best, a * dx * dx + 2 * b * dx * dye + c * dye * dye)
    return np.where(inside, 0.0, best)


def _check_frame(sc, rs, lists, stats, tiles_checked=None, pair_sample=None, seed=0):
    """All the checks of the module docstring on one frame. tiles_checked: {view: local tiles}
    for the superset check (all tiles when None); pair_sample: number of listed pairs given the
    tightness check (all when None)."""
    n = sc.n
    views = sc.views
    tw, th = rs.tile_w, rs.tile_h
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    pjs = [O.project(p, v, st) for v in views]
    tiles_per_view = [(v.width // tw) * ((v.height + th - 1) // th) for v in views]
    tile_base = np.concatenate([[0], np.cumsum(tiles_per_view)])
    n_items = n * len(views)

    dkeys, ditems = lists["depth_keys"].astype(np.int64), lists["depth_items"].astype(np.int64)
    ptiles, pitems = lists["pair_tiles"].astype(np.int64), lists["pair_items"].astype(np.int64)
    ranges = lists["ranges"].astype(np.int64)

    # depth order: a permutation of all items, strictly increasing in (key, item)
    assert np.array_equal(np.sort(ditems), np.arange(n_items))
    inc = (dkeys[1:] > dkeys[:-1]) | ((dkeys[1:] == dkeys[:-1]) & (ditems[1:] > ditems[:-1]))
    assert inc.all(), f"depth order broken at {np.nonzero(~inc)[0][:5]}"
    key_of = np.empty(n_items, np.int64)
    key_of[ditems] = dkeys
    # keys of the listed items equal the oracle's float32 keys bit for bit
    okey = np.concatenate([pj[:, O.PJ_KEY] for pj in pjs]).astype(np.int64)
    ovalid = np.concatenate([pj[:, O.PJ_VALID] > 0 for pj in pjs])
    listed = key_of != NO_KEY
    assert listed.sum() == stats["visible"]
    assert ovalid[listed].all(), "an item the oracle culls has a depth key"
    bad = listed & (key_of != okey)
    assert not bad.any(), f"{bad.sum()} depth keys differ from the oracle's, e.g. item {np.nonzero(bad)[0][:3]}"

    # pairs: sorted by tile, per-tile (key, item) order, ranges, totals
    assert len(ptiles) == stats["pairs_sorted"] == stats["pairs"]
    assert (np.diff(ptiles) >= 0).all()
    assert ptiles.size == 0 or (ptiles[0] >= 0 and ptiles[-1] < tile_base[-1])
    lo = np.searchsorted(ptiles, np.arange(tile_base[-1]), "left")
    hi = np.searchsorted(ptiles, np.arange(tile_base[-1]), "right")
    empty = lo == hi
    assert np.array_equal(ranges[~empty, 0], lo[~empty]) and np.array_equal(ranges[~empty, 1], hi[~empty])
    assert (ranges[empty] == 0).all()
    assert (hi - lo).sum() == len(ptiles)
    k = key_of[pitems]
    same = ptiles[1:] == ptiles[:-1]
    ordered = (k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (pitems[1:] > pitems[:-1]))
    assert ordered[same].all(), "a tile's list is not in (depth key, item) order"
    assert (k != NO_KEY).all() and listed[pitems].all()
    # every pair's item belongs to the pair's view
    view_of_tile = np.searchsorted(tile_base, ptiles, "right") - 1
    assert np.array_equal(pitems // n, view_of_tile)

    # no list holds a Gaussian whose (inflated) ellipse misses the tile's pixel-centre rectangle
    rng = np.random.default_rng(seed)
    sel = np.arange(len(ptiles)) if pair_sample is None or pair_sample >= len(ptiles) else \
        rng.choice(len(ptiles), pair_sample, replace=False)
    for vi, v in enumerate(views):
        m = sel[view_of_tile[sel] == vi]
        if m.size == 0:
            continue
        g = pitems[m] - vi * n
        lt = ptiles[m] - tile_base[vi]
        a, b, c, Q, eu, _, ok = _conic_bounds(pjs[vi])
        assert ok[g].all()
        tiles_x = v.width // tw
        x0 = (lt % tiles_x) * tw + 0.5
        y0 = (lt // tiles_x) * th + 0.5
        x1 = x0 + tw - 1
        y1 = np.minimum((lt // tiles_x) * th + th, v.height) - 0.5
        s = 0.02
        u, vv = pjs[vi][g, O.PJ_U], pjs[vi][g, O.PJ_V]
        qmin = np.full(m.size, np.inf)
        # ERP: the binning lists a tile when any periodic copy u + k W of the ellipse meets it (a
        # pole-stretched ellipse can span several image widths); pinhole views have one copy
        kmax = int(np.ceil((eu[g].max() + 2 * v.width) / v.width)) if v.model == 0 else 0
        for k in range(-kmax, kmax + 1):
            sh = k * v.width
            qmin = np.minimum(qmin, _rect_min_q(a[g], b[g], c[g], u + sh, vv, x0 - s, x1 + s, y0 - s, y1 + s))
        Qb = (Q[g] * (1 + 1e-4) + 1e-4) * (1 + 1e-3) + 1e-3
        loose = qmin > Qb
        assert not loose.any(), f"view {vi}: {loose.sum()} listed pairs outside the footprint, e.g. tile " \
                                f"{lt[loose][:3]} item {g[loose][:3]}"

    # every tile lists every Gaussian that reaches alpha >= 1/255 at one of its pixel centres
    for vi, v in enumerate(views):
        tl = range(tiles_per_view[vi]) if tiles_checked is None else tiles_checked.get(vi, [])
        for t in tl:
            gt = tile_base[vi] + t
            have = set((pitems[ranges[gt, 0]:ranges[gt, 1]] - vi * n).tolist()) if ranges[gt, 1] > ranges[gt, 0] \
                else set()
            need = _required_items(pjs[vi], v, tw, th, t)
            missing = need - have
            assert not missing, f"view {vi} tile {t}: missing Gaussians {sorted(missing)[:5]}"


def _render_lists(sc, rs, rast=None):
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    rast = rast or Rasterizer()
    rast.forward(*to_torch(sc), sc.views, rs, want_T=False)
    torch.cuda.synchronize()
    assert rast.status() == 0
    return rast, rast.debug_lists(), rast.stats()


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_keys_order_lists_and_ranges_small_frame(tile):
    sc = _scene()
    rs = _rs(sh_degree=1, tile_w=tile[0], tile_h=tile[1])
    _, lists, stats = _render_lists(sc, rs)
    assert stats["pairs"] > 2 * sc.n
    _check_frame(sc, rs, lists, stats)


def test_lists_rebuilt_in_the_backward_pass_are_identical():
    import torch
    sc = _scene(seed=6)
    rs = _rs(sh_degree=1, recompute_lists=True)
    rast, first, _ = _render_lists(sc, rs)
    rast.backward([torch.ones((3, v.height, v.width), device="cuda") for v in sc.views])
    torch.cuda.synchronize()
    assert rast.status() == 0
    again = rast.debug_lists()
    for k in first:
        assert np.array_equal(first[k], again[k]), k


def test_keys_order_lists_and_ranges_config2_full_size():
    """The 1M-Gaussian, 2048x1024 frame with its pole and seam clusters: all keys, the whole
    order and every range; the footprint bound on 300k sampled pairs; the superset check on the
    eight pole and seam tiles and 24 random tiles."""
    sc = S.config2()
    rs = _rs(sh_degree=3)
    _, lists, stats = _render_lists(sc, rs)
    v = sc.views[0]
    rng = np.random.default_rng(2)
    tiles_x = v.width // 16
    stress = [ty * tiles_x + tx for tx, ty in S.stress_tiles(v.width, v.height)]
    rand = rng.choice(tiles_x * (v.height // 16), 24, replace=False).tolist()
    _check_frame(sc, rs, lists, stats, tiles_checked={0: stress + rand}, pair_sample=300_000)
