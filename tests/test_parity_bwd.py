"""GPU backward parity: gradients of all five parameter tensors against the oracle's FP64
adjoint (itself pinned to central differences), for a linear loss L = sum(g * C) whose weights g
vanish on pixels with a discrete decision (skip, termination or the 0.99 clamp) within rounding
of its threshold."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import (EPS_CLAMP, EPS_SKIP, EPS_TERM, SUM_BOUND, assert_grads_close, oracle_settings, rel_l2,
                           screen_abs_xy_to_slice, screen_slice_to_xy, screen_xy_to_slice, to_torch)

pytestmark = pytest.mark.gpu
NAMES = ("means", "scales", "quats", "opacity", "sh")


def _rs(**kw):
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    return RenderSettings(**kw)


def _weights(scene, rs, seed):
    """Random dL/dC per view, zeroed on ambiguous pixels (forward and clamp decisions)."""
    p = O.Params.of(scene)
    st = oracle_settings(rs)
    rng = np.random.default_rng(seed)
    out = []
    for v in scene.views:
        _, _, _, margins = O.render(p, v, st)
        amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
        g = rng.normal(size=(3, v.height, v.width)) * (~amb)[None]
        out.append(g)
    return out


def _gpu_grads(scene, rs, weights, rast=None):
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    rast = rast or Rasterizer()
    m, s, q, o, sh = to_torch(scene)
    rast.forward(m, s, q, o, sh, scene.views, rs, want_T=False)
    gi = [torch.tensor(w, dtype=torch.float32, device="cuda") for w in weights]
    g = rast.backward(gi)
    torch.cuda.synchronize()
    assert rast.status() == 0
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def _oracle_grads(scene, rs, weights):
    p = O.Params.of(scene)
    st = oracle_settings(rs)
    tot = None
    for v, w in zip(scene.views, weights):
        g = O.backward(p, v, st, w)
        tot = g if tot is None else {k: tot[k] + g[k] for k in NAMES}
    return tot


def _assert_close(gpu, ref):
    assert_grads_close(gpu, ref, NAMES)


@pytest.mark.parametrize("deg", [0, 3])
def test_gradients_small_scene(deg):
    view = S.yaw_view(96, 48, (0.2, -0.1, 0.05), 1.3)
    sc = S.random_scene(400, 96, 48, seed=80 + deg, sh_degree=deg, views=[view], log_scale=(-2.5, 0.5))
    rs = _rs(sh_degree=deg, bg=(0.3, 0.2, 0.1))
    w = _weights(sc, rs, 1)
    _assert_close(_gpu_grads(sc, rs, w), _oracle_grads(sc, rs, w))


def test_gradients_ragged_tiles_and_seam():
    rng = np.random.default_rng(3)
    sc = S.random_scene(500, 112, 60, seed=90, sh_degree=2, log_scale=(-2.4, 0.4))
    # a third of the Gaussians straddle the longitude seam
    k = 150
    r = rng.uniform(1.5, 4.0, k)
    phi = np.pi - rng.uniform(-0.05, 0.05, k)
    sc.means[:k] = np.stack([r * np.sin(phi), rng.uniform(-0.5, 0.5, k), r * np.cos(phi)], 1).astype(np.float32)
    rs = _rs(sh_degree=2)
    w = _weights(sc, rs, 2)
    _assert_close(_gpu_grads(sc, rs, w), _oracle_grads(sc, rs, w))


def test_gradients_multiple_views_accumulate():
    views = [S.View.identity(64, 32), S.yaw_view(128, 64, (0.1, 0.0, 0.2), 2.1), S.yaw_view(32, 16, (0, 0, 0), -0.4)]
    sc = S.random_scene(300, 64, 32, seed=95, sh_degree=1, views=views, log_scale=(-2.3, 0.4))
    rs = _rs(sh_degree=1)
    w = _weights(sc, rs, 3)
    _assert_close(_gpu_grads(sc, rs, w), _oracle_grads(sc, rs, w))


def test_recomputed_lists_give_the_same_gradients():
    sc = S.random_scene(800, 128, 64, seed=97, sh_degree=3, log_scale=(-2.6, 0.5))
    w = _weights(sc, _rs(sh_degree=3), 4)
    a = _gpu_grads(sc, _rs(sh_degree=3), w)
    b = _gpu_grads(sc, _rs(sh_degree=3, recompute_lists=True), w)
    for k in NAMES:
        assert rel_l2(b[k], a[k]) < 1e-6, k


def test_backward_accumulators_start_from_zero():
    """The per-(view, Gaussian) accumulators of the backward blend start from zero on every call:
    a second backward of the same forward, and the next frame after a backward, give the oracle's
    gradients as the first backward does."""
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sc = S.random_scene(600, 96, 48, seed=99, sh_degree=2, log_scale=(-2.5, 0.5))
    rs = _rs(sh_degree=2)
    w = _weights(sc, rs, 5)
    ref = _oracle_grads(sc, rs, w)
    rast = Rasterizer()
    first = _gpu_grads(sc, rs, w, rast)
    gi = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in w]
    again = rast.backward(gi)
    torch.cuda.synchronize()
    again = {k: v.cpu().numpy().astype(np.float64) for k, v in again.items()}
    nxt = _gpu_grads(sc, rs, w, rast)
    for g in (first, again, nxt):
        _assert_close(g, ref)
    for k in NAMES:  # the same sums, up to the order of the atomic additions
        assert rel_l2(again[k], first[k]) < 1e-6, k
        assert rel_l2(nxt[k], first[k]) < 1e-6, k


@pytest.mark.parametrize("tile_w,tile_h,ppt,ppt_bwd", [(16, 16, 2, 4), (32, 8, 1, 1), (32, 16, 2, 2), (8, 8, 1, 2),
                                                     (16, 16, 4, 2)])
def test_gradients_across_thread_layouts(tile_w, tile_h, ppt, ppt_bwd):
    # Tile shapes and pixels per thread of both blend kernels (one to eight warps per tile in the
    # backward pass; a forward thread's pixels spread over several backward threads in the last
    # case): against the oracle, and against the same frame with its lists rebuilt for the
    # backward pass (equal up to the order of the atomic sums).
    sc = S.random_scene(900, 128, 64, seed=98, sh_degree=2, log_scale=(-2.6, 0.5))
    kw = dict(sh_degree=2, tile_w=tile_w, tile_h=tile_h, pixels_per_thread=ppt, pixels_per_thread_bwd=ppt_bwd)
    w = _weights(sc, _rs(**kw), 6)
    a = _gpu_grads(sc, _rs(**kw), w)
    b = _gpu_grads(sc, _rs(recompute_lists=True, **kw), w)
    for k in NAMES:
        assert rel_l2(b[k], a[k]) < 1e-6, k
    _assert_close(a, _oracle_grads(sc, _rs(**kw), w))


def test_autograd_function_matches_direct_backward():
    import torch
    from paper_2410_20686_gb300.rasterizer import render
    sc = S.random_scene(300, 64, 32, seed=99, sh_degree=2, log_scale=(-2.4, 0.4))
    rs = _rs(sh_degree=2)
    w = _weights(sc, rs, 5)
    params = to_torch(sc, requires_grad=True)
    (img,) = render(*params, sc.views, rs)
    loss = (img * torch.tensor(w[0], dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    direct = _gpu_grads(sc, rs, w)
    for k, t in zip(NAMES, params):
        assert np.allclose(t.grad.cpu().numpy(), direct[k], rtol=1e-5, atol=1e-7), k


def test_gradients_config1_sampled_loss():
    sc = S.config1()
    rs = _rs(sh_degree=3)
    v = sc.views[0]
    pix = S.sample_pixels(v.width, v.height, 1024, S.stress_tiles(v.width, v.height)[:2], seed=7)
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    _, _, _, margins = O.render(p, v, st, pix=pix)
    amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
    rng = np.random.default_rng(7)
    gp = rng.normal(size=(len(pix), 3)) * (~amb)[:, None]
    ref = O.backward(p, v, st, gp, pix=pix)
    full = np.zeros((3, v.height * v.width))
    full[:, pix] = gp.T
    gpu = _gpu_grads(sc, rs, [full.reshape(3, v.height, v.width)])
    _assert_close(gpu, ref)


def test_gradients_largest_view_16384x8192():
    """Backward at the largest supported view (pixel anchors up to 16383 in their 16-bit fields,
    524,288 tiles) on a sampled loss: dL/dC is non-zero only on the sampled pixels (random ones,
    the seam and pole tiles, the tiles of the first Gaussians' centres), so the oracle's adjoint
    of those pixels is the whole gradient."""
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sc = S.random_scene(5000, 16384, 8192, seed=23, sh_degree=1, radius=(0.5, 3.0), log_scale=(-3.0, 0.5))
    rs = _rs(sh_degree=1)
    v = sc.views[0]
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    pj = O.project(p, v, st)
    vis = pj[:, O.PJ_VALID] > 0
    centres = [(int(u) // 16, int(w) // 16) for u, w in pj[vis][:12, [O.PJ_U, O.PJ_V]]]
    pix = S.sample_pixels(v.width, v.height, 4096, S.stress_tiles(v.width, v.height) + centres, seed=25)
    _, _, nc, margins = O.render(p, v, st, pix=pix)
    amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
    rng = np.random.default_rng(25)
    gp = rng.normal(size=(len(pix), 3)) * (~amb)[:, None]
    ref = O.backward(p, v, st, gp, pix=pix)
    rast = Rasterizer()
    m, s, q, o, sh = to_torch(sc)
    rast.forward(m, s, q, o, sh, sc.views, rs, want_T=False)
    g = torch.zeros(3, v.height * v.width, device="cuda")
    g[:, torch.from_numpy(pix.astype(np.int64)).cuda()] = torch.tensor(gp.T, dtype=torch.float32, device="cuda")
    out = rast.backward([g.view(3, v.height, v.width)])
    torch.cuda.synchronize()
    assert rast.status() == 0
    gpu = {k: t.cpu().numpy().astype(np.float64) for k, t in out.items()}
    assert (nc > 0).sum() > 1000
    assert (np.abs(ref["opacity"]) > 0).sum() > 50  # many Gaussians receive a gradient
    _assert_close(gpu, ref)


def _degenerate_scene():
    sc = S.random_scene(300, 128, 64, seed=61, sh_degree=1, log_scale=(-2.5, 0.5))
    m, s, o = sc.means, sc.scales, sc.opacity
    m[0] = [0.0, 2.0, 0.0]  # on the pole axis (rho = 0): culled
    m[1] = [0.0, -1.5, 0.0]  # on the other pole axis: culled
    m[2] = [0.0, 0.0, 0.0]  # at the camera centre: culled
    m[3] = [0.05, 0.05, 0.05]  # inside the near sphere: culled
    m[4] = [0.5, 0.1, 1.5]
    o[4] = 0.0  # zero opacity: culled
    m[5] = [1.0, 0.2, 2.0]
    s[5] = 0.0  # all scales zero: the splat is the dilation alone
    o[5] = 0.8
    m[6] = [-1.0, 0.1, 1.5]
    s[6] = [0.3, 0.3, 0.0]  # flat disc
    o[6] = 0.7
    m[7] = [0.006, -2.0, 0.0]  # rho / r = 3e-3: kept, stretched over the top rows
    s[7] = 0.05
    o[7] = 0.9
    return sc


def test_degenerate_gaussians_forward_and_gradients():
    """Gaussians on the pole axes, at the camera centre, inside the near sphere and with zero
    opacity are culled on both sides (image unchanged, gradients exactly zero); a Gaussian with
    all scales zero renders as its screen-space dilation and gets exactly zero scale and rotation
    gradients; a flat disc and a near-pole Gaussian follow the oracle."""
    from tests.helpers import compare_image, gpu_render
    sc = _degenerate_scene()
    rs = _rs(sh_degree=1)
    v = sc.views[0]
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    pj = O.project(p, v, st)
    assert list(pj[:8, O.PJ_VALID]) == [0, 0, 0, 0, 0, 1, 1, 1]
    imgs, _, _ = gpu_render(sc, rs)
    ref, _, nc, margins = O.render(p, v, st)
    compare_image(imgs[0], ref, margins)
    assert (nc > 0).mean() > 0.3
    w = _weights(sc, rs, 3)
    gpu = _gpu_grads(sc, rs, w)
    _assert_close(gpu, _oracle_grads(sc, rs, w))
    for k in NAMES:
        assert np.all(gpu[k][:5] == 0.0), k
    assert np.all(gpu["scales"][5] == 0.0) and np.all(gpu["quats"][5] == 0.0)
    assert np.abs(gpu["means"][5]).max() > 0 and np.abs(gpu["means"][7]).max() > 0


def test_gaussians_exactly_on_the_seam():
    """Means straight behind the camera (azimuth exactly +-180 deg, u = W on the wrapped image),
    one with a negative-zero x, one a hair past the seam, and one straight ahead: images and all
    five gradients against the oracle."""
    from tests.helpers import compare_image, gpu_render
    sc = S.random_scene(200, 128, 64, seed=71, sh_degree=1, log_scale=(-2.5, 0.5))
    m, s, o = sc.means, sc.scales, sc.opacity
    m[0] = [0.0, 0.0, -2.0]
    m[1] = [-0.0, 0.3, -1.5]
    m[2] = [0.0, 0.0, 2.0]
    m[3] = [1e-7, -0.2, -3.0]
    s[0:4] = np.array([0.15, 0.1, 0.1, 0.2], np.float32)[:, None]
    o[0:4] = [0.9, 0.8, 0.9, 0.7]
    rs = _rs(sh_degree=1)
    v = sc.views[0]
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    imgs, _, _ = gpu_render(sc, rs)
    ref, _, nc, margins = O.render(p, v, st)
    compare_image(imgs[0], ref, margins)
    assert (nc[:, 0] > 0).sum() > 10 and (nc[:, -1] > 0).sum() > 10  # both image edges covered
    w = _weights(sc, rs, 4)
    _assert_close(_gpu_grads(sc, rs, w), _oracle_grads(sc, rs, w))


def test_gaussians_within_a_twentieth_of_a_degree_of_the_poles():
    """Means 0.006-0.05 deg from either pole (rho / r from 1.2e-4, just above the 1e-4 cull, to
    8.7e-4), where J_omni's 1 / rho terms are largest and each footprint stretches over whole
    rows: images and all five gradients against the oracle."""
    from tests.helpers import compare_image, gpu_render
    rng = np.random.default_rng(9)
    n, W, H = 80, 128, 64
    sc = S.random_scene(n, W, H, seed=91, sh_degree=1, log_scale=(-2.5, 0.4))
    r = rng.uniform(1.0, 3.0, n)
    eps = np.radians(rng.uniform(0.006, 0.05, n))
    phi = rng.uniform(-np.pi, np.pi, n)
    theta = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0) * (np.pi / 2 - eps)
    sc.means[:] = np.stack([r * np.cos(theta) * np.sin(phi), -r * np.sin(theta), r * np.cos(theta) * np.cos(phi)],
                           1).astype(np.float32)
    rs = _rs(sh_degree=1)
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    assert O.project(p, sc.views[0], st)[:, O.PJ_VALID].sum() == n
    imgs, _, _ = gpu_render(sc, rs)
    ref, _, nc, margins = O.render(p, sc.views[0], st)
    compare_image(imgs[0], ref, margins)
    assert (nc[0] > 0).all() and (nc[-1] > 0).all()
    w = _weights(sc, rs, 5)
    _assert_close(_gpu_grads(sc, rs, w), _oracle_grads(sc, rs, w))


def test_needle_gaussians_blend_and_chain_separately():
    """Needle-like Gaussians (one axis 30-300x the others, 1-5 m from the cameras, so that
    cond(Sigma_2D) exceeds 1e3 for 839 of the visible items, 1e4 for 67, and reaches 2.7e5) in
    three views. The backward pass is checked in its two halves, each against FP64: the
    per-(view, Gaussian) screen-space gradients of the reverse blend (Eq. 2-3) against the
    oracle's (converted to the library's slice-form conic), and the parameter gradients against
    the oracle's chain rule (App. A.3) applied to the GPU's own screen-space gradients; then the
    whole against the oracle adjoint."""
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    views = [S.yaw_view(256, 128, (0.05, -0.02, 0.1), 0.6), S.yaw_view(128, 64, (0.3, 0.1, -0.2), -1.9),
             S.View.identity(192, 96)]
    sc = S.random_scene(1500, 256, 128, seed=131, sh_degree=1, radius=(1.0, 5.0), log_scale=(-4.5, 0.3),
                        views=views)
    rng = np.random.default_rng(131)
    long_axis = rng.integers(0, 3, sc.n)
    sc.scales[np.arange(sc.n), long_axis] *= np.exp(rng.uniform(np.log(30), np.log(300), sc.n)).astype(np.float32)
    rs = _rs(sh_degree=1)
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    conds = []
    for v in views:
        pj = O.project(p, v, st)
        ok = pj[:, O.PJ_VALID] > 0
        c = pj[ok][:, O.PJ_COV2:O.PJ_COV2 + 3]
        tr, det = c[:, 0] + c[:, 2], c[:, 0] * c[:, 2] - c[:, 1] ** 2
        l1 = tr / 2 + np.sqrt(np.maximum(tr * tr / 4 - det, 0))
        conds.append(l1 * l1 / det)
    conds = np.concatenate(conds)
    assert (conds > 1e3).sum() > 500 and (conds > 1e4).sum() > 30 and conds.max() > 1e5  # the stress is there
    w = _weights(sc, rs, 13)
    rast = Rasterizer()
    m, s, q, o, sh = to_torch(sc)
    rast.forward(m, s, q, o, sh, views, rs, want_T=False)
    g = rast.backward([torch.tensor(x, dtype=torch.float32, device="cuda") for x in w])
    torch.cuda.synchronize()
    assert rast.status() == 0
    gpu = {k: t.cpu().numpy().astype(np.float64) for k, t in g.items()}
    screen = rast.debug_screen_grads().astype(np.float64).reshape(len(views), sc.n, 9)
    ref_screen, ref_abs, chain, ref = [], [], None, None
    for i, (v, wv) in enumerate(zip(views, w)):
        pj = O.project(p, v, st)
        r = O.backward(p, v, st, wv, want_g2=True, want_abs=True)
        # the library reports the conic gradient in slice form; the oracle in image-axis entries
        ref_screen.append(screen_xy_to_slice(r.pop("screen"), pj))
        ref_abs.append(screen_abs_xy_to_slice(r.pop("screen_abs"), pj))
        ref = r if ref is None else {k: ref[k] + r[k] for k in NAMES}
        c = O.chain(p, v, st, screen_slice_to_xy(screen[i], pj))
        chain = c if chain is None else {k: chain[k] + c[k] for k in NAMES}
    ref_screen, ref_abs = np.stack(ref_screen), np.stack(ref_abs)
    names = ("u", "v", "a", "beta", "gamma", "opacity", "r", "g", "b")
    # 1. the reverse blend: each screen-space gradient is a sum of per-pixel contributions whose
    #    signs follow the random loss weights, so some sums cancel by factors of 1e3-1e4; the band
    #    adds the float32 summation bound SUM_BOUND * sum|contribution| (the oracle's own sums)
    assert_grads_close({nm: screen[..., j] for j, nm in enumerate(names)},
                       {nm: ref_screen[..., j] for j, nm in enumerate(names)}, names,
                       slack={nm: SUM_BOUND * ref_abs[..., j] for j, nm in enumerate(names)}, what="screen ")
    # 2. the chain rule alone, element by element at the plain band
    assert_grads_close(gpu, chain, NAMES, what="chain ")
    # 3. the whole, per tensor (relative L2): its elements are covered by 1. and 2.
    for k in NAMES:
        assert rel_l2(gpu[k], ref[k]) <= 1e-3, k
