"""Densification on the device (Sec. 3.3) against the numpy oracle of ``oracle/densify.py``:
statistics gathered by the backward pass, the clone / split / prune decision (bit-exact: both
sides decide in float32 with the same operation order) and the densified arrays."""
import ctypes as C

import numpy as np
import pytest

from oracle import densify as OD
from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import EPS_CLAMP, EPS_SKIP, EPS_TERM, oracle_settings, rel_l2, to_torch


def _scene():
    sc = S.random_scene(3000, 256, 128, seed=11, sh_degree=3, radius=(1.0, 6.0))
    rot = S.yaw_view(256, 128, (0.1, 0.0, -0.2), 1.1)
    sc.views = [sc.views[0], rot, S.View(128, 64, rot.R_wc, rot.t_wc)]
    return sc


def _weights(scene, rs, seed):
    p = O.Params.of(scene)
    st = oracle_settings(rs)
    rng = np.random.default_rng(seed)
    out = []
    for v in scene.views:
        _, _, _, margins = O.render(p, v, st)
        amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
        out.append(rng.normal(size=(3, v.height, v.width)) * (~amb)[None])
    return out


# ------------------------------------------------------------------ host-side (no GPU)

def test_scratch_size_and_argument_checks():
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300 import build as B
    B.build()
    lib = L.load()
    a, b = C.c_size_t(), C.c_size_t()
    assert lib.odgs_densify_scratch_size(1000, C.byref(a)) == 0
    assert lib.odgs_densify_scratch_size(100000, C.byref(b)) == 0
    assert 0 < a.value < b.value
    assert lib.odgs_densify_scratch_size(-1, C.byref(a)) == L.ODGS_ERR_INVALID_ARG
    prm = L.DensifyParams(2e-5, 1e-4, 1e-3, 0.0, 0.005, 0.0)  # scene extent must be > 0
    null = C.c_void_p(0)
    assert lib.odgs_densify_select(null, null, null, null, null, 10, C.byref(prm), null, null) == L.ODGS_ERR_INVALID_ARG
    prm.scene_extent = 1.0
    assert lib.odgs_densify_select(null, null, null, null, null, 0, C.byref(prm), null, null) == 0
    assert lib.odgs_densify_select(null, null, null, null, null, 10, C.byref(prm), null, null) == L.ODGS_ERR_INVALID_ARG


# ------------------------------------------------------------------ device

@pytest.mark.gpu
def test_statistics_match_the_oracle_over_three_views():
    import torch
    from paper_2410_20686_gb300.densify import DensifyStats
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = _scene()
    rs = RenderSettings(sh_degree=3)
    ws = _weights(sc, rs, 3)
    stats = DensifyStats(sc.n)
    rast = Rasterizer()
    params = to_torch(sc)
    rast.forward(*params, sc.views, rs, want_T=False)
    rast.backward([torch.tensor(w, dtype=torch.float32, device="cuda") for w in ws], densify=stats)
    # a second frame adds to the running sums
    rast.forward(*params, sc.views[:1], rs, want_T=False)
    rast.backward([torch.tensor(ws[0], dtype=torch.float32, device="cuda")], densify=stats)
    torch.cuda.synchronize()
    assert rast.status() == 0
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    g3, e3, c3 = OD.stats(p, sc.views, st, ws)
    g1, e1, c1 = OD.stats(p, sc.views[:1], st, ws[:1])
    grad, elev, count = g3 + g1, e3 + e1, c3 + c1
    gc = stats.count.cpu().numpy()
    assert np.count_nonzero(gc != count) <= 2  # visibility: the same culls, up to threshold ties
    same = gc == count
    assert rel_l2(stats.grad.cpu().numpy()[same].astype(np.float64), grad[same]) <= 1e-3
    np.testing.assert_allclose(stats.elev.cpu().numpy()[same], elev[same], rtol=1e-5, atol=1e-6)
    assert count.sum() > sc.n  # most Gaussians are seen in several views


@pytest.mark.gpu
def test_select_is_bit_exact_against_the_oracle_rule():
    import torch
    from paper_2410_20686_gb300.densify import DensifyParams, DensifyStats, select
    rng = np.random.default_rng(5)
    n = 200_003
    # statistics clustered around the thresholds, so that many decisions are close calls
    count = rng.integers(0, 6, n).astype(np.uint32)
    elev = (rng.uniform(0, 1, n) * count).astype(np.float32)
    tau = OD.TAU_MIN + elev / np.maximum(count, 1) * (OD.TAU_MAX - OD.TAU_MIN)
    grad = (tau * count * rng.uniform(0.98, 1.02, n)).astype(np.float32)
    scales = rng.uniform(1e-4, 4e-3, (n, 3)).astype(np.float32)
    opac = rng.uniform(0.0, 0.02, n).astype(np.float32)
    prm = DensifyParams(scene_extent=1.5, max_scale=3.9e-3)
    st = DensifyStats(n)
    st.grad.copy_(torch.from_numpy(grad))
    st.elev.copy_(torch.from_numpy(elev))
    st.count.copy_(torch.from_numpy(count.astype(np.int32)))
    act = select(st, torch.from_numpy(scales).cuda(), torch.from_numpy(opac).cuda(), prm).cpu().numpy()
    ref = OD.select(grad, elev, count, scales, opac, OD.DensifyParams(**prm.__dict__))
    np.testing.assert_array_equal(act, ref)
    assert all(np.count_nonzero(ref == a) > 1000 for a in (OD.KEEP, OD.CLONE, OD.SPLIT, OD.PRUNE))


@pytest.mark.gpu
@pytest.mark.parametrize("n,k", [(1, 1), (1023, 16), (5000, 4), (70_001, 16)])
def test_apply_matches_the_oracle(n, k):
    import torch
    from paper_2410_20686_gb300.densify import apply
    rng = np.random.default_rng(n)
    means = rng.normal(size=(n, 3)).astype(np.float32)
    scales = rng.uniform(0.01, 0.1, (n, 3)).astype(np.float32)
    quats = rng.normal(size=(n, 4)).astype(np.float32)
    opac = rng.uniform(0.1, 0.9, n).astype(np.float32)
    sh = rng.normal(size=(n, k, 3)).astype(np.float32)
    action = rng.choice(np.array([0, 1, 2, 4], np.uint8), n, p=[0.55, 0.2, 0.15, 0.1])
    noise = rng.normal(size=(n, 2, 3)).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (means, scales, quats, opac, sh)]
    out = apply(*t, torch.from_numpy(action).cuda(), torch.from_numpy(noise).cuda())
    ref = OD.apply(means, scales, quats, opac, sh, action, noise)
    assert len(out[0]) == len(ref[0])
    nk = int(((action == 0) | (action == 1)).sum()) + int((action == 1).sum())
    for i, (a, b) in enumerate(zip(out, ref)):
        a = a.cpu().numpy()
        if i == 0:  # split children's positions: float32 arithmetic against FP64
            np.testing.assert_array_equal(a[:nk], b[:nk])
            np.testing.assert_allclose(a[nk:], b[nk:], rtol=0, atol=2e-6 * (1 + np.abs(b[nk:]).max(initial=0.0)))
        elif i == 1:  # scales / 1.6 rounded once
            np.testing.assert_array_equal(a[:nk], b[:nk])
            np.testing.assert_allclose(a[nk:], b[nk:], rtol=1e-7)
        else:
            np.testing.assert_array_equal(a, b.astype(np.float32))


@pytest.mark.gpu
def test_one_densification_round_on_a_rendered_scene():
    import torch
    from paper_2410_20686_gb300.densify import DensifyParams, DensifyStats, apply, select
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = S.config1()
    rs = RenderSettings(sh_degree=3)
    params = to_torch(sc)
    target = torch.tensor(S.target_images(sc, 1)[0], device="cuda")
    stats = DensifyStats(sc.n)
    rast = Rasterizer()
    for _ in range(3):
        imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
        g = torch.sign(imgs[0] - target) / imgs[0].numel()
        rast.backward([g], densify=stats)
    prm = DensifyParams(scene_extent=5.0)
    act = select(stats, params[1], params[3], prm)
    out = apply(*params, act, generator=torch.Generator(device="cuda").manual_seed(0))
    a = act.cpu().numpy()
    expect = int(((a == 0) | (a == 1)).sum() + (a == 1).sum() + 2 * (a == 2).sum())
    assert out[0].shape[0] == expect
    assert (a == 1).any() or (a == 2).any()
    # the densified scene still renders
    imgs2, _ = rast.forward(*out, sc.views, rs, want_T=False)
    torch.cuda.synchronize()
    assert rast.status() == 0 and torch.isfinite(imgs2[0]).all()
