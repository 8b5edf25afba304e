"""Parity at the full workload sizes, in the launch configurations the bench times.

The oracle costs O(Gaussians x pixels), so it checks seeded pixel samples (uniform pixels plus
pole and seam tiles): images per sampled pixel, and gradients of a loss that lives on the
sampled pixels only (the GPU backpropagates the same masked loss through the whole frame).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import EPS_CLAMP, EPS_SKIP, EPS_TERM, assert_grads_close, compare_image, oracle_settings

pytestmark = pytest.mark.gpu
NAMES = ("means", "scales", "quats", "opacity", "sh")


def _rs(**kw):
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    return RenderSettings(**kw)


def _masked_weights(p, view, st, pix, seed):
    _, _, _, margins = O.render(p, view, st, pix=pix)
    amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
    g = np.random.default_rng(seed).normal(size=(len(pix), 3)) * (~amb)[:, None]
    full = np.zeros((3, view.height * view.width), np.float32)
    full[:, pix] = g.T
    return g, full.reshape(3, view.height, view.width)


def _assert_grads(gpu, ref):
    assert_grads_close(gpu, ref, NAMES)


def test_config2_sampled_images_and_gradients():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sc = S.config2()
    rs = _rs(sh_degree=3)
    v = sc.views[0]
    pix = S.sample_pixels(v.width, v.height, 1024, S.stress_tiles(v.width, v.height), seed=22)
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    rast = Rasterizer()
    imgs, _ = rast.forward(*params, [v], rs, want_T=False)
    col, _, _, margins = O.render(p, v, st, pix=pix)
    compare_image(imgs[0].cpu().numpy().astype(np.float64).reshape(3, -1)[:, pix].T, col, margins)
    g, full = _masked_weights(p, v, st, pix, 22)
    ref = O.backward(p, v, st, g, pix=pix)
    gpu = rast.backward([torch.tensor(full, device="cuda")])
    torch.cuda.synchronize()
    assert rast.status() == 0
    _assert_grads({k: t.cpu().numpy().astype(np.float64) for k, t in gpu.items()}, ref)


def test_config3_all_views_in_one_frame():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    sc = S.config3()
    rs = _rs(sh_degree=3)
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    rast = Rasterizer()
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    weights, refs, amb = [], [], []
    for i, v in enumerate(sc.views):  # every view: 128 random pixels plus one pole or seam tile each
        stress = S.stress_tiles(v.width, v.height)
        pix = S.sample_pixels(v.width, v.height, 128, [stress[i % len(stress)]], seed=30 + i)
        col, _, _, margins = O.render(p, v, st, pix=pix)
        # a view's sample is small (one ambiguous pixel is ~0.3 %): the fraction is bounded over the frame
        compare_image(imgs[i].cpu().numpy().astype(np.float64).reshape(3, -1)[:, pix].T, col, margins, max_amb_frac=1.0)
        amb.append(O.ambiguous(margins, EPS_SKIP, EPS_TERM))
        g, full = _masked_weights(p, v, st, pix, 30 + i)
        refs.append(O.backward(p, v, st, g, pix=pix))
        weights.append(torch.tensor(full, device="cuda"))
    assert np.concatenate(amb).mean() <= 2e-3
    gpu = rast.backward(weights)
    torch.cuda.synchronize()
    assert rast.status() == 0
    ref = {k: sum(r[k] for r in refs) for k in NAMES}
    _assert_grads({k: t.cpu().numpy().astype(np.float64) for k, t in gpu.items()}, ref)


def test_config4_grouped_frame_with_recomputed_lists():
    import torch
    from paper_2410_20686_gb300.graph import GroupedFrame
    sc = S.config4()
    rs = _rs(sh_degree=3)
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    p = O.Params.of(sc)
    st = oracle_settings(rs)
    weights, refs, samples = [], [], {}
    for i, v in enumerate(sc.views):  # every view: 96 random pixels plus one pole or seam tile each
        stress = S.stress_tiles(v.width, v.height)
        pix = S.sample_pixels(v.width, v.height, 96, [stress[i % len(stress)]], seed=40 + i)
        g, full = _masked_weights(p, v, st, pix, 40 + i)
        refs.append(O.backward(p, v, st, g, pix=pix))
        weights.append(torch.tensor(full, device="cuda"))
        samples[i] = pix

    def fixed_weights(images, targets):  # linear loss: dL/dC = weights
        return None, weights

    gf = GroupedFrame(params, sc.views, weights, rs, group_size=2, loss_fn=fixed_weights)
    gf.step()
    torch.cuda.synchronize()
    assert gf.status() == 0
    amb = []
    for i, v in enumerate(sc.views):
        col, _, _, margins = O.render(p, v, st, pix=samples[i])
        compare_image(gf.images[i].cpu().numpy().astype(np.float64).reshape(3, -1)[:, samples[i]].T, col, margins,
                      max_amb_frac=1.0)
        amb.append(O.ambiguous(margins, EPS_SKIP, EPS_TERM))
    assert np.concatenate(amb).mean() <= 2e-3
    ref = {k: sum(r[k] for r in refs) for k in NAMES}
    _assert_grads({k: t.cpu().numpy().astype(np.float64) for k, t in gf.grads.items()}, ref)
