"""The fused ERP L1 + D-SSIM loss kernel against the float64 oracle of ``oracle/loss.py``."""
import numpy as np
import pytest

from oracle import loss as OL

pytestmark = pytest.mark.gpu


def _pair(W, H, seed):
    rng = np.random.default_rng(seed)
    y = rng.uniform(size=(3, H, W)).astype(np.float32)
    # smooth-ish image near the target, as in training
    x = np.clip(y + rng.normal(scale=0.1, size=y.shape), 0, 1).astype(np.float32)
    return x, y


@pytest.mark.parametrize("W,H,area,wrap", [(256, 128, True, True), (200, 100, False, True), (96, 40, True, False)])
def test_loss_and_gradient_match_the_oracle(W, H, area, wrap):
    import torch
    from paper_2410_20686_gb300.loss import l1_dssim
    x, y = _pair(W, H, W + H)
    loss, grads = l1_dssim([torch.from_numpy(x).cuda()], [torch.from_numpy(y).cuda()], area_weight=area, wrap_u=wrap)
    ref_loss, ref_grad = OL.loss_and_grad(x, y, area_weight=area, wrap_u=wrap)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
    g = grads[0].cpu().numpy().astype(np.float64)
    err = np.linalg.norm(g - ref_grad) / np.linalg.norm(ref_grad)
    assert err <= 1e-4, err
    np.testing.assert_allclose(g, ref_grad, rtol=0, atol=1e-4 * np.abs(ref_grad).max())


@pytest.mark.parametrize("W,H,area", [(256, 128, True), (200, 50, False), (2048, 1024, False)])
def test_l1_alone_matches_the_oracle(W, H, area):
    import torch
    from paper_2410_20686_gb300.loss import l1_dssim
    x, y = _pair(W, H, 3 * W + H)
    loss, grads = l1_dssim([torch.from_numpy(x).cuda()], [torch.from_numpy(y).cuda()], lam=0.0, area_weight=area)
    ref_loss, ref_grad = OL.loss_and_grad(x, y, lam=0.0, area_weight=area)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
    np.testing.assert_allclose(grads[0].cpu().numpy(), ref_grad, rtol=1e-5, atol=1e-5 * np.abs(ref_grad).max())
    if not area:  # the plain mean absolute error: gradient sign(x - y) / (3 W H)
        np.testing.assert_array_equal(grads[0].cpu().numpy() != 0, x != y)


def test_identical_images_give_zero_loss_and_gradient():
    import torch
    from paper_2410_20686_gb300.loss import l1_dssim
    x, _ = _pair(128, 64, 5)
    t = torch.from_numpy(x).cuda()
    loss, grads = l1_dssim([t], [t.clone()])
    assert abs(float(loss)) < 1e-6
    assert float(grads[0].abs().max()) < 1e-7


def test_views_accumulate_into_one_loss():
    import torch
    from paper_2410_20686_gb300.loss import l1_dssim
    pairs = [_pair(128, 64, 7), _pair(256, 128, 8)]
    xs = [torch.from_numpy(p[0]).cuda() for p in pairs]
    ys = [torch.from_numpy(p[1]).cuda() for p in pairs]
    total, grads = l1_dssim(xs, ys)
    each = [float(l1_dssim([a], [b])[0]) for a, b in zip(xs, ys)]
    assert float(total) == pytest.approx(sum(each), rel=1e-6)
    for (x, y), g in zip(pairs, grads):
        _, ref = OL.loss_and_grad(x, y)
        assert np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-4


def test_full_size_view():
    import torch
    from paper_2410_20686_gb300.loss import l1_dssim
    x, y = _pair(2048, 1024, 11)
    loss, grads = l1_dssim([torch.from_numpy(x).cuda()], [torch.from_numpy(y).cuda()])
    ref_loss, ref_grad = OL.loss_and_grad(x, y)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
    g = grads[0].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref_grad) / np.linalg.norm(ref_grad) <= 1e-4


def test_drives_a_graphed_frame():
    import torch
    from paper_2410_20686_gb300 import scenes as S
    from paper_2410_20686_gb300.graph import GraphedFrame
    from paper_2410_20686_gb300.loss import l1_dssim
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    sc = S.config1()
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    targets = [torch.tensor(t, device="cuda") for t in S.target_images(sc, 1)]
    gf = GraphedFrame(params, sc.views, targets, RenderSettings(sh_degree=3), loss_fn=l1_dssim)
    l0 = float(gf.replay())
    torch.cuda.synchronize()
    assert gf.status() == 0 and np.isfinite(l0) and l0 > 0
    ref_loss, _ = OL.loss_and_grad(gf.images[0].cpu().numpy(), targets[0].cpu().numpy())
    assert l0 == pytest.approx(ref_loss, rel=1e-5)
    assert all(torch.isfinite(g).all() for g in gf.grads.values())
