"""Pins of the ERP L1 + D-SSIM loss oracle against closed forms, a library filter and finite
differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from scipy import ndimage  # noqa: E402

from oracle import loss as OL  # noqa: E402


def test_window_is_the_normalised_sigma_1p5_gaussian():
    g = OL.window_1d()
    assert len(g) == 11 and g.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
    for k in range(1, 6):
        assert g[5] / g[5 + k] == pytest.approx(np.exp(k * k / (2 * 1.5 ** 2)), rel=1e-13)


def test_row_weights_integrate_to_the_sphere():
    H = 512
    area = OL.row_weights(H).sum() * (np.pi / H) * (2 * np.pi)  # midpoint rule over theta, times 2 pi in phi
    assert area == pytest.approx(4 * np.pi, rel=1e-5)


def test_blur_matches_scipy_correlation_with_wrap_and_zero_boundaries():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 20, 33))
    g = OL.window_1d()
    ours = OL._blur(torch.tensor(x), g, wrap_u=True).numpy()
    ref = ndimage.correlate1d(ndimage.correlate1d(x, g, axis=2, mode="wrap"), g, axis=1, mode="constant", cval=0.0)
    np.testing.assert_allclose(ours, ref, rtol=1e-12, atol=1e-14)
    ours0 = OL._blur(torch.tensor(x), g, wrap_u=False).numpy()
    ref0 = ndimage.correlate1d(ndimage.correlate1d(x, g, axis=2, mode="constant"), g, axis=1, mode="constant")
    np.testing.assert_allclose(ours0, ref0, rtol=1e-12, atol=1e-14)


def test_identical_images_give_ssim_one_and_zero_loss():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(3, 24, 48))
    s = OL.ssim_map(torch.tensor(x), torch.tensor(x)).numpy()
    np.testing.assert_allclose(s, 1.0, rtol=0, atol=1e-12)
    loss, grad = OL.loss_and_grad(x, x)
    assert abs(loss) < 1e-12
    np.testing.assert_allclose(grad, 0.0, atol=1e-12)


def test_constant_images_match_the_closed_form_away_from_the_edges():
    a, b = 0.3, 0.7
    x = np.full((3, 30, 40), a)
    y = np.full((3, 30, 40), b)
    s = OL.ssim_map(torch.tensor(x), torch.tensor(y)).numpy()
    expect = (2 * a * b + OL.C1) / (a * a + b * b + OL.C1)  # zero variances: the structure term is 1
    np.testing.assert_allclose(s[:, 5:-5, :], expect, rtol=1e-12)


def test_affine_images_match_the_ssim_formula_of_their_local_statistics():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(3, 26, 37))
    a, b = 0.6, 0.15
    y = a * x + b
    g = OL.window_1d()
    mu = OL._blur(torch.tensor(x), g, True).numpy()
    var = OL._blur(torch.tensor(x * x), g, True).numpy() - mu * mu
    muy = a * mu + b
    expect = ((2 * mu * muy + OL.C1) * (2 * a * var + OL.C2)) / ((mu * mu + muy * muy + OL.C1) * ((1 + a * a) * var + OL.C2))
    s = OL.ssim_map(torch.tensor(x), torch.tensor(y)).numpy()
    # mu_y = a mu_x + b needs the window's full mass: rows within 5 of the zero-padded edges lose part of b
    np.testing.assert_allclose(s[:, 5:-5], expect[:, 5:-5], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("area_weight,wrap_u", [(True, True), (False, False)])
def test_gradient_matches_central_differences(area_weight, wrap_u):
    rng = np.random.default_rng(3)
    y = rng.uniform(size=(3, 16, 24))
    x = np.clip(y + rng.normal(scale=0.2, size=y.shape), 0, 1)
    x[np.abs(x - y) < 1e-3] += 2e-3  # keep |x - y| away from the L1 kink
    loss, grad = OL.loss_and_grad(x, y, area_weight=area_weight, wrap_u=wrap_u)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 7, 23), (2, 15, 11), (0, 3, 5), (2, 8, 0)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (OL.loss_and_grad(x + e, y, area_weight=area_weight, wrap_u=wrap_u)[0]
              - OL.loss_and_grad(x - e, y, area_weight=area_weight, wrap_u=wrap_u)[0]) / (2 * h)
        assert grad[idx] == pytest.approx(fd, rel=1e-6, abs=1e-11)
