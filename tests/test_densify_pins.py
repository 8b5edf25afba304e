"""Pins of the densification oracle (Sec. 3.3, App. A.1) against values fixed outside it."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import densify as D
from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S

TAU = 2.0 * np.pi


def _view(W, H, R=None):
    return S.View(W, H, np.eye(3) if R is None else np.asarray(R, float), np.zeros(3))


def _single(t, sigma=0.05, o=0.9):
    dc = (np.array([0.8, 0.3, 0.55]) - 0.5) * 2.0 * np.sqrt(np.pi)
    return O.Params(np.atleast_2d(t), np.full((1, 3), sigma), np.array([[0.9, 0.1, -0.3, 0.2]]),
                    np.array([o]), dc.reshape(1, 1, 3))


def _at(r, theta, phi):
    """Camera-space point at distance r, elevation theta, azimuth phi (inverse of Eq. 4's angles)."""
    return r * np.array([np.cos(theta) * np.sin(phi), -np.sin(theta), np.cos(theta) * np.cos(phi)])


def test_threshold_follows_the_elevation_formula_with_the_papers_values():
    # App. A.1: tau_min = 2e-5, tau_max = 1e-4; Sec. 3.3: tau = tau_min + (1 - cos theta)(tau_max - tau_min)
    assert D.tau(1 - np.cos(0.0)) == pytest.approx(2e-5, rel=1e-12)
    assert D.tau(1 - np.cos(np.pi / 3)) == pytest.approx(6e-5, rel=1e-12)
    assert D.tau(1 - np.cos(np.pi / 2)) == pytest.approx(1e-4, rel=1e-12)
    assert D.tau(1 - np.cos(-np.pi / 2)) == pytest.approx(1e-4, rel=1e-12)


@pytest.mark.parametrize("theta_deg", [0.0, 30.0, -55.0, 80.0])
def test_elevation_statistic_and_visibility_of_a_placed_gaussian(theta_deg):
    W, H = 256, 128
    th = np.deg2rad(theta_deg)
    p = _single(_at(3.0, th, 0.7))
    st = O.Settings(sh_degree=0)
    w = np.ones((3, H, W))
    _, elev, count = D.stats(p, [_view(W, H)], st, [w])
    assert count[0] == 1
    assert elev[0] == pytest.approx(1 - np.cos(th), abs=1e-12)
    # inside the near shell: not visible, no statistics
    p2 = _single(_at(0.1, th, 0.7))
    g2, e2, c2 = D.stats(p2, [_view(W, H)], st, [w])
    assert (g2[0], e2[0], c2[0]) == (0.0, 0.0, 0)


def test_gradient_statistic_equals_the_yaw_finite_difference():
    # A Gaussian on the equator (v = H/2, a row boundary) under a loss whose weights do not depend
    # on the row: by the vertical symmetry dL/dv = 0, so the statistic is |dL/du| W/2. A camera
    # yaw psi moves the Gaussian along u only (Eq. 4), so dL/du = (dL/dpsi) / (du/dpsi).
    W, H = 256, 128
    p = _single(_at(2.0, 0.0, 0.4123), sigma=0.03, o=0.8)
    st = O.Settings(sh_degree=0)
    xs = np.arange(W) + 0.5
    wx = np.sin(xs * 0.37) + 0.2 * np.cos(xs * 0.11)
    w = np.stack([wx, -0.5 * wx, 0.3 * wx])[:, None, :].repeat(H, axis=1)

    def at_yaw(psi):
        c, s = np.cos(psi), np.sin(psi)
        R = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]]).T
        img, _, _, _ = O.render(p, _view(W, H, R), st)
        u = O.project(p, _view(W, H, R), st)[0, O.PJ_U]
        return float((img * w).sum()), u

    eps = 1e-6
    lp, up = at_yaw(eps)
    lm, um = at_yaw(-eps)
    dL_du = (lp - lm) / (up - um)
    grad, _, count = D.stats(p, [_view(W, H)], st, [w])
    g = O.backward(p, _view(W, H), st, w, want_g2=True)["screen"][0]
    assert abs(g[1]) < 1e-9 * max(1.0, abs(g[0]))
    assert count[0] == 1
    assert grad[0] == pytest.approx(abs(dL_du) * W / 2, rel=1e-6)


def test_statistics_add_over_views():
    W, H = 128, 64
    sc = S.random_scene(40, W, H, seed=5, sh_degree=1, radius=(1.5, 4.0))
    p = O.Params.of(sc)
    st = O.Settings(sh_degree=1)
    views = [_view(W, H), _view(W, H, Rotation.from_euler("y", 0.6).as_matrix())]
    rng = np.random.default_rng(0)
    ws = [rng.normal(size=(3, H, W)) for _ in views]
    both = D.stats(p, views, st, ws)
    each = [D.stats(p, [v], st, [w]) for v, w in zip(views, ws)]
    for k in range(3):
        np.testing.assert_allclose(both[k], each[0][k] + each[1][k], rtol=1e-12, atol=0)


def test_select_rule_on_hand_worked_cases():
    prm = D.DensifyParams(scene_extent=2.0)  # clone / split boundary: max scale 2e-3
    cases = [
        # (grad sum, elev sum, count, max scale, opacity) -> action
        ((4e-5, 0.0, 2, 1e-3, 0.5), D.CLONE),    # mean 2e-5 at the equator reaches tau_min exactly
        ((4e-5, 0.0, 2, 3e-3, 0.5), D.SPLIT),    # same gradient, large Gaussian
        ((3.9e-5, 0.0, 2, 1e-3, 0.5), D.KEEP),   # just below tau_min
        ((1.3e-4, 1.0, 2, 1e-3, 0.5), D.CLONE),  # mean 6.5e-5 at mean 1 - cos = 0.5: tau = 6e-5
        ((1.0e-4, 1.0, 2, 1e-3, 0.5), D.KEEP),   # mean 5e-5 < 6e-5
        ((1.9e-4, 2.0, 2, 1e-3, 0.5), D.KEEP),   # poles: tau = 1e-4 > 9.5e-5
        ((1.0, 0.0, 0, 1e-3, 0.5), D.KEEP),      # never visible: no mean gradient
        ((1.0, 0.0, 3, 5e-3, 0.004), D.PRUNE),   # transparent: removed whatever its gradient
    ]
    g = np.array([c[0][0] for c in cases], np.float32)
    e = np.array([c[0][1] for c in cases], np.float32)
    n = np.array([c[0][2] for c in cases], np.uint32)
    s = np.array([[c[0][3] * 0.5, c[0][3], c[0][3] * 0.1] for c in cases], np.float32)
    o = np.array([c[0][4] for c in cases], np.float32)
    np.testing.assert_array_equal(D.select(g, e, n, s, o, prm), [c[1] for c in cases])
    big = D.DensifyParams(scene_extent=2.0, max_scale=4e-3)
    assert D.select(g[1:2], e[1:2], n[1:2], s[1:2] * 2, o[1:2], big)[0] == D.PRUNE


def test_apply_clones_splits_and_prunes():
    rng = np.random.default_rng(7)
    n = 9
    means = rng.normal(size=(n, 3))
    scales = rng.uniform(0.01, 0.1, size=(n, 3))
    quats = rng.normal(size=(n, 4))
    opac = rng.uniform(0.1, 0.9, n)
    sh = rng.normal(size=(n, 4, 3))
    action = np.array([0, 1, 2, 4, 0, 2, 1, 0, 4], np.uint8)
    noise = rng.normal(size=(n, 2, 3))
    out = D.apply(means, scales, quats, opac, sh, action, noise)
    keep = [0, 1, 4, 6, 7]
    clones = [1, 6]
    splits = [2, 5]
    assert len(out[0]) == len(keep) + len(clones) + 2 * len(splits)
    for k, a in enumerate((means, scales, quats, opac, sh)):
        np.testing.assert_array_equal(out[k][:5], a[keep])
        np.testing.assert_array_equal(out[k][5:7], a[clones])
    for k, a in enumerate((quats, opac, sh)):
        np.testing.assert_array_equal(out[k + 2][7:9], a[splits])
        np.testing.assert_array_equal(out[k + 2][9:11], a[splits])
    np.testing.assert_allclose(out[1][7:], np.concatenate([scales[splits], scales[splits]]) / 1.6, rtol=1e-15)
    # a child sits at mu + R S z: its Mahalanobis distance under the parent's Sigma = R S^2 R^T is |z|
    for c in range(2):
        for j, i in enumerate(splits):
            R = Rotation.from_quat(np.roll(quats[i], -1)).as_matrix()  # scipy takes (x, y, z, w)
            Sig = R @ np.diag(scales[i] ** 2) @ R.T
            d = out[0][7 + 2 * c + j] - means[i]
            assert d @ np.linalg.solve(Sig, d) == pytest.approx(noise[i, c] @ noise[i, c], rel=1e-10)


def test_raw_parameter_mode_agrees_with_activated_mode():
    # log-scales and opacity logits: the same decisions away from the thresholds, and children whose
    # activated scales are the activated mode's children
    rng = np.random.default_rng(3)
    n = 4000
    count = rng.integers(1, 5, n).astype(np.uint32)
    elev = (rng.uniform(0, 1, n) * count).astype(np.float32)
    grad = (rng.uniform(0, 2e-4, n) * count).astype(np.float32)
    scales = rng.uniform(5e-4, 6e-3, (n, 3))
    opac = rng.uniform(0.0, 0.02, n)
    prm = D.DensifyParams(scene_extent=2.0, max_scale=5e-3)
    raw = D.DensifyParams(scene_extent=2.0, max_scale=5e-3, raw_params=True)
    a = D.select(grad, elev, count, scales.astype(np.float32), opac.astype(np.float32), prm)
    b = D.select(grad, elev, count, np.log(scales).astype(np.float32),
                 np.log(opac / (1 - opac)).astype(np.float32), raw)
    smax = scales.max(axis=1)
    far = (np.abs(smax / 2e-3 - 1) > 1e-5) & (np.abs(smax / 5e-3 - 1) > 1e-5) & (np.abs(opac / 0.005 - 1) > 1e-5)
    np.testing.assert_array_equal(a[far], b[far])
    assert far.mean() > 0.99
    q = rng.normal(size=(n, 4))
    mu = rng.normal(size=(n, 3))
    sh = rng.normal(size=(n, 1, 3))
    noise = rng.normal(size=(n, 2, 3))
    act = a.copy()
    act[act == D.PRUNE] = D.SPLIT
    x = D.apply(mu, scales, q, opac, sh, act, noise)
    y = D.apply(mu, np.log(scales), q, opac, sh, act, noise, raw_params=True)
    np.testing.assert_allclose(x[0], y[0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(x[1], np.exp(y[1]), rtol=1e-12)


def test_paper_hyperparameters_are_the_defaults():
    """The densification constants of App. A.1 (stored as text with their citation) are the
    oracle's constants and the defaults of the GPU path's parameter block."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "app_a1_densify.txt")
    vals = {}
    for ln in open(path):
        ln = ln.split("#", 1)[0].split()
        if ln:
            vals[ln[0]] = float(ln[1])
    assert (D.TAU_MIN, D.TAU_MAX, D.PERCENT_DENSE) == (
        vals["densify_grad_threshold_min"], vals["densify_grad_threshold_max"], vals["percent_dense"])
    from paper_2410_20686_gb300.densify import DensifyParams
    p = DensifyParams()
    assert (p.tau_min, p.tau_max, p.percent_dense) == (D.TAU_MIN, D.TAU_MAX, D.PERCENT_DENSE)
    assert vals["densify_until_iter"] < vals["iterations"]


@pytest.mark.parametrize("raw", [False, True])
def test_float32_selection_equals_the_fp64_rule_wherever_rounding_cannot_decide(raw):
    """``select`` decides in float32 (the kernel's precision, so that the GPU's decisions can be
    compared bit for bit); here it is pinned to the FP64 rule of Sec. 3.3 / App. A.1 applied to
    the same stored statistics: densify when the mean gradient reaches tau_mu at the mean
    1 - cos theta, clone when the largest scale is at most percent_dense x extent (split
    otherwise), prune below min_opacity or above max_scale. Every case whose FP64 margin exceeds
    float32 rounding (a relative 1e-5) must agree; near-threshold cases are drawn on purpose."""
    rng = np.random.default_rng(17 + raw)
    n = 400_000
    prm = D.DensifyParams(scene_extent=3.0, min_opacity=0.005, max_scale=0.05, raw_params=raw)
    count = rng.integers(0, 6, n).astype(np.uint32)
    emean = rng.uniform(0.0, 1.0, n)
    tau64 = D.tau(emean)
    # a third of the means straddle their threshold by under 1e-4 relative
    ratio = np.where(rng.uniform(size=n) < 0.33, 1.0 + rng.uniform(-1e-4, 1e-4, n), rng.uniform(0.2, 3.0, n))
    grad = (tau64 * ratio * count).astype(np.float32)
    elev = (emean * count).astype(np.float32)
    smax_target = np.where(rng.uniform(size=n) < 0.3, 3e-3 * (1 + rng.uniform(-1e-4, 1e-4, n)),
                           rng.uniform(5e-4, 0.08, n))
    scales = (smax_target[:, None] * rng.uniform(0.2, 1.0, (n, 3))).astype(np.float64)
    scales[np.arange(n), rng.integers(0, 3, n)] = smax_target
    opacity = np.where(rng.uniform(size=n) < 0.2, 0.005 * (1 + rng.uniform(-1e-4, 1e-4, n)), rng.uniform(1e-3, 1, n))
    s32 = (np.log(scales) if raw else scales).astype(np.float32)
    o32 = (np.log(opacity / (1 - opacity)) if raw else opacity).astype(np.float32)
    act = D.select(grad, elev, count, s32, o32, prm)

    # the FP64 rule on the stored (float32) values
    s64 = np.exp(s32.astype(np.float64)) if raw else s32.astype(np.float64)
    o64 = 1.0 / (1.0 + np.exp(-o32.astype(np.float64))) if raw else o32.astype(np.float64)
    seen = count > 0
    c = np.maximum(count, 1).astype(np.float64)
    g = grad.astype(np.float64) / c
    t = D.tau(elev.astype(np.float64) / c)
    smax = s64.max(axis=1)
    big_thr = prm.percent_dense * prm.scene_extent
    hot = seen & (g >= t)
    prune = (o64 < prm.min_opacity) | (smax > prm.max_scale)
    rule = np.where(prune, D.PRUNE, np.where(hot, np.where(smax > big_thr, D.SPLIT, D.CLONE), D.KEEP))
    # decisions float32 rounding can flip: any compared quantity within 1e-5 relative of its threshold
    eps = 1e-5
    near = seen & (np.abs(g - t) <= eps * t)
    near |= np.abs(smax - big_thr) <= eps * big_thr
    near |= np.abs(smax - prm.max_scale) <= eps * prm.max_scale
    near |= np.abs(o64 - prm.min_opacity) <= eps * prm.min_opacity
    assert near.mean() < 0.5 and (~near).sum() > 100_000
    assert np.array_equal(act[~near], rule[~near]), np.nonzero(act[~near] != rule[~near])[0][:5]
    # every kind of decision is exercised
    for a in (D.KEEP, D.CLONE, D.SPLIT, D.PRUNE):
        assert (rule[~near] == a).sum() > 1000
