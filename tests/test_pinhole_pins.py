"""Pins of the oracle's pinhole (perspective, Eq. 1) camera model, the 3DGS(P) baseline's
projection: Jacobian, covariance, the tangent-point equivalence with the ERP model (P2 at image
level), culling, the depth key, cube faces and the adjoint."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S


def _params(means, scales, quats, opacity, sh):
    return O.Params(np.atleast_2d(means), np.atleast_2d(scales), np.atleast_2d(quats),
                    np.atleast_1d(opacity), np.asarray(sh, float).reshape(len(np.atleast_1d(opacity)), -1, 3))


def _pi_p(t, v):
    return np.array([v.fx * t[0] / t[2] + v.cx, v.fy * t[1] / t[2] + v.cy])


def test_jacobian_is_the_derivative_of_the_pinhole_projection():
    rng = np.random.default_rng(0)
    R = Rotation.random(random_state=4).as_matrix().astype(np.float32)
    v = S.pinhole_view(640, 480, 500.0, 480.0, 300.0, 250.0, R, [0.2, -0.1, 0.3])
    checked = 0
    for _ in range(300):
        mu = rng.normal(size=3) * 2
        p = _params(mu, [0.01] * 3, [1, 0, 0, 0], 0.5, np.zeros(3))
        pj = O.project(p, v, O.Settings(sh_degree=0))[0]
        if pj[O.PJ_VALID] == 0:
            continue
        t = pj[O.PJ_T:O.PJ_T + 3]
        J = pj[O.PJ_J:O.PJ_J + 6].reshape(2, 3)
        h = 1e-6
        fd = np.stack([(_pi_p(t + h * e, v) - _pi_p(t - h * e, v)) / (2 * h) for e in np.eye(3)], 1)
        np.testing.assert_allclose(J, fd, rtol=1e-7, atol=1e-7 * np.abs(fd).max())
        np.testing.assert_allclose(pj[O.PJ_U:O.PJ_V + 1], _pi_p(t, v), rtol=1e-13)
        checked += 1
    assert checked > 10


def test_cov2d_is_the_linearised_covariance_of_projected_sigma_points():
    rng = np.random.default_rng(1)
    R = Rotation.random(random_state=5).as_matrix().astype(np.float32)
    v = S.pinhole_view(800, 600, 600.0, 610.0, R_wc=R, t_wc=[0.0, 0.1, -0.2])
    checked = 0
    for _ in range(400):
        mu = rng.normal(size=3) * 2
        quat = rng.normal(size=4)
        scales = np.exp(rng.normal(-7, 0.5, size=3))
        p = _params(mu, scales, quat, 0.5, np.zeros(3))
        pj = O.project(p, v, O.Settings(sh_degree=0, dilation=0.0))[0]
        if pj[O.PJ_VALID] == 0:
            continue
        qq = quat / np.linalg.norm(quat)
        L = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix() @ np.diag(scales)
        pts = [mu + sgn * L[:, k] for k in range(3) for sgn in (1, -1)]
        uv = np.array([_pi_p(v.R_wc.astype(np.float64) @ x + v.t_wc, v) for x in pts])
        cov = (uv - uv.mean(0)).T @ (uv - uv.mean(0)) / 2.0
        A, B, C = pj[O.PJ_COV2:O.PJ_COV2 + 3]
        np.testing.assert_allclose(np.array([[A, B], [B, C]]), cov, rtol=1e-4, atol=1e-4 * np.abs(cov).max())
        checked += 1
    assert checked > 10


@pytest.mark.parametrize("sigma,dil", [(0.01, 0.3), (0.03, 0.0)])
def test_p2_erp_and_pinhole_images_agree_at_the_tangent_point(sigma, dil):
    # a Gaussian on the optical axis: both models put its mean at the image centre and their
    # Jacobians coincide (f = W / 2 pi, H / pi), so the affine splats are the same image
    W, H = 256, 128
    rgb = np.array([0.8, 0.3, 0.55])
    p = _params([0.0, 0.0, 2.0], [sigma] * 3, [0.9, 0.1, -0.3, 0.2], 0.85, (rgb - 0.5) * 2 * np.sqrt(np.pi))
    st = O.Settings(sh_degree=0, dilation=dil, bg=(0.1, 0.0, 0.2))
    erp, Te, _, _ = O.render(p, S.View.identity(W, H), st)
    # focal lengths in float64 (pinhole_view rounds them to float32, 3e-8 away from W / 2 pi)
    pv = S.View(W, H, np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 1, W / (2 * np.pi), H / np.pi,
                W / 2.0, H / 2.0)
    pin, Tp, _, _ = O.render(p, pv, st)
    np.testing.assert_allclose(pin, erp, atol=1e-12)
    np.testing.assert_allclose(Tp, Te, atol=1e-12)
    assert (Te < 1.0).sum() > 4


def test_culling_near_far_behind_and_outside_the_guard_band():
    v = S.pinhole_view(200, 100, 150.0, 150.0)
    st = O.Settings(sh_degree=0, r_near=0.2, r_far=50.0)
    pts = {
        "in front": ([0.0, 0.0, 3.0], True),
        "behind": ([0.0, 0.0, -3.0], False),
        "too near": ([0.0, 0.0, 0.1], False),
        "too far": ([0.0, 0.0, 60.0], False),
        "just outside the image": ([0.76, 0.0, 1.0], True),   # u = 214 < 1.3 W = 260
        "beyond the guard band": ([1.2, 0.0, 1.0], False),    # u = 280
        "beyond the guard band in v": ([0.0, 0.6, 1.0], False),  # v = 140 > 130
    }
    for name, (t, visible) in pts.items():
        p = _params(t, [0.01] * 3, [1, 0, 0, 0], 0.5, np.zeros(3))
        assert (O.project(p, v, st)[0, O.PJ_VALID] > 0) == visible, name


def test_depth_key_is_the_float32_z_in_fixed_order():
    R = Rotation.from_euler("xyz", [0.3, -0.2, 0.5]).as_matrix().astype(np.float32)
    t = np.array([0.1, -0.3, 0.25], np.float32)
    v = S.pinhole_view(64, 64, 50.0, 50.0, R_wc=R, t_wc=t)
    mu = np.array([0.7, -0.4, 3.1], np.float32)
    f = np.float32
    z = (f(R[2, 0]) * mu[0] + f(R[2, 1]) * mu[1]) + f(R[2, 2]) * mu[2]
    z = f(z + t[2])
    assert O.depth_f32(mu.astype(np.float64), v) == z


def test_cube_faces_centre_points_on_the_axes():
    views = S.cubemap_views(64)
    st = O.Settings(sh_degree=0)
    axes = [[0, 0, 5], [0, 0, -5], [5, 0, 0], [-5, 0, 0], [0, 5, 0], [0, -5, 0]]
    for k, a in enumerate(axes):
        p = _params(a, [0.01] * 3, [1, 0, 0, 0], 0.5, np.zeros(3))
        for j, v in enumerate(views):
            pj = O.project(p, v, st)[0]
            if j == k:
                assert pj[O.PJ_VALID] > 0
                np.testing.assert_allclose(pj[O.PJ_U:O.PJ_V + 1], [32.0, 32.0], atol=1e-12)
            else:
                assert pj[O.PJ_VALID] == 0  # behind the face or beyond its guard band


@pytest.mark.parametrize("seed", [0, 1])
def test_pinhole_adjoint_matches_central_differences(seed):
    W, H = 40, 30
    sc = S.random_scene(10, W, H, seed=200 + seed, sh_degree=3, radius=(1.0, 3.0), log_scale=(-1.8, 0.3))
    p = O.Params.of(sc)
    R = Rotation.from_euler("xyz", [0.1, 0.2, -0.1]).as_matrix()
    # a wide-angle camera so that most Gaussians of the shell are in front and in view
    v = S.pinhole_view(W, H, 12.0, 12.0, R_wc=R, t_wc=[0.0, 0.0, 3.5])
    st = O.Settings(sh_degree=3, bg=(0.3, 0.1, 0.2))
    rng = np.random.default_rng(seed)
    wts = rng.normal(size=(3, H, W))
    g = O.backward(p, v, st, wts)
    _, _, nc0, _ = O.render(p, v, st)
    checked = 0
    for name, arr in p.arrays().items():
        for idx in rng.choice(arr.size, size=min(arr.size, 14), replace=False):
            h = 1e-6 * max(1.0, abs(arr.flat[idx]))
            x0 = arr.flat[idx]
            arr.flat[idx] = x0 + h
            _, _, ncp, _ = O.render(p, v, st)
            arr.flat[idx] = x0 - h
            _, _, ncm, _ = O.render(p, v, st)
            arr.flat[idx] = x0
            if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)):
                continue
            fd = O.fd_grad(p, v, st, wts, name, idx, h)
            ad = g[name].flat[idx]
            scale = max(abs(fd), 1e-3 * np.abs(g[name]).max(), 1e-9)
            assert abs(ad - fd) <= 2e-6 * scale + 1e-9, (name, idx, ad, fd)
            checked += 1
    assert checked > 30
