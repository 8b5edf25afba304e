"""Pins of the FP64 oracle against what the ODGS paper and plain mathematics fix.

None of these tests re-types the oracle's formulas: each checks the oracle against an
independent route (finite differences of Eq. 4, closed forms, library routines, invariants,
brute-force enumeration), so that a dropped term, wrong sign, wrong index or transposed
operand in ``oracle/odgs_oracle.c`` fails at least one of them.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S

TAU = 2.0 * np.pi


def _view(W, H, R=None, t=None):
    return S.View(W, H, np.eye(3) if R is None else np.asarray(R, float),
                  np.zeros(3) if t is None else np.asarray(t, float))


def _params(means, scales, quats, opacity, sh):
    return O.Params(np.atleast_2d(means), np.atleast_2d(scales), np.atleast_2d(quats),
                    np.atleast_1d(opacity), np.asarray(sh, float).reshape(len(np.atleast_1d(opacity)), -1, 3))


def _pi_o(t, W, H):
    """ERP projection of Eq. 4, evaluated directly from the camera-space point."""
    phi = np.arctan2(t[0], t[2])
    theta = np.arctan2(-t[1], np.hypot(t[0], t[2]))
    return np.array([W / TAU * phi + W / 2.0, -H / np.pi * theta + H / 2.0])


def _dc_for(rgb):
    """SH degree-0 coefficient giving colour rgb (band-0 basis = 1 / (2 sqrt(pi)))."""
    return (np.asarray(rgb, float) - 0.5) * 2.0 * np.sqrt(np.pi)


def _dir_at_pixel(W, H, px, py, r):
    """Camera-space point at distance r whose ERP projection is (px, py) (inverse of Eq. 4)."""
    phi = (px - W / 2.0) * TAU / W
    theta = -(py - H / 2.0) * np.pi / H
    return r * np.array([np.cos(theta) * np.sin(phi), -np.sin(theta), np.cos(theta) * np.cos(phi)])


# ------------------------------------------------------------------ P1: Eq. 8 == d pi_o / d mu

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_p1_jacobian_equals_derivative_of_erp_projection(seed):
    rng = np.random.default_rng(seed)
    W, H = 2048, 1024
    n = 64
    means = rng.normal(size=(n, 3)) * 3
    p = _params(means, np.full((n, 3), 0.05), np.tile([1.0, 0, 0, 0], (n, 1)), np.full(n, 0.5), np.zeros((n, 1, 3)))
    pj = O.project(p, _view(W, H), O.Settings(sh_degree=0))
    for i in range(n):
        t = means[i]
        if np.hypot(t[0], t[2]) < 0.05 * np.linalg.norm(t):  # stay away from the poles
            continue
        if abs(abs(np.arctan2(t[0], t[2])) - np.pi) < 0.05:  # and from the seam
            continue
        Jfd = np.zeros((2, 3))
        for k in range(3):
            h = 1e-6 * np.linalg.norm(t)
            e = np.zeros(3); e[k] = h
            Jfd[:, k] = (_pi_o(t + e, W, H) - _pi_o(t - e, W, H)) / (2 * h)
        J = pj[i, O.PJ_J:O.PJ_J + 6].reshape(2, 3)
        np.testing.assert_allclose(J, Jfd, rtol=1e-7, atol=1e-7 * np.abs(Jfd).max())
        # the projected mean itself is Eq. 4
        np.testing.assert_allclose(pj[i, [O.PJ_U, O.PJ_V]], _pi_o(t, W, H), rtol=0, atol=1e-9)


def test_p1_jacobian_under_camera_rotation_pose():
    """With a rotated, translated camera J still equals the derivative of Eq. 4 w.r.t. the
    camera-space mean, and the oracle's (u, v) respond to world-space motion as J W."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(7)
    R = Rotation.random(random_state=3).as_matrix()
    tw = rng.normal(size=3)
    W, H = 1024, 512
    view = _view(W, H, R, tw)
    mu = np.array([0.7, -0.4, 2.2])
    st = O.Settings(sh_degree=0)
    base = _params(mu, [0.05] * 3, [1, 0, 0, 0], 0.5, np.zeros(3))
    pj = O.project(base, view, st)[0]
    J = pj[O.PJ_J:O.PJ_J + 6].reshape(2, 3)
    JW_fd = np.zeros((2, 3))
    for k in range(3):
        h = 1e-6
        e = np.zeros(3); e[k] = h
        up = O.project(_params(mu + e, [0.05] * 3, [1, 0, 0, 0], 0.5, np.zeros(3)), view, st)[0]
        dn = O.project(_params(mu - e, [0.05] * 3, [1, 0, 0, 0], 0.5, np.zeros(3)), view, st)[0]
        JW_fd[:, k] = (up[[O.PJ_U, O.PJ_V]] - dn[[O.PJ_U, O.PJ_V]]) / (2 * h)
    np.testing.assert_allclose(J @ R, JW_fd, rtol=1e-6, atol=1e-8)


# ------------------------------------------------------------------ P2: tangent-point reduction

def test_p2_reduces_to_perspective_jacobian_on_the_optical_axis():
    from scipy.spatial.transform import Rotation
    W, H = 1536, 768
    r = 3.7
    fx, fy = W / TAU, H / np.pi
    q = Rotation.random(random_state=11).as_quat()  # x, y, z, w
    quat = [q[3], q[0], q[1], q[2]]
    scales = [0.05, 0.2, 0.11]
    p = _params([0.0, 0.0, r], scales, quat, 0.8, np.zeros(3))
    for dil in (0.0, 0.3):
        pj = O.project(p, _view(W, H), O.Settings(sh_degree=0, dilation=dil))[0]
        # Eq. 1 at mu = (0, 0, r) with focal lengths W / 2 pi and H / pi
        Jp = np.array([[fx / r, 0, -fx * 0 / r ** 2], [0, fy / r, -fy * 0 / r ** 2]])
        np.testing.assert_allclose(pj[O.PJ_J:O.PJ_J + 6].reshape(2, 3), Jp, rtol=1e-12, atol=1e-12)
        Rm = Rotation.from_quat(q).as_matrix()
        Sig = Rm @ np.diag(np.square(scales)) @ Rm.T
        S2 = Jp @ Sig @ Jp.T + dil * np.eye(2)
        A, B, C = pj[O.PJ_COV2:O.PJ_COV2 + 3]
        np.testing.assert_allclose([[A, B], [B, C]], S2, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(pj[[O.PJ_U, O.PJ_V]], [W / 2, H / 2], atol=1e-12)


# ------------------------------------------------------------------ covariance pins

def test_world_covariance_matches_library_rotation():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(5)
    n = 32
    quats = rng.normal(size=(n, 4)) * rng.uniform(0.2, 3.0, size=(n, 1))  # un-normalised
    scales = np.exp(rng.normal(-2, 0.5, size=(n, 3)))
    means = rng.normal(size=(n, 3)) + [0, 0, 4]
    p = O.Params(means, scales, quats, np.full(n, 0.5), np.zeros((n, 1, 3)))
    pj = O.project(p, _view(512, 256), O.Settings(sh_degree=0))
    for i in range(n):
        qq = quats[i] / np.linalg.norm(quats[i])
        Rm = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        Sig = Rm @ np.diag(scales[i] ** 2) @ Rm.T
        c = pj[i, O.PJ_COV3:O.PJ_COV3 + 6]
        got = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        np.testing.assert_allclose(got, Sig, rtol=1e-12, atol=1e-15)


def test_cov2d_is_the_linearised_covariance_of_projected_sigma_points():
    """Sigma_2D (no dilation) equals the covariance of the ERP projection of a small 3D
    Gaussian to first order: push symmetric sigma points through Eq. 4 and compare."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(9)
    Rc = Rotation.random(random_state=21).as_matrix()
    view = _view(2000, 1000, Rc, [0.3, -0.2, 0.1])
    for trial in range(12):
        mu = rng.normal(size=3) * 3
        quat = rng.normal(size=4)
        scales = np.exp(rng.normal(-7, 0.5, size=3))  # tiny: the linearisation is exact to O(s^2)
        p = _params(mu, scales, quat, 0.5, np.zeros(3))
        pj = O.project(p, view, O.Settings(sh_degree=0, dilation=0.0))[0]
        if pj[O.PJ_VALID] == 0:
            continue
        t = Rc @ mu + view.t_wc
        if abs(abs(np.arctan2(t[0], t[2])) - np.pi) < 0.05:
            continue
        qq = quat / np.linalg.norm(quat)
        Rm = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        L = Rm @ np.diag(scales)
        pts = [mu + sgn * L[:, k] for k in range(3) for sgn in (1, -1)]
        uv = np.array([_pi_o(Rc @ x + view.t_wc, 2000, 1000) for x in pts])
        cov = (uv - uv.mean(0)).T @ (uv - uv.mean(0)) / 2.0
        A, B, C = pj[O.PJ_COV2:O.PJ_COV2 + 3]
        got = np.array([[A, B], [B, C]])
        np.testing.assert_allclose(got, cov, rtol=1e-4, atol=1e-4 * np.abs(cov).max())
        a, b, c = pj[O.PJ_CONIC:O.PJ_CONIC + 3]
        np.testing.assert_allclose(np.array([[a, b], [b, c]]) @ got, np.eye(2), atol=1e-9)


# ------------------------------------------------------------------ P3: single-Gaussian closed form

@pytest.mark.parametrize("theta_deg,phi_deg", [(0, 20), (60, -75), (85, 130), (-70, 179.9), (30, -179.9)])
@pytest.mark.parametrize("dil", [0.0, 0.3])
def test_p3_isotropic_gaussian_closed_form_image(theta_deg, phi_deg, dil):
    W, H = 256, 128
    r, sigma, o = 2.5, 0.04, 0.9
    th, ph = np.deg2rad(theta_deg), np.deg2rad(phi_deg)
    t = r * np.array([np.cos(th) * np.sin(ph), -np.sin(th), np.cos(th) * np.cos(ph)])
    rgb = np.array([0.8, 0.3, 0.55])
    bg = (0.1, 0.2, 0.05)
    p = _params(t, [sigma] * 3, [0.3, -0.2, 0.9, 0.1], o, _dc_for(rgb))
    img, T, _, _ = O.render(p, _view(W, H), O.Settings(sh_degree=0, dilation=dil, bg=bg))
    # closed form: rows of J_omni are orthogonal, so Sigma_2D is diagonal for isotropic Sigma
    suu = sigma ** 2 * (W / (TAU * r * np.cos(th))) ** 2 + dil
    svv = sigma ** 2 * (H / (np.pi * r)) ** 2 + dil
    u = W / TAU * ph + W / 2
    v = -H / np.pi * th + H / 2
    xs = np.arange(W) + 0.5
    ys = np.arange(H) + 0.5
    d = xs[None, :] - u
    dx = (d + W / 2) % W - W / 2
    dy = ys[:, None] - v
    a = o * np.exp(-0.5 * (dx ** 2 / suu + dy ** 2 / svv))
    a = np.minimum(a, 0.99)
    a = np.where(a < 1 / 255, 0.0, a)
    expect = rgb[:, None, None] * a[None] + (1 - a)[None] * np.asarray(bg)[:, None, None]
    np.testing.assert_allclose(img, expect, atol=1e-12)
    np.testing.assert_allclose(T, 1 - a, atol=1e-12)


# ------------------------------------------------------------------ P4: yaw = horizontal roll

@pytest.mark.parametrize("k", [1, 7, 64, 128])
def test_p4_yaw_by_whole_pixels_rolls_the_image(k):
    W, H = 256, 128
    sc = S.random_scene(150, W, H, seed=3, sh_degree=1, radius=(1.5, 5.0))
    p = O.Params.of(sc)
    st = O.Settings(sh_degree=1, bg=(0.05, 0.1, 0.2))
    base, _, _, _ = O.render(p, _view(W, H), st)
    psi = k * TAU / W
    c, s = np.cos(psi), np.sin(psi)
    R_cw = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    # the SH colour is view-direction dependent only through mean - camera centre, which a pure
    # rotation about the camera centre leaves unchanged
    rot, _, _, _ = O.render(p, _view(W, H, R_cw.T), st)
    np.testing.assert_allclose(rot, np.roll(base, -k, axis=2), atol=1e-10)


# ------------------------------------------------------------------ P5: blend algebra

def _stack_at_pixel(W, H, px, py, depths, opac, rgbs, scale=0.01):
    n = len(depths)
    means = np.array([_dir_at_pixel(W, H, px, py, d) for d in depths])
    sh = np.array([_dc_for(c) for c in rgbs]).reshape(n, 1, 3)
    return O.Params(means, np.full((n, 3), scale), np.tile([1.0, 0, 0, 0], (n, 1)), np.asarray(opac, float), sh)


def test_p5_two_layers_and_depth_swap():
    W, H = 64, 32
    px, py = 20.5, 11.5
    c1, c2 = np.array([0.9, 0.2, 0.1]), np.array([0.1, 0.6, 0.8])
    o1, o2 = 0.6, 0.7
    st = O.Settings(sh_degree=0, dilation=0.0)
    pix = [11 * W + 20]
    p = _stack_at_pixel(W, H, px, py, [2.0, 3.0], [o1, o2], [c1, c2])
    col, T, nc, _ = O.render(p, _view(W, H), st, pix=pix)
    np.testing.assert_allclose(col[0], c1 * o1 + c2 * o2 * (1 - o1), atol=1e-12)
    np.testing.assert_allclose(T[0], (1 - o1) * (1 - o2), atol=1e-12)
    assert nc[0] == 2
    q = _stack_at_pixel(W, H, px, py, [3.0, 2.0], [o1, o2], [c1, c2])
    col2, _, _, _ = O.render(q, _view(W, H), st, pix=pix)
    np.testing.assert_allclose(col[0] - col2[0], o1 * o2 * (c1 - c2), atol=1e-12)


def test_p5_termination_after_thirteen_half_layers():
    W, H = 64, 32
    st = O.Settings(sh_degree=0, dilation=0.0)
    c = np.array([0.3, 0.5, 0.7])
    p = _stack_at_pixel(W, H, 30.5, 9.5, np.linspace(2, 4, 20), [0.5] * 20, [c] * 20)
    col, T, nc, _ = O.render(p, _view(W, H), st, pix=[9 * W + 30])
    assert nc[0] == 13  # 0.5**13 >= 1e-4 > 0.5**14
    np.testing.assert_allclose(T[0], 0.5 ** 13, rtol=1e-12)
    np.testing.assert_allclose(col[0], c * (1 - 0.5 ** 13), atol=1e-12)


def test_p5_clamp_and_skip():
    W, H = 64, 32
    st = O.Settings(sh_degree=0, dilation=0.0)
    c = np.array([0.4, 0.4, 0.4])
    p = _stack_at_pixel(W, H, 10.5, 5.5, [2.0], [0.999], [c])
    col, T, _, _ = O.render(p, _view(W, H), st, pix=[5 * W + 10])
    np.testing.assert_allclose(T[0], 0.01, atol=1e-12)  # alpha clamped to 0.99
    q = _stack_at_pixel(W, H, 10.5, 5.5, [2.0], [0.99 / 255], [c])
    col, T, nc, _ = O.render(q, _view(W, H), st, pix=[5 * W + 10])
    assert nc[0] == 0 and T[0] == 1.0  # opacity below 1/255: culled


# ------------------------------------------------------------------ P6: brute force enumeration

def _brute_force(pj, W, H, st):
    """Eq. 3 by enumeration: all (Gaussian, pixel) alphas at once in global order, then the
    skip / clamp / termination rules applied with cumulative products."""
    vis = np.flatnonzero(pj[:, O.PJ_VALID] != 0)
    order = vis[np.lexsort((vis, pj[vis, O.PJ_KEY]))]
    xs = (np.arange(W) + 0.5)[None, None, :]
    ys = (np.arange(H) + 0.5)[None, :, None]
    u = pj[order, O.PJ_U][:, None, None]
    v = pj[order, O.PJ_V][:, None, None]
    a, b, c = (pj[order, O.PJ_CONIC + i][:, None, None] for i in range(3))
    dx = xs - u
    dx = dx - W * np.floor(dx / W + 0.5)
    dy = ys - v
    alpha = np.minimum(0.99, pj[order, O.PJ_OPAC][:, None, None] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy))
    alpha = np.where(alpha < 1 / 255, 0.0, alpha)
    T_after = np.cumprod(1 - alpha, axis=0)
    keep = np.cumprod(T_after >= 1e-4, axis=0).astype(bool)  # stop before the first T' < 1e-4
    alpha = np.where(keep, alpha, 0.0)
    T_before = np.cumprod(np.concatenate([np.ones((1, H, W)), 1 - alpha[:-1]], 0), axis=0)
    w = alpha * T_before
    rgb = pj[order][:, O.PJ_RGB:O.PJ_RGB + 3]
    img = np.einsum("kc,khw->chw", rgb, w)
    Tf = np.prod(1 - alpha, axis=0)
    return img + Tf[None] * np.asarray(st.bg)[:, None, None], Tf


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_p6_brute_force_tiny_scenes(seed):
    W, H = 32, 16
    sc = S.random_scene(16, W, H, seed=seed, sh_degree=2, radius=(0.8, 3.0), log_scale=(-1.6, 0.4))
    p = O.Params.of(sc)
    st = O.Settings(sh_degree=2, bg=(0.2, 0.1, 0.3))
    img, T, _, _ = O.render(p, sc.views[0], st)
    pj = O.project(p, sc.views[0], st)
    ref, Tf = _brute_force(pj, W, H, st)
    np.testing.assert_allclose(img, ref, atol=1e-12)
    np.testing.assert_allclose(T, Tf, atol=1e-12)


# ------------------------------------------------------------------ P7: SH basis

def _real_sh_from_scipy(l, m, polar, azim):
    from scipy.special import sph_harm_y
    if m == 0:
        return sph_harm_y(l, 0, polar, azim).real
    y = sph_harm_y(l, abs(m), polar, azim)
    return np.sqrt(2.0) * (-1) ** m * (y.real if m > 0 else y.imag)


def test_p7_sh_matches_library_complex_harmonics():
    rng = np.random.default_rng(0)
    for _ in range(40):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        Y = O.sh_eval(3, d)
        polar, azim = np.arccos(d[2]), np.arctan2(d[1], d[0])
        ref = [_real_sh_from_scipy(l, m, polar, azim) for l in range(4) for m in range(-l, l + 1)]
        np.testing.assert_allclose(Y, ref, atol=1e-13)
        # explicit low-order forms: Y00 = 1/(2 sqrt pi); (Y1-1, Y10, Y11) = sqrt(3/4pi) (y, z, x)
        np.testing.assert_allclose(Y[0], 0.5 / np.sqrt(np.pi), atol=1e-15)
        np.testing.assert_allclose(Y[1:4], np.sqrt(3 / (4 * np.pi)) * d[[1, 2, 0]], atol=1e-14)


def test_p7_sh_orthonormal_by_quadrature():
    xg, wg = np.polynomial.legendre.leggauss(12)  # exact for the degree <= 6 products in cos
    nphi = 16
    phis = np.arange(nphi) * TAU / nphi
    G = np.zeros((16, 16))
    for x, w in zip(xg, wg):
        s = np.sqrt(1 - x * x)
        for ph in phis:
            Y = O.sh_eval(3, [s * np.cos(ph), s * np.sin(ph), x])
            G += w * (TAU / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_colour_uses_world_direction_from_camera_centre():
    """Colour = max(0, sum sh Y(d) + 0.5) with d from the camera centre (not the origin)."""
    W, H = 64, 32
    c = np.array([1.0, -0.5, 2.0])
    view = _view(W, H, np.eye(3), -c)
    mu = np.array([2.0, 0.5, 5.0])
    rng = np.random.default_rng(1)
    sh = rng.normal(0, 0.3, size=(16, 3))
    p = _params(mu, [0.05] * 3, [1, 0, 0, 0], 0.5, sh)
    pj = O.project(p, view, O.Settings(sh_degree=3))[0]
    d = (mu - c) / np.linalg.norm(mu - c)
    Y = np.array([_real_sh_from_scipy(l, m, np.arccos(d[2]), np.arctan2(d[1], d[0]))
                  for l in range(4) for m in range(-l, l + 1)])
    np.testing.assert_allclose(pj[O.PJ_RGB:O.PJ_RGB + 3], np.maximum(0, Y @ sh + 0.5), atol=1e-13)


# ------------------------------------------------------------------ depth key, culling

def test_depth_key_is_ieee_single_in_fixed_order():
    rng = np.random.default_rng(4)
    from scipy.spatial.transform import Rotation
    R = Rotation.random(random_state=2).as_matrix().astype(np.float32)
    t = rng.normal(size=3).astype(np.float32)
    view = S.View(64, 32, R, t)
    for _ in range(200):
        mu = (rng.normal(size=3) * 4).astype(np.float32)
        f = np.float32
        tt = [f(f(f(f(R[i, 0] * mu[0]) + f(R[i, 1] * mu[1])) + f(R[i, 2] * mu[2])) + t[i]) for i in range(3)]
        q = f(f(f(tt[0] * tt[0]) + f(tt[1] * tt[1])) + f(tt[2] * tt[2]))
        assert O.depth_f32(mu, view) == np.sqrt(q, dtype=np.float32)


def test_spherical_shell_and_pole_culling():
    W, H = 64, 32
    st = O.Settings(sh_degree=0, r_near=0.5, r_far=10.0)
    means = np.array([[0, 0, 0.3], [0, 0, 12.0], [0, 0, 3.0], [0, -3.0, 1e-5], [0, 0, -3.0]])
    n = len(means)
    p = O.Params(means, np.full((n, 3), 0.05), np.tile([1.0, 0, 0, 0], (n, 1)), np.full(n, 0.5), np.zeros((n, 1, 3)))
    pj = O.project(p, _view(W, H), st)
    assert list(pj[:, O.PJ_VALID]) == [0, 0, 1, 0, 1]  # near, far, kept, pole, kept (behind)


# ------------------------------------------------------------------ P9: adjoint vs finite differences

def _tiny_scene(seed, deg):
    W, H = 40, 20
    sc = S.random_scene(10, W, H, seed=100 + seed, sh_degree=deg, radius=(1.0, 3.0), log_scale=(-1.8, 0.3))
    return sc, O.Params.of(sc)


@pytest.mark.parametrize("seed", [0, 1])
def test_p9_adjoint_matches_central_differences(seed):
    from scipy.spatial.transform import Rotation
    deg = 3
    sc, p = _tiny_scene(seed, deg)
    W, H = sc.views[0].width, sc.views[0].height
    R = Rotation.from_euler("xyz", [0.2, -0.7, 0.3]).as_matrix()
    view = _view(W, H, R, [0.1, -0.2, 0.05])
    st = O.Settings(sh_degree=deg, bg=(0.3, 0.1, 0.2))
    rng = np.random.default_rng(seed)
    wts = rng.normal(size=(3, H, W))
    g = O.backward(p, view, st, wts)
    _, _, nc0, margins = O.render(p, view, st)
    checked = 0
    for name, arr in p.arrays().items():
        for idx in rng.choice(arr.size, size=min(arr.size, 14), replace=False):
            h = 1e-6 * max(1.0, abs(arr.flat[idx]))
            # skip elements whose +-h perturbation flips a discrete decision somewhere
            x0 = arr.flat[idx]
            arr.flat[idx] = x0 + h
            _, _, ncp, _ = O.render(p, view, st)
            arr.flat[idx] = x0 - h
            _, _, ncm, _ = O.render(p, view, st)
            arr.flat[idx] = x0
            if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)):
                continue
            fd = O.fd_grad(p, view, st, wts, name, idx, h)
            ad = g[name].flat[idx]
            scale = max(abs(fd), 1e-3 * np.abs(g[name]).max(), 1e-9)
            assert abs(ad - fd) <= 2e-6 * scale + 1e-9, (name, idx, ad, fd)
            checked += 1
    assert checked > 40


@pytest.mark.parametrize("z", [2.0, -1.5])
def test_p9_adjoint_on_the_sh_axis_matches_central_differences(z):
    """A mean straight above or below the camera centre along world z, the axis on which the
    SH basis's angle chart (polar angle from +z, azimuth atan2(y, x)) is singular: the colour
    is smooth there, and the adjoint's mean gradient must equal central differences."""
    deg = 3
    W, H = 40, 20
    sc = S.random_scene(6, W, H, seed=131, sh_degree=deg, radius=(1.0, 3.0), log_scale=(-1.8, 0.3))
    p = O.Params.of(sc)
    from scipy.spatial.transform import Rotation
    R = Rotation.from_euler("xyz", [0.3, 0.2, -0.4]).as_matrix()
    cam = np.array([0.1, -0.2, 0.3])
    view = _view(W, H, R, -R @ cam)  # camera centre at cam
    p.means[0] = cam + np.array([0.0, 0.0, z])
    p.scales[0] = [0.2, 0.15, 0.25]
    p.opacity[0] = 0.9
    st = O.Settings(sh_degree=deg, bg=(0.3, 0.1, 0.2))
    assert O.project(p, view, st)[0, O.PJ_VALID] == 1
    wts = np.random.default_rng(7).normal(size=(3, H, W))
    g = O.backward(p, view, st, wts)
    assert np.all(np.isfinite(g["means"]))
    for j in range(3):
        fd = O.fd_grad(p, view, st, wts, "means", j, 1e-6)
        ad = g["means"][0, j]
        assert abs(ad - fd) <= 2e-6 * max(abs(fd), 1e-3 * np.abs(g["means"]).max()) + 1e-9, (j, ad, fd)


@pytest.mark.parametrize("mean,scale,R", [
    ([0.0, 0.0, -2.0], 0.2, None),        # straight behind: azimuth exactly 180 deg, on the seam
    ([1e-9, 0.3, -2.0], 0.2, None),       # a hair to one side of the seam
    ([-1e-9, 0.3, -2.0], 0.2, None),      # and to the other
    ([0.0, -2.0, 4e-4], 0.05, None),      # 0.011 deg from the upper pole (rho / r = 2e-4)
    ([0.0, 2.0, 1e-3], 0.05, None),       # 0.029 deg from the lower pole
    ([0.12, 0.1, 0.15], 0.02, None),      # just outside the near sphere (r = 0.22)
    ([0.0, 0.0, 2.0], 0.2, [[0, 0, 1], [0, 1, 0], [-1, 0, 0]]),  # rotated view, on the SH basis's axis
])
def test_p9_adjoint_at_special_points(mean, scale, R):
    """One anisotropic Gaussian at a point where the projection or the SH basis is special: the
    adjoint of every parameter element against central differences."""
    rng = np.random.default_rng(3)
    W, H = 64, 32
    quat = rng.normal(size=(1, 4))
    p = O.Params(np.array([mean], float), np.array([[scale, 0.6 * scale, 0.3 * scale]]), quat / np.linalg.norm(quat),
                 np.array([0.8]), rng.normal(scale=0.3, size=(1, 16, 3)))
    view = _view(W, H, R)
    st = O.Settings(sh_degree=3, bg=(0.2, 0.1, 0.3))
    assert O.project(p, view, st)[0, O.PJ_VALID] == 1
    wts = rng.normal(size=(3, H, W))
    g = O.backward(p, view, st, wts)
    _, _, nc0, _ = O.render(p, view, st)
    checked = 0
    for name, arr in p.arrays().items():
        for idx in range(arr.size):
            x0 = arr.flat[idx]
            h = 1e-6 * max(1.0, abs(x0))
            arr.flat[idx] = x0 + h
            _, _, ncp, _ = O.render(p, view, st)
            arr.flat[idx] = x0 - h
            _, _, ncm, _ = O.render(p, view, st)
            arr.flat[idx] = x0
            if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)):
                continue
            fd = O.fd_grad(p, view, st, wts, name, idx, h)
            scale_ = max(abs(fd), 1e-3 * np.abs(g[name]).max(), 1e-9)
            assert abs(g[name].flat[idx] - fd) <= 1e-5 * scale_, (name, idx, g[name].flat[idx], fd)
            checked += 1
    assert checked >= 50


def test_screen_space_gradients_match_finite_differences_of_the_blend():
    """dL/d(u, v, conic, opacity, rgb) of the reverse blend, checked by perturbing a single
    Gaussian's screen-space quantities through its 3D parameters is covered above; here the
    rgb part is isolated: with SH degree 0, dL/dk00 = Y00 * dL/drgb."""
    sc, p = _tiny_scene(5, 0)
    view = sc.views[0]
    st = O.Settings(sh_degree=0)
    wts = np.random.default_rng(3).normal(size=(3, view.height, view.width))
    g = O.backward(p, view, st, wts, want_g2=True)
    Y00 = 0.5 / np.sqrt(np.pi)
    pj = O.project(p, view, st)
    for i in range(p.n):
        for c in range(3):
            if pj[i, O.PJ_VALID] and not pj[i, O.PJ_CLAMP + c]:
                assert np.isclose(g["sh"][i, 0, c], Y00 * g["screen"][i, 6 + c], rtol=1e-12, atol=1e-15)


def test_eq12_first_row_agrees_and_second_row_is_sign_flipped():
    """Reading of App. A.3, Eq. 12: the derivative of J_omni (Eq. 8) w.r.t. the camera-space
    mean, taken here by central differences of the oracle's J, agrees with Eq. 12's
    coefficients of dL/dJ_(1,k) and has the opposite sign for every dL/dJ_(2,k) term."""
    W, H = 2048, 1024
    t = np.array([0.8, -0.6, 1.9])
    tx, ty, tz = t
    rho2 = tx * tx + tz * tz
    rho = np.sqrt(rho2)
    r2 = rho2 + ty * ty
    # Eq. 12 coefficients c[k][(i,j)] = printed factor multiplying dL/dJ_(i,j) in dL/dt_k
    c = {
        0: {(0, 0): -W / np.pi * tx * tz / rho2 ** 2, (0, 2): W / TAU * (tx * tx - tz * tz) / rho2 ** 2,
            (1, 0): H / np.pi * ty * (tz * tz * r2 - 2 * tx * tx * rho2) / (r2 ** 2 * rho ** 3),
            (1, 1): H / np.pi * tx * (r2 - 2 * ty * ty) / (r2 ** 2 * rho),
            (1, 2): -H / np.pi * tx * ty * tz * (2 * rho2 + r2) / (r2 ** 2 * rho ** 3)},
        1: {(1, 0): H / np.pi * tx * (r2 - 2 * ty * ty) / (r2 ** 2 * rho),
            (1, 1): 2 * H / np.pi * ty * rho / r2 ** 2,
            (1, 2): H / np.pi * tz * (r2 - 2 * ty * ty) / (r2 ** 2 * rho)},
        2: {(0, 0): W / TAU * (tx * tx - tz * tz) / rho2 ** 2, (0, 2): W / np.pi * tx * tz / rho2 ** 2,
            (1, 0): -H / np.pi * tx * ty * tz * (2 * rho2 + r2) / (r2 ** 2 * rho ** 3),
            (1, 1): H / np.pi * tz * (r2 - 2 * ty * ty) / (r2 ** 2 * rho),
            (1, 2): H / np.pi * ty * (tx * tx * r2 - 2 * tz * tz * rho2) / (r2 ** 2 * rho ** 3)},
    }
    st = O.Settings(sh_degree=0)
    for k in range(3):
        h = 1e-6
        e = np.zeros(3); e[k] = h
        Jp = O.project(_params(t + e, [0.05] * 3, [1, 0, 0, 0], 0.5, np.zeros(3)), _view(W, H), st)[0]
        Jm = O.project(_params(t - e, [0.05] * 3, [1, 0, 0, 0], 0.5, np.zeros(3)), _view(W, H), st)[0]
        dJ = ((Jp[O.PJ_J:O.PJ_J + 6] - Jm[O.PJ_J:O.PJ_J + 6]) / (2 * h)).reshape(2, 3)
        for (i, j), coef in c[k].items():
            sign = 1.0 if i == 0 else -1.0
            np.testing.assert_allclose(dJ[i, j], sign * coef, rtol=1e-6, atol=1e-6 * abs(coef) + 1e-9)


def test_chain_alone_reproduces_the_adjoint_from_its_screen_space_gradients():
    """orc_chain (the chain rule of App. A.3 applied to given screen-space gradients) is the second
    half of orc_backward: fed orc_backward's own screen-space gradients it returns the same
    parameter gradients, and fed zeros it returns zeros."""
    sc = S.random_scene(60, 64, 32, seed=13, sh_degree=2, log_scale=(-2.5, 0.6))
    p = O.Params.of(sc)
    st = O.Settings(sh_degree=2)
    v = S.yaw_view(64, 32, (0.1, 0.0, -0.2), 0.7)
    w = np.random.default_rng(13).normal(size=(3, 32, 64))
    full = O.backward(p, v, st, w, want_g2=True)
    assert np.abs(full["screen"]).max() > 0
    part = O.chain(p, v, st, full["screen"])
    for k in ("means", "scales", "quats", "opacity", "sh"):
        assert np.array_equal(part[k], full[k]), k
    zero = O.chain(p, v, st, np.zeros((p.n, 9)))
    assert all(not np.any(zero[k]) for k in zero)


def test_slice_form_conversion_of_screen_gradients_matches_finite_differences():
    """The tests compare the library's screen-space conic gradients, taken w.r.t. the slice form
    (a, beta, gamma) of the conic (a dx^2 + 2 b dx dy + c dy^2 = a (dx - beta dy)^2 + gamma dy^2),
    with the oracle's, taken w.r.t. the entries (a, b, c). The conversion is checked against
    central differences of a function of the entries through the slice parametrisation."""
    from tests.helpers import screen_slice_to_xy, screen_xy_to_slice
    rng = np.random.default_rng(5)
    n = 6
    pj = np.zeros((n, O.PJ_NFIELDS))
    a, beta, gam = rng.uniform(0.2, 3, n), rng.uniform(-2, 2, n), rng.uniform(0.1, 2, n)
    pj[:, O.PJ_CONIC], pj[:, O.PJ_CONIC + 1], pj[:, O.PJ_CONIC + 2] = a, -a * beta, gam + a * beta ** 2

    def loss(x, w):  # a smooth non-linear function of the entries
        return w[0] * np.sin(x[0]) + w[1] * x[1] ** 3 + w[2] * np.exp(0.3 * x[2]) + w[3] * x[0] * x[1]

    w = rng.normal(size=(n, 4))
    g_xy = np.zeros((n, 9))
    g_sl_fd = np.zeros((n, 9))
    for i in range(n):
        ent = lambda s: np.array([s[0], -s[0] * s[1], s[2] + s[0] * s[1] ** 2])  # noqa: E731
        x = ent((a[i], beta[i], gam[i]))
        g_xy[i, 2:5] = [w[i, 0] * np.cos(x[0]) + w[i, 3] * x[1], 3 * w[i, 1] * x[1] ** 2 + w[i, 3] * x[0],
                        0.3 * w[i, 2] * np.exp(0.3 * x[2])]
        for k in range(3):
            s0 = np.array([a[i], beta[i], gam[i]])
            h = 1e-6
            sp, sm = s0.copy(), s0.copy()
            sp[k] += h
            sm[k] -= h
            g_sl_fd[i, 2 + k] = (loss(ent(sp), w[i]) - loss(ent(sm), w[i])) / (2 * h)
    g_sl = screen_xy_to_slice(g_xy, pj)
    assert np.allclose(g_sl[:, 2:5], g_sl_fd[:, 2:5], rtol=1e-6, atol=1e-8)
    assert np.allclose(screen_slice_to_xy(g_sl, pj), g_xy, rtol=1e-12, atol=1e-12)


def test_absolute_contribution_sums_bound_the_screen_gradients():
    """The adjoint's optional sums of absolute per-pixel contributions bound the screen-space
    gradients (|sum| <= sum |.|), and equal them for the colour gradients of a single Gaussian
    under positive weights (every contribution alpha T g is then positive)."""
    sc = S.random_scene(40, 64, 32, seed=21, sh_degree=1, log_scale=(-2.5, 0.5))
    p = O.Params.of(sc)
    st = O.Settings(sh_degree=1)
    w = np.random.default_rng(21).normal(size=(3, 32, 64))
    g = O.backward(p, sc.views[0], st, w, want_g2=True, want_abs=True)
    assert np.all(g["screen_abs"] >= np.abs(g["screen"]) * (1 - 1e-12))
    assert g["screen_abs"].max() > 0
    one = O.Params(p.means[:1], p.scales[:1], p.quats[:1], p.opacity[:1], p.sh[:1])
    one.means[0] = [0.2, 0.1, 2.0]
    g1 = O.backward(one, sc.views[0], st, np.abs(w), want_g2=True, want_abs=True)
    assert g1["screen"][0, 6] > 0
    assert np.allclose(g1["screen_abs"][0, 6:9], g1["screen"][0, 6:9], rtol=1e-12)
