"""Seeded synthetic ERP scenes shared by the CUDA path, its tests, the bench and the oracle.

This module only draws random inputs. It holds none of the rasterizer's arithmetic: every value
here is a sample of a stated distribution (means, activated scales, raw quaternions, activated
opacities, SH coefficients, camera poses, target images). Draws are made in float64 with
``numpy.random.Generator(PCG64(20241027 + config))`` and stored as float32, so the CUDA path
and the FP64 oracle read bit-identical inputs.

The scene shapes stand in for the paper's omnidirectional captures (Sec. 4.1): egocentric
scenes (camera rotating in place or on a short path, ~2000x1000 ERP) and roaming scenes
(2048x1024 and larger, long camera paths). None of the datasets' images or poses are used.

Conventions (Sec. 3.2): camera axes follow OpenCV (x right, y down, z forward); a view maps a
world point to camera space as ``t = R_wc @ mu + t_wc``; quaternions are (w, x, y, z) and
un-normalised; scales and opacities are already activated; SH coefficients are laid out
``[N, K, 3]`` with ``K = (degree + 1) ** 2`` in the order ``l = 0..3, m = -l..l``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20241027


@dataclass
class View:
    width: int
    height: int
    R_wc: np.ndarray  # [3, 3] float32, world -> camera rotation (row-major)
    t_wc: np.ndarray  # [3] float32
    model: int = 0    # 0: ERP; 1: pinhole with focal lengths fx, fy and principal point cx, cy (pixels)
    fx: float = 0.0
    fy: float = 0.0
    cx: float = 0.0
    cy: float = 0.0

    @staticmethod
    def identity(width: int, height: int, center=(0.0, 0.0, 0.0)) -> "View":
        c = np.asarray(center, dtype=np.float64)
        return View(width, height, np.eye(3, dtype=np.float32), (-c).astype(np.float32))


@dataclass
class Scene:
    means: np.ndarray     # [N, 3] float32
    scales: np.ndarray    # [N, 3] float32, > 0
    quats: np.ndarray     # [N, 4] float32, (w, x, y, z), not normalised
    opacity: np.ndarray   # [N] float32 in (0, 1)
    sh: np.ndarray        # [N, K, 3] float32
    sh_degree: int
    views: list = field(default_factory=list)
    name: str = "custom"
    recompute_lists: bool = False

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity[idx].copy(), self.sh[idx].copy(), self.sh_degree,
                     list(self.views), self.name, self.recompute_lists)


def _rng(offset: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + offset))


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _common(rng, n, log_mu, log_sigma, sh_degree, dc_mode="normal"):
    """Scales, rotations, opacities and SH coefficients (distributions per config)."""
    scales = np.exp(rng.normal(log_mu, log_sigma, size=(n, 3)))
    quats = rng.normal(0.0, 1.0, size=(n, 4))
    opacity = _sigmoid(rng.normal(0.0, 1.0, size=n))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    if dc_mode == "rgb":
        # DC drawn so that the DC-only colour is uniform in [0, 1]: the band-0 basis
        # function is the constant 1 / (2 sqrt(pi)), so k00 = (rgb - 0.5) * 2 sqrt(pi).
        sh[:, 0, :] = (rng.uniform(0.0, 1.0, size=(n, 3)) - 0.5) * (2.0 * np.sqrt(np.pi))
    else:
        sh[:, 0, :] = rng.normal(0.5, 0.2, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, k - 1, 3))
    return scales, quats, opacity, sh


def _pack(means, scales, quats, opacity, sh, deg, views, name, recompute=False) -> Scene:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f(means), f(scales), f(quats), f(opacity), f(sh), deg, views, name, recompute)


def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def pinhole_view(width, height, fx, fy, cx=None, cy=None, R_wc=None, t_wc=None) -> View:
    """Pinhole camera: pixel (i, j) is sampled at (i + 1/2, j + 1/2) of the plane
    u = fx tx / tz + cx, v = fy ty / tz + cy (principal point at the image centre by default)."""
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    return View(width, height, np.eye(3, dtype=np.float32) if R_wc is None else np.asarray(R_wc, np.float32),
                np.zeros(3, np.float32) if t_wc is None else np.asarray(t_wc, np.float32), 1, f32(fx), f32(fy),
                f32(width / 2.0 if cx is None else cx), f32(height / 2.0 if cy is None else cy))


# camera -> world rotations of the six cube faces (camera axes: x right, y down, z forward)
_CUBE_FACES = {
    "+z": np.eye(3),
    "-z": np.array([[-1.0, 0, 0], [0, 1, 0], [0, 0, -1]]),
    "+x": np.array([[0.0, 0, 1], [0, 1, 0], [-1, 0, 0]]),
    "-x": np.array([[0.0, 0, -1], [0, 1, 0], [1, 0, 0]]),
    "+y": np.array([[1.0, 0, 0], [0, 0, 1], [0, -1, 0]]),
    "-y": np.array([[1.0, 0, 0], [0, 0, -1], [0, 1, 0]]),
}


def cubemap_views(face, center=(0.0, 0.0, 0.0)):
    """Six 90-degree pinhole views (face x face pixels) looking along +z, -z, +x, -x, +y, -y of the
    world from ``center``: the 3DGS(P) cubemap rendering of a 360-degree scene."""
    c = np.asarray(center, dtype=np.float64)
    out = []
    for name in ("+z", "-z", "+x", "-x", "+y", "-y"):
        R_wc = _CUBE_FACES[name].T
        out.append(pinhole_view(face, face, face / 2.0, face / 2.0, R_wc=R_wc, t_wc=-R_wc @ c))
    return out


def yaw_view(width, height, center, yaw) -> View:
    """Camera at ``center`` rotated by ``yaw`` about the (down-pointing) y axis."""
    c, s = np.cos(yaw), np.sin(yaw)
    R_cw = np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])  # camera -> world
    R_wc = R_cw.T
    t_wc = -R_wc @ np.asarray(center, dtype=np.float64)
    return View(width, height, R_wc.astype(np.float32), t_wc.astype(np.float32))


# --------------------------------------------------------------------------------------
# The five workload configurations
# --------------------------------------------------------------------------------------

def config0() -> Scene:
    """1,000 Gaussians in a spherical shell r in [1, 5] (uniform by volume), SH degree 0,
    one 256x128 view with identity pose."""
    rng = _rng(0)
    n = 1000
    r = (1.0 + rng.uniform(size=n) * 124.0) ** (1.0 / 3.0)
    means = _unit_vectors(rng, n) * r[:, None]
    scales, quats, opacity, sh = _common(rng, n, -3.0, 0.5, 0, dc_mode="rgb")
    return _pack(means, scales, quats, opacity, sh, 0, [View.identity(256, 128)], "config0")


def config1() -> Scene:
    """100k Gaussians uniform in a 10x4x10 m box around the camera, SH degree 3, 1024x512."""
    rng = _rng(1)
    n = 100_000
    means = rng.uniform([-5, -2, -5], [5, 2, 5], size=(n, 3))
    scales, quats, opacity, sh = _common(rng, n, -3.0, 0.5, 3)
    return _pack(means, scales, quats, opacity, sh, 3, [View.identity(1024, 512)], "config1")


def _pole_points(rng, n, half_y, min_elev_deg):
    """Points of a uniform-in-room draw conditioned on |elevation| >= min_elev_deg (half per
    pole). Given |y| the accepted (x, z) set is a disk of radius |y| / tan(min_elev), so the
    conditional law is: |y| with density proportional to y^2, then uniform in the disk."""
    ay = half_y * rng.uniform(size=n) ** (1.0 / 3.0)
    sign = np.where(np.arange(n) < n // 2, -1.0, 1.0)
    rad = ay / np.tan(np.deg2rad(min_elev_deg)) * np.sqrt(rng.uniform(size=n))
    ang = rng.uniform(0.0, 2.0 * np.pi, size=n)
    return np.stack([rad * np.cos(ang), sign * ay, rad * np.sin(ang)], axis=1)


def _seam_points(rng, n, half_x, half_y, half_z, max_dev_deg):
    """Points of a uniform-in-room draw conditioned on |azimuth| >= 180 - max_dev_deg, i.e.
    behind the camera in a thin wedge around the -z axis: |z| has density proportional to
    |z| and x is uniform across the wedge."""
    az = half_z * np.sqrt(rng.uniform(size=n))
    w = az * np.tan(np.deg2rad(max_dev_deg))
    x = rng.uniform(-1.0, 1.0, size=n) * np.minimum(w, half_x)
    y = rng.uniform(-half_y, half_y, size=n)
    return np.stack([x, y, -az], axis=1)


def config2(n: int = 1_000_000, width: int = 2048) -> Scene:
    """1M Gaussians: 20% within 10 deg of the poles, 20% within 5 deg of the +-180 deg
    longitude seam, 60% uniform in a 20x5x20 m room; log-scales N(-4, 0.7); SH degree 3;
    one 2048x1024 view with identity pose."""
    rng = _rng(2)
    n_pole = n // 5
    n_seam = n // 5
    n_room = n - n_pole - n_seam
    pole = _pole_points(rng, n_pole, 2.5, 80.0)
    seam = _seam_points(rng, n_seam, 10.0, 2.5, 10.0, 5.0)
    room = rng.uniform([-10, -2.5, -10], [10, 2.5, 10], size=(n_room, 3))
    means = np.concatenate([pole, seam, room], axis=0)
    perm = rng.permutation(n)
    means = means[perm]
    scales, quats, opacity, sh = _common(rng, n, -4.0, 0.7, 3)
    return _pack(means, scales, quats, opacity, sh, 3, [View.identity(width, width // 2)],
                 "config2")


def config3(n: int = 500_000, sizes=None) -> Scene:
    """500k shared Gaussians uniform in the 20x5x20 m room, SH degree 3, and 16 views of
    mixed size (4x512x256, 4x1024x512, 8x2048x1024) whose centres sit on a 3 m straight path
    with +-5 cm jitter and uniformly random yaw."""
    rng = _rng(3)
    means = rng.uniform([-10, -2.5, -10], [10, 2.5, 10], size=(n, 3))
    scales, quats, opacity, sh = _common(rng, n, -4.0, 0.7, 3)
    if sizes is None:
        sizes = [(512, 256)] * 4 + [(1024, 512)] * 4 + [(2048, 1024)] * 8
    views = []
    m = len(sizes)
    for i, (w, h) in enumerate(sizes):
        c = np.array([-1.5 + 3.0 * i / max(m - 1, 1), 0.0, 0.0]) + rng.uniform(-0.05, 0.05, 3)
        views.append(yaw_view(w, h, c, rng.uniform(-np.pi, np.pi)))
    return _pack(means, scales, quats, opacity, sh, 3, views, "config3")


def config4(n: int = 3_000_000, n_views: int = 8, width: int = 4096) -> Scene:
    """3M Gaussians along a 50x3x4 m corridor (70% uniform, 30% in 100 isotropic clusters of
    sigma 0.3 m), SH degree 3, 8 views of 4096x2048 stepping every 6 m, lists recomputed in
    the backward pass."""
    rng = _rng(4)
    lo = np.array([0.0, -1.5, -2.0])
    hi = np.array([50.0, 1.5, 2.0])
    n_cl = int(round(0.3 * n))
    n_un = n - n_cl
    uni = rng.uniform(lo, hi, size=(n_un, 3))
    centres = rng.uniform(lo, hi, size=(100, 3))
    lab = rng.integers(0, 100, size=n_cl)
    cl = centres[lab] + rng.normal(0.0, 0.3, size=(n_cl, 3))
    bad = np.any((cl < lo) | (cl > hi), axis=1)
    while bad.any():  # rejection-clip: redraw points that left the corridor
        cl[bad] = centres[lab[bad]] + rng.normal(0.0, 0.3, size=(int(bad.sum()), 3))
        bad = np.any((cl < lo) | (cl > hi), axis=1)
    means = np.concatenate([uni, cl], axis=0)[rng.permutation(n)]
    scales, quats, opacity, sh = _common(rng, n, -4.0, 0.7, 3)
    views = [View.identity(width, width // 2, (4.0 + 6.0 * k, 0.0, 0.0)) for k in range(n_views)]
    return _pack(means, scales, quats, opacity, sh, 3, views, "config4", recompute=True)


CONFIGS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}


def target_images(scene: Scene, cfg: int = 0):
    """Seeded uniform-noise target image per view, [3, H, W] float32."""
    rng = _rng(cfg + 1)
    return [rng.uniform(0.0, 1.0, size=(3, v.height, v.width)).astype(np.float32)
            for v in scene.views]


def random_scene(n, width, height, seed, sh_degree=3, radius=(1.0, 6.0), log_scale=(-3.0, 0.5),
                 views=None) -> Scene:
    """Small scene for parity tests: means uniform by volume in a shell around the origin."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1000 + seed))
    r0, r1 = radius
    r = (r0 ** 3 + rng.uniform(size=n) * (r1 ** 3 - r0 ** 3)) ** (1.0 / 3.0)
    means = _unit_vectors(rng, n) * r[:, None]
    scales, quats, opacity, sh = _common(rng, n, log_scale[0], log_scale[1], sh_degree)
    if views is None:
        views = [View.identity(width, height)]
    return _pack(means, scales, quats, opacity, sh, sh_degree, views, f"random{seed}")


def sample_pixels(width, height, n_random, tiles, seed, tile=16):
    """Seeded pixel sample: ``n_random`` uniform pixels plus every pixel of the listed
    ``(tile_x, tile_y)`` tiles. Returns sorted unique flat indices y * width + x (int32)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 5000 + seed))
    idx = [rng.integers(0, width * height, size=n_random)]
    for tx, ty in tiles:
        ys, xs = np.meshgrid(np.arange(ty * tile, min((ty + 1) * tile, height)),
                             np.arange(tx * tile, min((tx + 1) * tile, width)), indexing="ij")
        idx.append((ys * width + xs).ravel())
    return np.unique(np.concatenate(idx)).astype(np.int32)


def stress_tiles(width, height, tile=16):
    """Eight tiles touching the poles and the longitude seam (Sec. 3.2's stretch regions)."""
    tx_n = width // tile
    ty_n = (height + tile - 1) // tile
    return [(0, 0), (tx_n - 1, 0), (tx_n // 2, 0), (0, ty_n - 1), (tx_n - 1, ty_n - 1),
            (tx_n // 2, ty_n - 1), (0, ty_n // 2), (tx_n - 1, ty_n // 2)]
