"""ctypes binding of ``odgs_oracle.c`` plus the finite-difference driver.

TEST INFRASTRUCTURE ONLY: see the package docstring. All arithmetic of the method lives in
``odgs_oracle.c`` (FP64); this file marshals numpy arrays and runs central differences.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "odgs_oracle.c")
_LIB = os.path.join(_HERE, "libodgs_oracle.so")

# per-Gaussian projection record fields (mirror of the enum in odgs_oracle.c)
PJ_VALID, PJ_KEY, PJ_DEPTH, PJ_R, PJ_PHI, PJ_THETA, PJ_U, PJ_V = range(8)
PJ_T, PJ_J, PJ_COV3, PJ_COV2, PJ_CONIC, PJ_RGB, PJ_CLAMP, PJ_DIR, PJ_OPAC = 8, 11, 17, 23, 26, 29, 32, 35, 38
PJ_NFIELDS = 40
G2_NAMES = ("u", "v", "conic_a", "conic_b", "conic_c", "opacity", "r", "g", "b")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _View(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("R", C.c_double * 9), ("t", C.c_double * 3),
                ("model", C.c_int), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double)]


class _Settings(C.Structure):
    _fields_ = [("sh_degree", C.c_int), ("sh_coeffs", C.c_int), ("dilation", C.c_double),
                ("r_near", C.c_double), ("r_far", C.c_double), ("bg", C.c_double * 3),
                ("pix_offset", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        vp = C.POINTER(_View)
        sp = C.POINTER(_Settings)
        L.orc_project.argtypes = [C.c_int, dp, dp, dp, dp, dp, vp, sp, dp]
        L.orc_render.argtypes = [C.c_int, dp, dp, dp, dp, dp, vp, sp, C.c_int, ip, dp, dp, ip, dp]
        L.orc_backward.argtypes = [C.c_int, dp, dp, dp, dp, dp, vp, sp, C.c_int, ip, dp,
                                   dp, dp, dp, dp, dp, dp, dp]
        L.orc_chain.argtypes = [C.c_int, dp, dp, dp, dp, dp, vp, sp, dp, dp, dp, dp, dp, dp]
        L.orc_sh_eval.argtypes = [C.c_int, dp, dp]
        L.orc_depth_f32.argtypes = [dp, vp]
        L.orc_depth_f32.restype = C.c_float
        L.orc_num_threads.restype = C.c_int
        L.orc_pj_nfields.restype = C.c_int
        assert L.orc_pj_nfields() == PJ_NFIELDS
        _lib = L
    return _lib


@dataclass
class Settings:
    sh_degree: int = 3
    dilation: float = 0.3
    r_near: float = 0.2
    r_far: float = 1e4
    bg: tuple = (0.0, 0.0, 0.0)
    pix_offset: float = 0.5


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def _cview(view):
    v = _View()
    v.width, v.height = int(view.width), int(view.height)
    v.R[:] = [float(x) for x in np.asarray(view.R_wc, dtype=np.float64).ravel()]
    v.t[:] = [float(x) for x in np.asarray(view.t_wc, dtype=np.float64).ravel()]
    v.model = int(getattr(view, "model", 0))
    v.fx, v.fy, v.cx, v.cy = (float(getattr(view, k, 0.0)) for k in ("fx", "fy", "cx", "cy"))
    return v


def _csettings(st: Settings, sh):
    s = _Settings()
    s.sh_degree = st.sh_degree
    s.sh_coeffs = int(sh.shape[1])
    s.dilation, s.r_near, s.r_far = st.dilation, st.r_near, st.r_far
    s.bg[:] = list(st.bg)
    s.pix_offset = st.pix_offset
    return s


class Params:
    """FP64 copies of the Gaussian parameters (upcast from the float32 scene)."""

    def __init__(self, means, scales, quats, opacity, sh):
        self.means, self.scales, self.quats = _d(means), _d(scales), _d(quats)
        self.opacity, self.sh = _d(opacity), _d(sh)

    @staticmethod
    def of(scene):
        return Params(scene.means, scene.scales, scene.quats, scene.opacity, scene.sh)

    @property
    def n(self):
        return self.means.shape[0]

    def arrays(self):
        return dict(means=self.means, scales=self.scales, quats=self.quats,
                    opacity=self.opacity, sh=self.sh)

    def copy(self):
        return Params(self.means.copy(), self.scales.copy(), self.quats.copy(),
                      self.opacity.copy(), self.sh.copy())


def project(p: Params, view, st: Settings):
    """Per-Gaussian projection records [N, PJ_NFIELDS] (float64)."""
    L = lib()
    out = np.zeros((max(p.n, 1), PJ_NFIELDS))
    L.orc_project(p.n, _ptr(p.means), _ptr(p.scales), _ptr(p.quats), _ptr(p.opacity), _ptr(p.sh),
                  C.byref(_cview(view)), C.byref(_csettings(st, p.sh)), _ptr(out))
    return out[: p.n]


def render(p: Params, view, st: Settings, pix=None):
    """Render all pixels (pix=None -> arrays shaped [3,H,W], [H,W]) or the listed flat pixel
    indices (-> [npix,3], [npix]). Returns (color, final_T, ncontrib, margins)."""
    L = lib()
    npix = view.width * view.height if pix is None else len(pix)
    pix_arr = None if pix is None else np.ascontiguousarray(pix, dtype=np.int32)
    color = np.zeros((npix, 3))
    T = np.zeros(npix)
    nc = np.zeros(npix, dtype=np.int32)
    margins = np.zeros((npix, 3))
    L.orc_render(p.n, _ptr(p.means), _ptr(p.scales), _ptr(p.quats), _ptr(p.opacity), _ptr(p.sh),
                 C.byref(_cview(view)), C.byref(_csettings(st, p.sh)), npix if pix is not None else 0,
                 _ptr(pix_arr, C.c_int32), _ptr(color), _ptr(T), _ptr(nc, C.c_int32), _ptr(margins))
    if pix is None:
        H, W = view.height, view.width
        return (color.reshape(H, W, 3).transpose(2, 0, 1).copy(), T.reshape(H, W),
                nc.reshape(H, W), margins.reshape(H, W, 3))
    return color, T, nc, margins


def backward(p: Params, view, st: Settings, dLdC, pix=None, want_g2=False, want_abs=False):
    """Adjoint of ``render`` for a loss whose gradient w.r.t. the colours is dLdC ([3,H,W] for
    the full image, or [npix,3] for listed pixels). Returns a dict of FP64 gradients; with
    want_g2 also "screen" [n, 9], the screen-space gradients, and with want_abs "screen_abs",
    the sums over pixels of the absolute values of their contributions."""
    L = lib()
    if pix is None:
        d = np.ascontiguousarray(np.asarray(dLdC, dtype=np.float64).transpose(1, 2, 0).reshape(-1, 3))
        npix_arg, pix_arr = 0, None
    else:
        d = np.ascontiguousarray(dLdC, dtype=np.float64)
        npix_arg, pix_arr = len(pix), np.ascontiguousarray(pix, dtype=np.int32)
    g = dict(means=np.zeros_like(p.means), scales=np.zeros_like(p.scales),
             quats=np.zeros_like(p.quats), opacity=np.zeros_like(p.opacity), sh=np.zeros_like(p.sh))
    g2 = np.zeros((max(p.n, 1), 9)) if want_g2 else None
    g2abs = np.zeros((max(p.n, 1), 9)) if want_abs else None
    L.orc_backward(p.n, _ptr(p.means), _ptr(p.scales), _ptr(p.quats), _ptr(p.opacity), _ptr(p.sh),
                   C.byref(_cview(view)), C.byref(_csettings(st, p.sh)), npix_arg,
                   _ptr(pix_arr, C.c_int32), _ptr(d), _ptr(g["means"]), _ptr(g["scales"]),
                   _ptr(g["quats"]), _ptr(g["opacity"]), _ptr(g["sh"]), _ptr(g2), _ptr(g2abs))
    if want_g2:
        g["screen"] = g2[: p.n]
    if want_abs:
        g["screen_abs"] = g2abs[: p.n]
    return g


def chain(p: Params, view, st: Settings, g2):
    """The chain rule alone (App. A.3): FP64 parameter gradients of one view from given
    per-Gaussian screen-space gradients g2 [n, 9] (order of G2_NAMES)."""
    L = lib()
    g2 = np.ascontiguousarray(g2, dtype=np.float64).reshape(p.n, 9)
    g = dict(means=np.zeros_like(p.means), scales=np.zeros_like(p.scales),
             quats=np.zeros_like(p.quats), opacity=np.zeros_like(p.opacity), sh=np.zeros_like(p.sh))
    L.orc_chain(p.n, _ptr(p.means), _ptr(p.scales), _ptr(p.quats), _ptr(p.opacity), _ptr(p.sh),
                C.byref(_cview(view)), C.byref(_csettings(st, p.sh)), _ptr(g2), _ptr(g["means"]),
                _ptr(g["scales"]), _ptr(g["quats"]), _ptr(g["opacity"]), _ptr(g["sh"]))
    return g


def sh_eval(deg, direction):
    out = np.zeros(16)
    lib().orc_sh_eval(int(deg), _ptr(_d(direction)), _ptr(out))
    return out[: (deg + 1) ** 2]


def depth_f32(mean, view):
    return np.float32(lib().orc_depth_f32(_ptr(_d(mean)), C.byref(_cview(view))))


def num_threads():
    return int(lib().orc_num_threads())


def ambiguous(margins, eps_skip=2e-5, eps_term=1e-4, eps_clamp=None):
    """Pixels whose discrete decisions lie within rounding of a threshold: the alpha >= 1/255
    test (relative band eps_skip), the T < 1e-4 termination (eps_term) and, for gradients,
    the 0.99 clamp (eps_clamp)."""
    m = np.asarray(margins)
    amb = (m[..., 0] < eps_skip) | (m[..., 1] < eps_term)
    if eps_clamp is not None:
        amb |= m[..., 2] < eps_clamp
    return amb


def fd_grad(p: Params, view, st: Settings, weights, name, index, h=None):
    """Central difference of L = sum(weights * image) w.r.t. one parameter element."""
    arr = getattr(p, name)
    x0 = arr.flat[index]
    if h is None:
        h = 1e-6 * max(1.0, abs(x0))
    arr.flat[index] = x0 + h
    cp, _, _, _ = render(p, view, st)
    arr.flat[index] = x0 - h
    cm, _, _, _ = render(p, view, st)
    arr.flat[index] = x0
    return float(np.sum(weights * (cp - cm)) / (2.0 * h))
