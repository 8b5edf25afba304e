"""odgs_render_fwd_static: the forward render for callers that cannot allocate device memory
(a plugin or frame callback that owns a fixed device-memory budget, or a real-time loop where
cudaMalloc would synchronize the device). It takes only inputs and outputs; its scratch is a
static device array inside the library.

Checked here through the C ABI against the workspace entry points (odgs_preprocess ->
odgs_bin_sort -> odgs_render_fwd) on two different frames rendered one after the other, so that
state left in the shared array by the first call cannot leak into the second.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2410_20686_gb300 import scenes as S
from tests.helpers import IMG_TOL

pytestmark = pytest.mark.gpu


def _static_render(lib, scene, rs):
    import torch
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import _ptr
    m, s, q, o, sh = (torch.tensor(a, device="cuda") for a in (scene.means, scene.scales, scene.quats,
                                                                 scene.opacity, scene.sh))
    v = scene.views[0]
    img = torch.full((3, v.height, v.width), -1.0, device="cuda")
    T = torch.full((v.height, v.width), -1.0, device="cuda")
    status = torch.full((1,), 0xFFFF, dtype=torch.int32, device="cuda")
    g = L.Gaussians(_ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(sh), scene.n)
    view = L.make_view(v.width, v.height, v.R_wc, v.t_wc)
    st = rs.c_struct(scene.sh.shape[1])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.odgs_render_fwd_static(C.byref(g), C.byref(view), C.byref(st), _ptr(img), _ptr(T), _ptr(status), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return img.cpu().numpy(), T.cpu().numpy(), int(status.item())


def _workspace_render(scene, rs):
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    params = [torch.tensor(a, device="cuda") for a in (scene.means, scene.scales, scene.quats, scene.opacity, scene.sh)]
    imgs, Ts = Rasterizer().forward(*params, scene.views, rs)
    torch.cuda.synchronize()
    return imgs[0].cpu().numpy(), Ts[0].cpu().numpy()


def test_static_entry_point_matches_workspace_path_on_two_calls_in_a_row():
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300 import build as B
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    B.build()
    lib = L.load()
    first = S.config0()
    second = S.random_scene(20000, 512, 256, seed=404, sh_degree=3,
                            views=[S.yaw_view(512, 256, (0.2, -0.1, 0.3), 0.9)])
    for scene, rs in ((first, RenderSettings(sh_degree=0)), (second, RenderSettings(sh_degree=3, bg=(0.1, 0.2, 0.3)))):
        img, T, status = _static_render(lib, scene, rs)
        ref, Tref = _workspace_render(scene, rs)
        assert status == 0
        assert np.abs(img - ref).max() <= IMG_TOL
        assert np.abs(T - Tref).max() <= IMG_TOL


def test_static_entry_point_rejects_sizes_beyond_its_limits():
    import torch
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    lib = L.load()
    rs = RenderSettings(sh_degree=0)
    dummy = torch.zeros(16, device="cuda")
    big = L.Gaussians(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 40000)
    view = L.make_view(256, 128, np.eye(3), np.zeros(3))
    st = rs.c_struct(1)
    p = C.c_void_p(dummy.data_ptr())
    assert lib.odgs_render_fwd_static(C.byref(big), C.byref(view), C.byref(st), p, p, p, None) == -1
    small = L.Gaussians(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 10)
    huge_view = L.make_view(2048, 1024, np.eye(3), np.zeros(3))
    assert lib.odgs_render_fwd_static(C.byref(small), C.byref(huge_view), C.byref(st), p, p, p, None) == -1
