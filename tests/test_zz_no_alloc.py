"""odgs_render_fwd_static: the forward render for callers that cannot allocate device memory
(a plugin or frame callback that owns a fixed device-memory budget, or a real-time loop where
cudaMalloc would synchronize the device). It takes only inputs and outputs; its scratch is a
static device array inside the library.

Checked here through the C ABI against the workspace entry points (odgs_preprocess ->
odgs_bin_sort -> odgs_render_fwd), which run the same kernels, so the images must be identical
bit for bit: on frames rendered one after the other (small, large, the small one again, and a
pinhole view), so that state left in the shared array by one call cannot leak into the next; on
a frame with more pairs than the array holds (reported in status_out, finite image) followed by
an exact one; and on arguments the workspace path rejects.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2410_20686_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _static_render(lib, scene, rs, view=None):
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
    view = view or L.make_view(v.width, v.height, v.R_wc, v.t_wc, v.model, v.fx, v.fy, v.cx, v.cy)
    st = rs.c_struct(scene.sh.shape[1])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.odgs_render_fwd_static(C.byref(g), C.byref(view), C.byref(st), _ptr(img), _ptr(T), _ptr(status), stream)
    torch.cuda.synchronize()
    return rc, img.cpu().numpy(), T.cpu().numpy(), int(status.item())


def _workspace_render(scene, rs):
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    params = [torch.tensor(a, device="cuda") for a in (scene.means, scene.scales, scene.quats, scene.opacity, scene.sh)]
    rast = Rasterizer()
    imgs, Ts = rast.forward(*params, scene.views, rs)
    torch.cuda.synchronize()
    return imgs[0].cpu().numpy(), Ts[0].cpu().numpy(), rast.stats()


def _lib():
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300 import build as B
    B.build()
    return L.load()


def test_static_entry_point_matches_workspace_path_on_calls_in_a_row():
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    lib = _lib()
    first = S.config0()
    second = S.random_scene(20000, 512, 256, seed=404, sh_degree=3,
                            views=[S.yaw_view(512, 256, (0.2, -0.1, 0.3), 0.9)])
    pinhole = S.random_scene(8000, 320, 240, seed=405, sh_degree=2, radius=(1.0, 6.0),
                             views=[S.pinhole_view(320, 240, 260.0, 250.0, 158.5, 121.0,
                                                   R_wc=np.asarray(S.yaw_view(8, 4, (0, 0, 0), 0.4).R_wc),
                                                   t_wc=np.array([0.1, -0.05, 0.2], np.float32))])
    frames = ((first, RenderSettings(sh_degree=0)),
              (second, RenderSettings(sh_degree=3, bg=(0.1, 0.2, 0.3))),
              (first, RenderSettings(sh_degree=0)),
              (pinhole, RenderSettings(sh_degree=2)))
    for scene, rs in frames:
        rc, img, T, status = _static_render(lib, scene, rs)
        ref, Tref, _ = _workspace_render(scene, rs)
        assert rc == 0 and status == 0
        assert np.array_equal(img, ref), np.abs(img - ref).max()
        assert np.array_equal(T, Tref)


def test_static_entry_point_reports_pairs_beyond_its_array_and_recovers():
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    lib = _lib()
    big = S.random_scene(32768, 1024, 512, seed=406, sh_degree=0, radius=(1.0, 2.5), log_scale=(-1.0, 0.3))
    rs = RenderSettings(sh_degree=0)
    _, _, stats = _workspace_render(big, rs)
    assert stats["pairs"] > 2_000_000  # well beyond the array's pair capacity
    rc, img, T, status = _static_render(lib, big, rs)
    assert rc == 0 and status & L.DEV_CAPACITY
    assert np.isfinite(img).all() and np.isfinite(T).all()
    small = S.random_scene(3000, 1024, 512, seed=407, sh_degree=0)
    rc, img, T, status = _static_render(lib, small, rs)
    ref, Tref, _ = _workspace_render(small, rs)
    assert rc == 0 and status == 0
    assert np.array_equal(img, ref) and np.array_equal(T, Tref)


def test_static_entry_point_rejects_what_the_workspace_path_rejects():
    import torch
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    lib = _lib()
    rs = RenderSettings(sh_degree=0)
    dummy = torch.zeros(16, device="cuda")
    d = dummy.data_ptr()
    p = C.c_void_p(d)
    st = rs.c_struct(1)
    small = L.Gaussians(d, d, d, d, d, 10)
    view = L.make_view(256, 128, np.eye(3), np.zeros(3))
    # sizes beyond the static array's limits
    big = L.Gaussians(d, d, d, d, d, 40000)
    assert lib.odgs_render_fwd_static(C.byref(big), C.byref(view), C.byref(st), p, p, p, None) == -1
    huge_view = L.make_view(2048, 1024, np.eye(3), np.zeros(3))
    assert lib.odgs_render_fwd_static(C.byref(small), C.byref(huge_view), C.byref(st), p, p, p, None) == -1
    # a non-finite pose, background or dilation, and flags other than 0 / 1
    nan_view = L.make_view(256, 128, [[1, 0, 0], [0, float("nan"), 0], [0, 0, 1]], np.zeros(3))
    assert lib.odgs_render_fwd_static(C.byref(small), C.byref(nan_view), C.byref(st), p, p, p, None) == -1
    inf_t = L.make_view(256, 128, np.eye(3), [0.0, float("inf"), 0.0])
    assert lib.odgs_render_fwd_static(C.byref(small), C.byref(inf_t), C.byref(st), p, p, p, None) == -1
    for field, value in (("bg", (0.0, float("nan"), 0.0)), ("cov_dilation", float("inf")), ("raw_params", 2),
                         ("checked", 3)):
        bad = rs.c_struct(1)
        if field == "bg":
            bad.bg[:] = list(value)
        else:
            setattr(bad, field, value)
        assert lib.odgs_render_fwd_static(C.byref(small), C.byref(view), C.byref(bad), p, p, p, None) == -1, field
