"""Checked mode (odgs_settings.checked): non-finite inputs are reported in the device status word
(ODGS_DEV_NONFINITE) without a fault. A Gaussian with a NaN or inf parameter is culled in every
view, exactly as a Gaussian of zero opacity is; a non-finite dL/dimage value counts as 0."""
import ctypes as C

import numpy as np
import pytest

from paper_2410_20686_gb300 import scenes as S
from tests.helpers import to_torch

pytestmark = pytest.mark.gpu


def _scene():
    return S.random_scene(2000, 256, 128, seed=71, sh_degree=2, radius=(0.8, 4.0))


def _render(params, views, rs, dl=None):
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer
    rast = Rasterizer()
    imgs, Ts = rast.forward(*params, views, rs, want_T=True)
    if dl is None:
        dl = [torch.ones_like(im) for im in imgs]
    g = rast.backward(dl)
    torch.cuda.synchronize()
    return rast, [im.cpu().numpy() for im in imgs], [t.cpu().numpy() for t in Ts], \
        {k: v.cpu().numpy() for k, v in g.items()}


def test_clean_inputs_give_the_unchecked_results():
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    sc = _scene()
    a = _render(to_torch(sc), sc.views, RenderSettings(sh_degree=2))
    b = _render(to_torch(sc), sc.views, RenderSettings(sh_degree=2, checked=True))
    assert b[0].status() == 0
    for x, y in zip(a[1] + a[2], b[1] + b[2]):
        np.testing.assert_array_equal(x, y)


def _raw(params):
    import torch
    m, s, q, o, sh = params
    return [m, torch.log(s), q, torch.log(o) - torch.log1p(-o), sh]


@pytest.mark.parametrize("raw", [False, True])
def test_nonfinite_gaussians_are_culled_and_reported(raw):
    import torch
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    sc = _scene()
    bad = [5, 17, 40, 333]
    poisoned = _raw(to_torch(sc)) if raw else to_torch(sc)
    poisoned[0][5, 0] = float("nan")       # mean
    poisoned[1][17, 1] = float("inf")      # scale (log-scale +inf: scale inf)
    poisoned[2][333, 2] = float("nan")     # quaternion
    poisoned[4][40, 2, 1] = float("nan")   # an SH coefficient
    reference = _raw(to_torch(sc)) if raw else to_torch(sc)
    reference[3][bad] = -1e30 if raw else 0.0  # zero opacity: culled by the alpha bound
    rs = RenderSettings(sh_degree=2, checked=True, raw_params=raw)
    rp, ip, Tp, gp = _render(poisoned, sc.views, rs)
    rr, ir, Tr, gr = _render(reference, sc.views, rs)
    assert rp.status() & L.DEV_NONFINITE and rr.status() == 0
    for x, y in zip(ip + Tp, ir + Tr):
        np.testing.assert_array_equal(x, y)
    keep = np.setdiff1d(np.arange(2000), bad)
    for k in gp:
        assert np.isfinite(gp[k]).all(), k
        assert not gp[k][bad].any(), k
        scale = max(float(np.abs(gr[k][keep]).max()), 1e-30)
        assert float(np.abs(gp[k][keep] - gr[k][keep]).max()) <= 1e-5 * scale, k
    # the status is what odgs_query_pairs returns
    p = C.c_size_t()
    st = rp.lib.odgs_query_pairs(rp.ctx, C.byref(p), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.ODGS_ERR_NONFINITE


def test_nonfinite_image_gradients_count_as_zero():
    import torch
    from paper_2410_20686_gb300 import _lib as L
    from paper_2410_20686_gb300.rasterizer import RenderSettings
    sc = _scene()
    rs = RenderSettings(sh_degree=2, checked=True)
    params = to_torch(sc)
    rng = np.random.default_rng(5)
    dl = rng.normal(size=(3, 128, 256)).astype(np.float32)
    where = [(0, 64, 100), (1, 10, 3), (2, 127, 255), (0, 0, 0)]
    clean = dl.copy()
    dirty = dl.copy()
    for (c, y, x), v in zip(where, (np.nan, np.inf, -np.inf, np.nan)):
        clean[c, y, x] = 0.0
        dirty[c, y, x] = v
    rd, _, _, gd = _render(params, sc.views, rs, [torch.tensor(dirty, device="cuda")])
    rc, _, _, gc = _render(params, sc.views, rs, [torch.tensor(clean, device="cuda")])
    assert rd.status() & L.DEV_NONFINITE and rc.status() == 0
    for k in gd:
        assert np.isfinite(gd[k]).all(), k
        scale = max(float(np.abs(gc[k]).max()), 1e-30)
        assert float(np.abs(gd[k] - gc[k]).max()) <= 1e-5 * scale, k
