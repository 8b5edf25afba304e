"""Host-side checks of the C ABI: the library builds, loads, exports every declared symbol, and
validates arguments without touching the GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2410_20686_gb300 import _lib as L
from paper_2410_20686_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def _declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(odgs_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert sorted(L.EXPORTED) == _declared_functions()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def _settings(**kw):
    s = L.Settings()
    s.sh_degree, s.sh_coeffs, s.tile_w, s.tile_h, s.batch = 3, 16, 16, 16, 64
    s.cov_dilation, s.r_near, s.r_far = 0.3, 0.2, 1e4
    s.bg[:] = [0.0, 0.0, 0.0]
    for k, v in kw.items():
        setattr(s, k, v)
    return s


def _views(*sizes):
    arr = (L.View * len(sizes))()
    for i, (w, h) in enumerate(sizes):
        arr[i] = L.make_view(w, h, [1, 0, 0, 0, 1, 0, 0, 0, 1], [0, 0, 0])
    return arr


def _ws(lib, n, views, nv, s):
    out = C.c_size_t()
    st = lib.odgs_workspace_size(n, views, nv, C.byref(s), C.byref(out))
    return st, out.value


def test_workspace_size_is_pure_and_monotone(lib):
    v = _views((256, 128))
    st0, b0 = _ws(lib, 1000, v, 1, _settings())
    st1, b1 = _ws(lib, 2000, v, 1, _settings())
    assert st0 == st1 == 0 and 0 < b0 < b1
    v2 = _views((256, 128), (512, 256))
    st2, b2 = _ws(lib, 1000, v2, 2, _settings())
    assert st2 == 0 and b2 > b0


@pytest.mark.parametrize("bad", [dict(sh_degree=4), dict(sh_coeffs=3), dict(tile_w=12), dict(tile_w=8, tile_h=2),
                                 dict(batch=300), dict(r_near=5.0, r_far=1.0), dict(cov_dilation=-1.0)])
def test_invalid_settings_rejected(lib, bad):
    st, _ = _ws(lib, 10, _views((256, 128)), 1, _settings(**bad))
    assert st == -1


def test_invalid_views_rejected(lib):
    assert _ws(lib, 10, _views((250, 128)), 1, _settings())[0] == -1  # W not a multiple of the tile
    assert _ws(lib, 10, _views((256, 0)), 1, _settings())[0] == -1
    assert _ws(lib, 10, _views((256, 128)), 0, _settings())[0] == -1
    assert _ws(lib, -1, _views((256, 128)), 1, _settings())[0] == -1


def test_pair_buffer_size(lib):
    out = C.c_size_t()
    assert lib.odgs_pair_buffer_size(1000, C.byref(out)) == 0 and out.value >= 16 * 1000
    assert lib.odgs_pair_buffer_size(1 << 30, C.byref(out)) == -1


def test_null_context_rejected(lib):
    v = _views((256, 128))
    s = _settings()
    g = L.Gaussians()
    assert lib.odgs_preprocess(None, C.byref(g), v, 1, C.byref(s), None, 0, None) == -1
    assert lib.odgs_bin_sort(None, None, 0, None) == -1
    assert lib.odgs_render_fwd(None, None, None, None) == -1
    assert lib.odgs_render_bwd(None, None, None) == -1
    assert lib.odgs_preprocess_bwd(None, None, None) == -1
    assert lib.odgs_create(None) == -1
    assert lib.odgs_status_string(-2).decode() == "pair capacity exceeded"


def test_status_codes_and_device_bits_agree_with_the_header():
    text = open(os.path.join(ROOT, "include", "odgs.h")).read()
    codes = dict((n, int(v)) for n, v in re.findall(r"\b(ODGS_(?:OK|ERR_[A-Z_]+))\s*=\s*(-?\d+)", text))
    for name, value in codes.items():
        assert getattr(L, name) == value, name
        assert L.STATUS_NAMES[value] == name
    bits = dict((n, int(v)) for n, v in re.findall(r"#define ODGS_DEV_([A-Z_]+) (\d+)u", text))
    assert bits == {"CAPACITY": L.DEV_CAPACITY, "TIMEOUT": L.DEV_TIMEOUT, "NONFINITE": L.DEV_NONFINITE}


def test_checked_setting_is_validated(lib):
    views = _views((256, 128))
    st, _ = _ws(lib, 100, views, 1, _settings(checked=2))
    assert st == L.ODGS_ERR_INVALID_ARG
    st, _ = _ws(lib, 100, views, 1, _settings(checked=1))
    assert st == L.ODGS_OK


def test_view_size_limits(lib):
    s = _settings()
    assert _ws(lib, 100, _views((16384, 8192)), 1, s)[0] == L.ODGS_OK
    assert _ws(lib, 100, _views((16400, 8192)), 1, s)[0] == L.ODGS_ERR_INVALID_ARG
    assert _ws(lib, 100, _views((256, 16385)), 1, s)[0] == L.ODGS_ERR_INVALID_ARG
    assert _ws(lib, 100, _views((250, 128)), 1, s)[0] == L.ODGS_ERR_INVALID_ARG  # not a multiple of the tile width
