"""Frame work counters and the throughput microbenchmark behind the blend kernels' rooflines."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import oracle_settings

pytestmark = pytest.mark.gpu


def test_counters_bound_each_other_and_match_the_oracle_culls():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc = S.config1()
    rs = RenderSettings(sh_degree=3)
    params = [torch.tensor(a, device="cuda") for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.sh)]
    rast = Rasterizer()
    imgs, _ = rast.forward(*params, sc.views, rs, want_T=False)
    rast.backward([torch.ones_like(im) for im in imgs])
    torch.cuda.synchronize()
    st = rast.stats()
    assert st["status"] == 0
    # visible items: the same culls as the oracle's projection (shell, pole, det, opacity);
    # only threshold ties between FP32 and FP64 may differ
    pj = O.project(O.Params.of(sc), sc.views[0], oracle_settings(rs))
    valid = int((pj[:, O.PJ_VALID] > 0).sum())
    assert abs(st["visible"] - valid) <= max(2, int(1e-4 * sc.n)), (st["visible"], valid)
    # a pixel stops no later than its tile; each tile processes at most its own list
    tile_px = rs.tile_w * rs.tile_h
    assert st["blended"] <= st["evals_fwd"] <= st["entries_tile"] * tile_px
    # the sorted pairs are the pairs of the footprints, less those cut at saturated tiles
    assert 0 < st["entries_tile"] <= st["pairs_sorted"] <= st["pairs"]
    # the backward walks each pixel's list from its last blended entry, so never further
    assert st["evals_bwd"] <= st["evals_fwd"]


def test_measured_peaks_are_plausible():
    import torch
    from paper_2410_20686_gb300.rasterizer import measure_peaks
    pk = measure_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert pk["sms"] == sms
    # at most the clock-derived FMA peak at 2.5 GHz; at least a tenth of it at 1 GHz
    top = sms * 128 * 2 * 2.5e9 / 1e12
    assert 0.1 * sms * 128 * 2 * 1.0e9 / 1e12 < pk["ffma_tflops"] < top
    # exp2f is a multi-function-unit operation: slower than an FMA, but well above 1% of it
    fma_per_s = pk["ffma_tflops"] * 1e12 / 2
    assert 0.01 * fma_per_s < pk["ex2_gops"] * 1e9 < fma_per_s
    assert np.isfinite(pk["ex2_gops"])
