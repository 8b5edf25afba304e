"""The bench's roofline accounting (host logic, no GPU): the algorithmic bytes and flops per unit
that the per-stage fractions divide by, as the kernel table of the design notes states them."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_per_unit_figures():
    # parameters of one Gaussian: mean 12 B, scales 12 B, quaternion 16 B, opacity 4 B, SH 3 x 4 B per coefficient
    assert bench.param_bytes(3) == 236 and bench.param_bytes(0) == 56
    assert bench.RECORD_BYTES == 8 + 12 + 4 + 12 + 4 + 12   # ERP mean, conic, opacity, colour, key, rectangle
    assert bench.ACC_BYTES == 9 * 4                         # the nine accumulated screen-space gradients
    assert (bench.FLOP_TESTED, bench.FLOP_BLEND_FWD, bench.FLOP_BLEND_BWD) == (11, 12, 34)


def test_stage_rooflines_divide_the_stated_work_by_the_stage_time():
    stats = dict(visible=900, pairs_sorted=5000, evals_fwd=40000, evals_bwd=30000, blended=7000)
    kern = dict(preprocess=0.5, bin_sort=1.0, render_fwd=0.25, render_bwd=0.5, preprocess_bwd=0.2)
    out = bench.stage_rooflines(kern, stats, n=1000, sh_degree=3, tiles=64, pair_passes=1, hbm_gbs=100.0,
                                alu_tflops=10.0, alu_measured=8.0)
    assert out["preprocess"]["bytes"] == 1000 * 236 + 900 * 52
    # per item: depth passes, digit counts, count + emission reads, the saturation bound's reads, the
    # sorted key and kept-pair word; per sorted pair; per tile its range and bucket tables
    assert out["bin_sort"]["bytes"] == 1000 * (4 * 16 + 4 + 40 + 32 + 12) + 5000 * (8 + 16 + 4) + 64 * (8 + 3 * 128)
    assert out["preprocess_bwd"]["bytes"] == 1000 * 2 * 236 + 900 * 36
    assert out["render_fwd"]["flops"] == 11 * 40000 + 12 * 7000
    assert out["render_bwd"]["flops"] == 11 * 30000 + 34 * 7000
    for k, v in out.items():
        work = v.get("bytes", v.get("flops"))
        scale = 1e9 if v["unit"] == "GB/s" else 1e12
        assert v["achieved"] == pytest.approx(work / (kern[k] * 1e-3) / scale)
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
    assert out["render_bwd"]["frac_of_measured_ffma"] == pytest.approx(out["render_bwd"]["achieved"] / 8.0)


def test_profiled_traffic_is_tied_to_the_kernel_sources():
    d = bench.kernel_sources_digest()
    assert isinstance(d, str) and len(d) == 64
    t = bench.profiled_traffic()
    assert t is None or t == bench.PROFILED_TRAFFIC["bytes"]
    other = dict(bench.PROFILED_TRAFFIC, sources=("render_fwd.cu",))
    assert bench.kernel_sources_digest(other) != d


def test_clock_summary_reports_median_lowest_and_reasons():
    # nvidia-smi csv,noheader,nounits lines: sm, max sm, power, active mask, then the four reason flags
    lines = ["2002, 2070, 250.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "2070, 2070, 420.5, 0x4, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 400.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "[N/A], 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
             "garbage"]
    c = bench.summarise_clocks(lines)
    assert (c["sm_mhz"], c["sm_min_mhz"], c["sm_max_mhz"], c["samples"]) == (2070.0, 2002.0, 2070.0, 3)
    assert c["reasons"] == ["sw_power_cap"] and c["power_w_max"] == 420.5
    assert bench.summarise_clocks([])["sm_mhz"] is None


def test_reference_arm_names_the_same_workload_as_the_gpu_arm():
    """Both arms' JSON lines carry the same config dict (workload_config), so that their lines
    compare: here the reference arm's line, from a one-step run of the oracle on this host."""
    import json
    import subprocess
    saved = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                            "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    finally:
        os.environ.update(saved)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        args = bench.parse()
    finally:
        sys.argv = argv
    assert line["impl"] == "reference"
    assert line["config"] == bench.workload_config(args, 1)
    assert line["dtype"] == "f64" and line["higher_is_better"] is True
