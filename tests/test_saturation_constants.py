"""The arithmetic behind the cut tile lists (CPU): the threshold on the coverage sums and the
bound on how many entries a pixel blends, as the device header states them (csrc/odgs_common.cuh).

A tile keeps the depth buckets up to the first at which sum -log2(1 - a_c) over the Gaussians
covering it reaches kCutThreshold / 256 bits; then every pixel of the tile has stopped, because its
transmittance after those Gaussians is below 2^-(threshold) times the rounding of at most 2350
float32 products, and a pixel blends at most 2350 entries (each with alpha >= 1/255) before its
transmittance falls below 1e-4."""
import math
import os
import re

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2410_20686_gb300", "csrc", "odgs_common.cuh")


def _constant(name):
    m = re.search(r"constexpr\s+\w+\s+%s\s*=\s*([0-9.]+)" % name, open(HEADER).read())
    assert m, name
    return float(m.group(1))


def test_threshold_is_log2_of_1e4_plus_a_quarter_bit_in_fixed_point():
    assert _constant("kCutThreshold") == math.ceil((math.log2(1e4) + 0.25) * 256)


def test_a_pixel_blends_at_most_2350_entries_before_it_stops():
    # every blended entry has alpha >= 1/255, so after n of them T <= (254/255)^n, and a pixel's T
    # never falls below 1e-4: n is below the first n with (254/255)^n < 1e-4, 2345
    first = math.ceil(math.log(1e-4) / math.log(254 / 255))
    assert (254 / 255) ** first < 1e-4 <= (254 / 255) ** (first - 1)
    assert first <= 2350


def test_the_threshold_covers_the_rounding_of_the_running_products():
    t = _constant("kCutThreshold") / 256.0
    u = 2.0 ** -24
    # each blend rounds 1 - alpha and the product: at most 2 roundings per factor, 2350 factors
    rounding = (1 + u) ** (2 * 2350)
    assert 2.0 ** -t * rounding < 1e-4
    # and the quarter bit is not needed to much more than that: the margin stays below 20 %
    assert 2.0 ** -t * rounding > 0.8e-4


def test_buckets_are_four_per_octave_of_depth():
    shift = int(_constant("kCutShift"))
    # the float bits of a positive depth, shifted right by 21, keep the exponent and the top two
    # mantissa bits: four buckets per doubling of the depth, monotone in the depth
    import struct
    bits = lambda x: struct.unpack("<I", struct.pack("<f", x))[0]
    b = [bits(x) >> shift for x in (1.0, 1.19, 1.25, 1.5, 1.75, 2.0)]
    assert b == sorted(b) and b[0] == b[1] and b[2] == b[0] + 1 and b[5] == b[0] + 4


def test_the_exponent_is_largest_at_a_corner_pixel_of_the_tile():
    # the coverage bound takes alpha at a tile's four corner pixel centres as the smallest over
    # the tile: the quadratic form a (dx - beta dy)^2 + gamma dy^2 is convex, so over the box of a
    # tile's pixel centres its maximum is at a corner (brute force over every pixel, float64)
    import numpy as np
    rng = np.random.default_rng(5)
    for _ in range(300):
        a, gam = np.exp(rng.uniform(-8, 2, 2))
        beta = rng.normal(0, 3)
        tw, th = int(rng.choice([8, 16, 32])), int(rng.integers(1, 33))
        x0, y0 = rng.uniform(-200, 200, 2)  # the tile's first pixel centre relative to the mean
        xs, ys = np.meshgrid(x0 + np.arange(tw), y0 + np.arange(th))
        q = a * (xs - beta * ys) ** 2 + gam * ys ** 2
        corners = [q[0, 0], q[0, -1], q[-1, 0], q[-1, -1]]
        assert q.max() == max(corners)
