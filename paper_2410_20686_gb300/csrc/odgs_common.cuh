// Device-side definitions shared by the ODGS kernels (sm_103a).
//
// Record layout per (view, Gaussian) item, written by the preprocess kernel and gathered by the
// blend kernels (16-byte vector loads):
//   rec_a = { du, dv, bits(c0 | r0 << 16), opacity }   mean = (c0 + 0.5 + du, r0 + 0.5 + dv)
//   (c0, r0 as 16-bit two's complement: pinhole centres may lie left of or above the image)
//   rec_b = { a, beta, gamma, Qb }                      inverse of Sigma_2D (Eq. 8, dilated) in
//                                                        slice form, see below; Qb the binning bound
//   rec_c = { r, g, b, 0 }                              SH colour
// The mean is stored as an integer pixel anchor plus a small float offset so that the offset
// from any pixel centre, (i - c0) - du, is formed without the rounding error of a float
// coordinate near W (about 1e-4 px at W = 2048).
//
// The conic is stored in slice (LDL^T) form: with Sigma_2D = [[A, B], [B, C]] and det = AC - B^2,
//   d^T Sigma_2D^-1 d = a (dx - beta dy)^2 + gamma dy^2,   a = C / det, beta = B / C, gamma = 1 / C,
// i.e. for each pixel row the quadratic form is a parabola in dx centred on the ellipse's
// horizontal slice, x = beta dy. Every one of a, beta, gamma is a quotient of positive, accurately
// formed quantities, and the form is evaluated as a (t t) + gamma dy^2 with t = dx - beta dy, a
// small number near the ellipse. The entries of the inverse in image axes, (C, -B, A) / det,
// would instead make a needle-like Gaussian's exponent a difference of terms about cond(Sigma_2D)
// times larger than itself.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace odgs {

constexpr int kMaxViews = 64;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
// alpha >= 1/255 is decided on the base-2 exponent p of alpha = 2^p: p >= log2(1/255).
constexpr float kLog2AlphaMin = -7.99435343685886f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kLog2_255 = 7.994353436858858f;
constexpr float kPi = 3.14159265358979323846f;

// device status bits (mirrors ODGS_DEV_* in odgs.h)
constexpr uint32_t kStCapacity = 1u;
constexpr uint32_t kStTimeout = 2u;
constexpr uint32_t kStNonfinite = 4u;

// Per-view constants, uploaded once per frame into the workspace.
struct ViewDev {
    int W, H, tiles_x, tiles_y;
    int tile_base;  // first global tile id of this view
    int pix_base;   // first global pixel index of this view
    int trig_u;     // float4 offset of the per-column (cos, sin) table
    int trig_v;     // float4 offset of the per-row (cos, sin) table
    float R[9];
    float t[3];
    float cam[3];   // camera centre in world space, -R^T t
    float fx, fy;   // ERP: W / (2 pi), H / pi; pinhole: the focal lengths in pixels
    int model;      // 0: ERP (Eq. 4, periodic in u); 1: pinhole u = fx tx/tz + cx (Eq. 1)
    float cx, cy;   // pinhole principal point
};

// Pixel anchor of a record: two signed 16-bit fields in the bits of a float.
__device__ __forceinline__ float pack_anchor(int c0, int r0) {
    return __uint_as_float(((uint32_t)c0 & 0xFFFFu) | ((uint32_t)r0 << 16));
}
__device__ __forceinline__ void unpack_anchor(float f, int& c0, int& r0) {
    const uint32_t packed = __float_as_uint(f);
    c0 = (int)(int16_t)(packed & 0xFFFFu);
    r0 = (int)(int16_t)(packed >> 16);
}

// Device header at the start of the workspace.
struct Header {
    unsigned long long pairs;         // total (tile, Gaussian) pairs counted by the preprocess
    unsigned long long pairs_emitted; // min(pairs, capacity) used by the tile sort
    unsigned long long visible;       // (view, Gaussian) items that survived culling
    // backward-blend counters, contiguous so that one memset clears them
    unsigned long long evals_bwd;     // (pixel, entry) evaluations of the last backward blend
    uint32_t work_bwd;
    uint32_t pad0;
    // forward counters, contiguous so that one memset clears them
    unsigned long long evals_fwd;     // (pixel, entry) evaluations of the last forward blend
    unsigned long long blended;       // (pixel, entry) pairs blended by the last forward pass
    unsigned long long entries_tile;  // sum over tiles of the entries processed until all the
                                      // tile's pixels had stopped
    uint32_t work_fwd;
    uint32_t pad1;
    uint32_t status;
    uint32_t n_items;                 // views * n
    uint32_t n_pairs_sort;            // 32-bit copy of pairs_emitted for the sort kernels
    uint32_t n_big;                   // items queued for the warp-wide emission
    uint32_t n_count_big;             // items queued for the warp-wide kept-pair count
    uint32_t pad[3];
};

struct Settings {
    int sh_degree, sh_coeffs;
    int tile_w, tile_h;
    float dilation, r_near, r_far;
    float bg[3];
    int raw;      // scales are log-scales and opacity logits
    int checked;  // flag and cull non-finite parameters
};

// Activation of the raw variables of 3DGS training: scale = exp(log-scale), opacity =
// sigmoid(logit) = 1 / (1 + exp(-logit)).
__device__ __forceinline__ float sigmoid_act(float x) { return 1.f / (1.f + expf(-x)); }

// ------------------------------------------------------------------ float-float arithmetic
// Unevaluated sums hi + lo (Dekker 1971; Knuth's TwoSum), used to place the ERP mean precisely and,
// in the backward chain rule, to rotate dL/dconic exactly. Every operation is written with
// round-to-nearest intrinsics so the compiler can neither contract nor reorder it.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float v = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    float c = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return quick_two_sum(p.hi, __fadd_rn(p.lo, c));
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
    ff p = two_prod(a.hi, b);
    return quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// a / b: a float quotient, then the quotient of the exact remainder
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = ff_add(a, ff_neg(ff_mulf(b, q1)));
    return quick_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
    float s = __fsqrt_rn(a.hi);
    if (!(s > 0.f)) return {s, 0.f};
    float r = __fmaf_rn(-s, s, a.hi);  // exact residual a.hi - s^2
    float e = __fdiv_rn(__fadd_rn(r, a.lo), __fmul_rn(2.f, s));
    return quick_two_sum(s, e);
}

// ------------------------------------------------------------------ blend evaluation
// Staged form of one list entry for a given tile (identical in the forward and backward
// kernels, so both take the same skip / clamp / termination decisions bit for bit).
struct Staged {
    float4 pos;  // fc (column anchor, incl. seam shift), fr (row anchor), du, dv
    float4 con;  // a k, beta, gamma k, log2(o) with k = -log2(e) / 2: p = log2(o) + k (a t^2 + gamma dy^2)
    float4 col;  // r, g, b, fsplit (first column using fc2; +inf if none)
    float fc2;   // column anchor right of the seam split
};

// Rotation matrix of the normalized quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Seam shift for pixel column i: the image of the Gaussian nearest to the pixel, so that the
// horizontal offset lies in [-W/2, W/2).
__device__ __forceinline__ int seam_shift(int i, int c0, float du, int W) {
    float dx0 = __fsub_rn((float)(i - c0), du);
    float half = 0.5f * (float)W;
    if (dx0 >= half) return W;
    if (dx0 < -half) return -W;
    return 0;
}

// periodic: ERP views (seam-wrapped offsets); pinhole views have no seam.
__device__ __forceinline__ Staged stage_entry(float4 ra, float4 rb, float4 rc, int x0, int tw, int W, bool periodic) {
    Staged s;
    int c0, r0;
    unpack_anchor(ra.z, c0, r0);
    int s0 = periodic ? seam_shift(x0, c0, ra.x, W) : 0;
    int s1 = periodic ? seam_shift(x0 + tw - 1, c0, ra.x, W) : 0;
    float fsplit = __int_as_float(0x7f800000);  // +inf
    float fc2 = (float)(c0 + s1);
    if (s0 != s1) {
        int xs = x0 + 1;
        while (xs < x0 + tw - 1 && seam_shift(xs, c0, ra.x, W) == s0) ++xs;
        fsplit = (float)xs;
    }
    s.pos = make_float4((float)(c0 + s0), (float)r0, ra.x, ra.y);
    const float k = -0.5f * kLog2e;
    s.con = make_float4(__fmul_rn(rb.x, k), rb.y, __fmul_rn(rb.z, k), log2f(ra.w));
    s.col = make_float4(rc.x, rc.y, rc.z, fsplit);
    s.fc2 = fc2;
    return s;
}

// Gathers an item's three records; an index past the end (possible only after a sort that gave
// up, with the status already set) yields an entry that never passes the alpha test.
__device__ __forceinline__ void gather_records(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                               const float4* __restrict__ rc, uint32_t idx, uint32_t n_items,
                                               float4& a, float4& b, float4& c) {
    if (idx < n_items) {
        a = ra[idx]; b = rb[idx]; c = rc[idx];
    } else {
        a = make_float4(0.f, 0.f, 0.f, 0.f);  // opacity 0 -> log2(o) = -inf
        b = make_float4(1.f, 0.f, 1.f, 0.f);
        c = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ------------------------------------------------------------------ footprint on tiles
// The set {alpha >= 1/255} of an item is the ellipse d^T conic d <= Q with Q = 2 ln(255 o);
// binning uses an inflated Qb (stored in rec_b.w). For each tile row the ellipse's slice over the
// row band's pixel-centre rows is one interval of columns, so the tiles an item is listed in are
// exactly the tiles of each row band that meet that interval (seam-wrapped). The preprocess
// counts them and the emission writes them with these same functions on the same stored floats,
// with fixed instructions only (round-to-nearest intrinsics, the hardware's approximate reciprocal
// and reciprocal square root), so both agree bit for bit.
struct Footprint {
    int c0, r0;
    float du, dv;
    float BC;        // beta = B / C: centre line x = beta y of the horizontal slices
    float k;         // 1 / sqrt(a): half-width scale of the slices
    float iC;        // gamma = 1 / C
    float Qb;
    float ev;        // vertical half extent sqrt(Qb C)
    float ystar;     // dy of the rightmost point, B sqrt(Qb / A)
};

// The footprint's quotients and square roots in the hardware's approximate reciprocal and
// reciprocal square root (a few ulp): the footprint only bounds the set alpha >= 1/255, with
// margins far larger than that (Qb is inflated by 1e-4, the slice edges by 0.01 px), and the same
// instructions give the same bits wherever it is evaluated.
__device__ __forceinline__ float fp_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float fp_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

__device__ __forceinline__ Footprint make_footprint(float4 ra, float4 rb) {
    Footprint f;
    unpack_anchor(ra.z, f.c0, f.r0);
    f.du = ra.x;
    f.dv = ra.y;
    f.BC = rb.y;
    f.iC = rb.z;
    f.Qb = rb.w;
    const float ia = fp_div(1.f, rb.x);
    f.k = fp_sqrt(ia);
    f.ev = fp_sqrt(fp_div(f.Qb, f.iC));
    // Sigma_2D from the slice form without cancellation: C = 1 / gamma, B = beta C, A = 1 / a + beta B
    const float C = fp_div(1.f, f.iC);
    const float B = __fmul_rn(f.BC, C);
    const float A = __fadd_rn(ia, __fmul_rn(f.BC, B));
    f.ystar = __fmul_rn(B, fp_sqrt(fp_div(f.Qb, A)));
    return f;
}

// a mod m in [0, m), for any sign of a: a mask when m is a power of two (the common tile counts),
// else two integer remainders.
__device__ __forceinline__ int pos_mod(int a, int m) {
    return (m & (m - 1)) == 0 ? (a & (m - 1)) : ((a % m) + m) % m;
}

// Pixel rows [jlo, jhi] the footprint can reach (clipped to the image); empty if jlo > jhi.
__device__ __forceinline__ void footprint_rows(const Footprint& f, int H, int& jlo, int& jhi) {
    const float ev = fminf(f.ev, 2.f * (float)H);
    jlo = max(0, f.r0 + (int)ceilf(__fsub_rn(f.dv, ev)));
    jhi = min(H - 1, f.r0 + (int)floorf(__fadd_rn(f.dv, ev)));
}

// The same rows from the records directly, without the rest of the footprint: the backward blend
// skips an entry for a warp whose pixel rows all lie outside them (x = jlo, y = jhi). The
// operations are footprint_rows(make_footprint(ra, rb), H)'s, so the rows are the same.
__device__ __forceinline__ int2 footprint_row_range(float4 ra, float4 rb, int H) {
    int c0, r0;
    unpack_anchor(ra.z, c0, r0);
    const float ev = fminf(fp_sqrt(fp_div(rb.w, rb.z)), 2.f * (float)H);
    return make_int2(max(0, r0 + (int)ceilf(__fsub_rn(ra.y, ev))), min(H - 1, r0 + (int)floorf(__fadd_rn(ra.y, ev))));
}

// Horizontal offset of the slice boundary at vertical offset y (side = +1 right, -1 left).
__device__ __forceinline__ float slice_edge(const Footprint& f, float y, float side) {
    const float q = fmaxf(__fsub_rn(f.Qb, __fmul_rn(__fmul_rn(y, y), f.iC)), 0.f);
    return __fadd_rn(__fmul_rn(f.BC, y), side * __fmul_rn(f.k, fp_sqrt(q)));
}

// Tile columns of the band of pixel rows [J0, J1]: start column (mod tiles_x) and count (0 if
// the slice holds no pixel centre). periodic: ERP views wrap around the seam; pinhole views clip
// the columns to the image.
__device__ __forceinline__ void band_columns(const Footprint& f, int J0, int J1, int W, int tw, int tiles_x,
                                             bool periodic, int& start, int& count) {
    const float d0 = fmaxf(__fsub_rn((float)(J0 - f.r0), f.dv), -f.ev);
    const float d1 = fminf(__fsub_rn((float)(J1 - f.r0), f.dv), f.ev);
    count = 0;
    start = 0;
    if (!(d0 <= d1)) return;
    const float yr = fminf(fmaxf(f.ystar, d0), d1);
    const float yl = fminf(fmaxf(-f.ystar, d0), d1);
    const float xmax = __fadd_rn(slice_edge(f, yr, 1.f), 0.01f);
    const float xmin = __fsub_rn(slice_edge(f, yl, -1.f), 0.01f);
    const float half = (float)W;
    int ilo, ihi;
    if (periodic) {
        if (!(xmax - xmin < half)) { start = 0; count = tiles_x; return; }
        ilo = f.c0 + (int)ceilf(__fadd_rn(f.du, xmin));
        ihi = f.c0 + (int)floorf(__fadd_rn(f.du, xmax));
    } else {  // clamp before the conversion: a wide footprint can reach far outside the image
        const float lo = fmaxf(__fadd_rn(f.du, xmin), (float)(-f.c0 - 1));
        const float hi = fminf(__fadd_rn(f.du, xmax), (float)(W - f.c0));
        ilo = max(f.c0 + (int)ceilf(lo), 0);
        ihi = min(f.c0 + (int)floorf(hi), W - 1);
    }
    if (ihi < ilo) return;
    if (ihi - ilo + 1 >= W) { start = 0; count = tiles_x; return; }
    // floor division by the tile width, a power of two (8, 16 or 32): an arithmetic shift
    const int sh = __ffs(tw) - 1;
    const int tlo = ilo >> sh, thi = ihi >> sh;
    const int n = thi - tlo + 1;
    if (n >= tiles_x) { start = 0; count = tiles_x; return; }
    start = pos_mod(tlo, tiles_x);
    count = n;
}

// Offset from the Gaussian centre to the pixel centre (fi, fj are the integer pixel indices).
__device__ __forceinline__ void pixel_offset(float fi, float fj, float fc, float4 pos, float& dx, float& dy) {
    dx = __fsub_rn(__fsub_rn(fi, fc), pos.z);
    dy = __fsub_rn(__fsub_rn(fj, pos.y), pos.w);
}

// 2^p by the hardware's base-2 exponential (PTX ex2.approx.ftz.f32: relative error below 2^-22;
// the blend evaluates it only for p >= log2(1/255), so no result is subnormal). Forward and
// backward both use it, so they compute the same alpha.
__device__ __forceinline__ float alpha_exp2(float p) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
    return r;
}

// Base-2 exponent of alpha before the clamp, log2(o) - 0.5 log2(e) d^T conic d (Eq. 2), in the
// slice form: per pixel row the slice centre du + beta dy and the row term gamma' dy^2 + log2(o)
// (row_terms), then per pixel t = (i - fc) - centre and p = (a' t) t + row term.
__device__ __forceinline__ void row_terms(float4 con, float du, float dy, float& centre, float& rowt) {
    centre = __fmaf_rn(con.y, dy, du);
    rowt = __fmaf_rn(__fmul_rn(con.z, dy), dy, con.w);
}
__device__ __forceinline__ float slice_exponent(float4 con, float t, float rowt) {
    return __fmaf_rn(__fmul_rn(con.x, t), t, rowt);
}

// ------------------------------------------------------------------ saturated-tile truncation
// A tile's list needs only the entries up to the point where every pixel of the tile has stopped
// (transmittance below 1e-4): later entries are never evaluated, by the forward or the backward
// blend. An item that reaches alpha >= a_c >= 1/255 at every pixel centre of a tile multiplies
// the transmittance of every pixel there by at most 1 - a_c, so once the items of the tile,
// taken in depth order, have sum -log2(1 - a_c) > log2(1e4) + 0.25 every pixel has stopped
// (the 0.25 bits cover the rounding of the blend's running products, which have at most 2350
// factors: each has alpha >= 1/255 and (254/255)^2350 < 1e-4). The sums are kept per depth
// bucket (kCutShift: four buckets per octave of depth, from r_near), in fixed point with 8
// fractional bits, rounded down, so that they are exact and independent of the order of the
// atomic additions: the truncated lists are deterministic.
constexpr int kCutBuckets = 32;
constexpr int kCutShift = 21;
constexpr uint32_t kCutThreshold = 3466;  // ceil((log2(1e4) + 0.25) * 256)
constexpr uint8_t kCutNone = 255;         // the tile keeps its whole list

// Depth bucket of a depth key (the float bits of a positive depth: monotone in the depth).
__device__ __forceinline__ int depth_bucket(uint32_t key, uint32_t base) {
    const int b = (int)(key >> kCutShift) - (int)base;
    return b < 0 ? 0 : (b >= kCutBuckets ? kCutBuckets - 1 : b);
}

// 2^p by the hardware's base-2 exponential (relative error below 2^-22; p >= -8 here).
__device__ __forceinline__ float exp2f_approx(float p) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
    return r;
}

// Fixed-point weight -log2(1 - a_c) * 256 (rounded down) of an item on the tile of pixel columns
// [x0, x1] and rows [y0, y1], with a_c a lower bound of the item's alpha at every pixel centre
// there; 0 if that bound is below 1/255. The exponent's quadratic form is convex, so over the
// tile its maximum is at one of the four corner pixels; a_c takes a relative 1e-4 off that corner
// value, far more than the blend's own rounding of the exponent and the error of the hardware's
// base-2 logarithm and exponential used here (below 2^-21). fc: the column anchor of the image of
// the item that every column of the tile uses; lo2: log2 of the item's opacity.
__device__ __forceinline__ uint32_t cover_weight(float4 ra, float4 rb, float lo2, float fc, int r0, int x0, int x1,
                                                 int y0, int y1) {
    float qmax = 0.f;
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
        const float dy = __fsub_rn((float)((cy ? y1 : y0) - r0), ra.y);
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
            const float t = __fsub_rn(__fsub_rn(__fsub_rn((float)(cx ? x1 : x0), fc), ra.x), rb.y * dy);
            qmax = fmaxf(qmax, rb.x * t * t + rb.z * dy * dy);
        }
    }
    const float lp = lo2 - 0.5f * kLog2e * qmax;
    if (!(lp >= -7.99f)) return 0u;  // alpha < 1/255 (or the opacity is 0)
    const float ac = fminf(exp2f_approx(lp), kAlphaMax) * (1.f - 1e-4f);
    if (!(ac >= 1.f / 255.f)) return 0u;
    return (uint32_t)(-__log2f(1.f - ac) * 256.f);
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void red_add_v4(float4* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

}  // namespace odgs
