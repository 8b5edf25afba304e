// Truncation of the tile lists at saturated tiles (sm_103a). Runs in the binning, on a second
// stream beside the depth sort, on the preprocess's per-item records and depth buckets:
//   k_cover   per depth bucket and tile, the fixed-point sum of -log2(1 - a_c) over the items
//             whose alpha is at least a_c >= 1/255 at every pixel centre of the tile
//             (cover_weight); an item is examined only if its ellipse is wide enough to hold
//             six tiles across (cover_candidate), and only on the tiles of each of its tile rows
//             that lie within its ellipse (inner_tiles)
//   k_cut     per tile, the first bucket at which the running sum crosses kCutThreshold: every
//             pixel of the tile stops within the items of that bucket and the nearer ones, so
//             the tile keeps exactly those (a prefix of its depth-ordered list)
//   k_prefix  per bucket b, the exclusive prefix over the tiles of [cut >= b], so that the number
//             of kept tiles in a run of one tile row is two loads
// The binning then counts and writes only the kept pairs (binning.cu). Decisions are taken in
// integers from per-item quantities, so the lists are deterministic, and a rebuild gives the
// same lists.
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

namespace {

__device__ __forceinline__ bool cover_candidate(uint4 rc, float4 rb, int tw, int th) {
    if (rc.y == 0u) return false;
    // items whose ellipse {q <= Qb} has a minor axis of at least six tiles' smaller side less a
    // pixel: 2 sqrt(Qb lambda_min) >= 6 min(tw, th) - 1, with Sigma_2D from the slice form
    // (C = 1 / gamma, B = beta C, A = 1 / a + beta B) and lambda_min = det / lambda_max,
    // det = 1 / (a gamma). Any subset of the items gives a valid bound. Saturation comes from the
    // few largest footprints: on the 1M-Gaussian frame the 2.8K items six tiles across (of the
    // 195K whose ellipse could hold one tile) cover 0.77M tiles and leave 0.4 % more pairs than all
    // of them (2.9M of 15.3M footprint-box pairs, a numpy estimate), where two tiles across (52K
    // items) cover 2.55M tiles. Evaluated in the hardware's approximate reciprocal and square root,
    // relaxed by 10 %.
    const float C = __fdividef(1.f, rb.z), B = rb.y * C, A = __fdividef(1.f, rb.x) + rb.y * B;
    const float h = 0.5f * (A - C), h2 = h * h + B * B;
    const float lmax = 0.5f * (A + C) + h2 * rsqrtf(fmaxf(h2, 1e-30f));
    const float lmin = __fdividef(1.f, rb.x * rb.z * lmax);
    const float d = (float)(6 * min(tw, th) - 1);
    return 4.f * rb.w * lmin >= 0.81f * d * d;
}

}  // namespace

// Tile columns [start, start + n) (mod tiles_x) of tile row ty whose four corner pixels all lie in
// the ellipse q <= Q of an item: the slice of the ellipse at a pixel row dy is the interval
// |dx - beta dy| <= sqrt((Q - gamma dy^2) / a), the box of the tile's pixel centres lies in the
// ellipse iff its corners do, so the columns are those within both of its rows' slices. Only a
// filter, in the hardware's approximate square root (cover_weight decides each tile; a tile missed
// here only weakens the bound). ia = 1 / a.
__device__ __forceinline__ void inner_tiles(float4 ra, float4 rb, float ia, float Q, int c0, int r0, int W, int H,
                                            int tiles_x, int model, int ty, int tw, int th, int& start, int& n) {
    start = 0;
    n = 0;
    const int y0 = ty * th, y1 = min(y0 + th - 1, H - 1);
    const float dy0 = (float)(y0 - r0) - ra.y, dy1 = (float)(y1 - r0) - ra.y;
    const float h0 = (Q - rb.z * dy0 * dy0) * ia, h1 = (Q - rb.z * dy1 * dy1) * ia;
    if (!(h0 > 0.f && h1 > 0.f)) return;
    const float s0 = h0 * rsqrtf(h0), s1 = h1 * rsqrtf(h1);
    const float lo = fmaxf(rb.y * dy0 - s0, rb.y * dy1 - s1), hi = fminf(rb.y * dy0 + s0, rb.y * dy1 + s1);
    if (!(hi - lo >= (float)(tw - 1))) return;
    const float span = 4.f * (float)W;  // clamp before the conversions
    const float xl = fminf(fmaxf((float)c0 + ra.x + lo, -span), span);
    const float xh = fminf(fmaxf((float)c0 + ra.x + hi, -span), span);
    const float itw = 1.f / (float)tw;  // exact: tw is 8, 16 or 32
    const int tlo = (int)ceilf(xl * itw), thi = (int)floorf((xh - (float)(tw - 1)) * itw);
    if (thi < tlo) return;
    if (model == 0) {
        n = min(thi - tlo + 1, tiles_x);
        start = pos_mod(tlo, tiles_x);
    } else {
        const int a0 = max(tlo, 0), a1 = min(thi, tiles_x - 1);
        if (a1 >= a0) { start = a0; n = a1 - a0 + 1; }
    }
}

constexpr int kCoverSlots = 128;  // (item, tile row) runs a warp holds before it takes their tiles

// An item of a round of k_cover in shared memory: written by its lane, read by the lanes that
// take its tile rows and its tiles.
struct CoverItem {
    float4 f0;  // du, dv, log2 o, Q = 2 ln(255 o)
    float4 f1;  // a, beta, gamma, 1 / a
    int4 i0;    // c0, r0, first tile row, tile rows
    int4 i1;    // depth bucket, W, H, tiles_x
    int4 i2;    // tile_base, model, 0, 0
};

// The lane l owning index g of a warp-wide sequence of segments, lane l's segment ending before
// incl_l (inclusive prefix, non-decreasing over the lanes): the number of lanes with incl <= g.
__device__ __forceinline__ int segment_owner(int g, int incl) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
        if (v <= g) lo += step;
    }
    return lo;
}

// Takes the tiles of the warp's listed runs, 32 at a time. Run rs holds the window's first index;
// the runs starting inside the window are marked in a bit mask, so each lane's run is rs plus the
// marks at or before it.
__device__ __forceinline__ void cover_flush(const SatArgs& a, const CoverItem* items, const int4* run, int* pre,
                                            int* cnt, int lane) {
    const unsigned full = 0xffffffffu;
    __syncwarp();
    const int nr = *cnt;
    int tot = 0;
    for (int e0 = 0; e0 < nr; e0 += 32) {
        const int n = e0 + lane < nr ? run[e0 + lane].z : 0;
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += y;
        }
        if (e0 + lane < nr) pre[e0 + lane] = tot + incl - n;
        tot += __shfl_sync(full, incl, 31);
    }
    __syncwarp();
    int rs = 0;
    for (int g0 = 0; g0 < tot; g0 += 32) {
        const int nx = rs + 1 + lane;
        const int p = nx < nr ? pre[nx] : 0x7fffffff;  // p > g0 for every following run
        const unsigned starts = __reduce_or_sync(full, p < g0 + 32 ? (1u << (p - g0)) : 0u);
        const int r = rs + __popc(starts & ((2u << lane) - 1u));
        rs += __popc(__ballot_sync(full, p <= g0 + 32));
        const int g = g0 + lane;
        if (g >= tot) continue;
        const int4 R = run[r];
        const CoverItem& it = items[R.w];
        const int tiles_x = it.i1.w, W = it.i1.y, H = it.i1.z, c0 = it.i0.x;
        int tx = R.y + (g - pre[r]);
        if (tx >= tiles_x) tx -= tiles_x;
        const int x0 = tx * a.tile_w, x1 = x0 + a.tile_w - 1;
        const int y0 = R.x * a.tile_h, y1 = min(y0 + a.tile_h - 1, H - 1);
        const float4 ra = make_float4(it.f0.x, it.f0.y, 0.f, 0.f), rb = it.f1;
        int sh = 0;
        if (it.i2.y == 0) {  // ERP: a tile split by the seam (two images of the item) adds nothing
            sh = seam_shift(x0, c0, ra.x, W);
            if (seam_shift(x1, c0, ra.x, W) != sh) continue;
        }
        const uint32_t w = cover_weight(ra, rb, it.f0.z, (float)(c0 + sh), it.i0.y, x0, x1, y0, y1);
        if (w)
            atomicAdd(a.cover + (size_t)it.i1.x * a.total_tiles + (size_t)it.i2.x + (size_t)R.x * tiles_x + tx, w);
    }
    __syncwarp();
    if (lane == 0) *cnt = 0;
    __syncwarp();
}

// Every lane takes one item and, if it is a candidate, puts it in the warp's shared item list;
// the warp then takes the candidates' tile rows 32 at a time, listing the runs of inner tiles in
// its shared run list, which it empties (cover_flush) whenever another step could overfill it.
__global__ void __launch_bounds__(256, 4) k_cover(SatArgs a) {
    __shared__ CoverItem s_item[8][32];
    __shared__ int4 s_run[8][kCoverSlots];  // tile row, first column, tiles, lane of the item
    __shared__ int s_pre[8][kCoverSlots];   // exclusive prefix of the runs' tiles
    __shared__ int s_cnt[8];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t stride = gridDim.x * blockDim.x;
    if (lane == 0) s_cnt[warp] = 0;
    __syncwarp();
    for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < a.n_items; i0 += stride) {
        const uint32_t item = i0 + threadIdx.x;
        int nb = 0;
        if (item < a.n_items) {
            const uint4 rc = a.rect[item];
            if (rc.y > 0u) {
                const float4 rb = a.rec_b[item];
                if (cover_candidate(rc, rb, a.tile_w, a.tile_h)) {
                    const float4 ra = a.rec_a[item];
                    const ViewDev& V = a.views[item / (uint32_t)a.n_per_view];
                    int c0, r0;
                    unpack_anchor(ra.z, c0, r0);
                    const float lo2 = __log2f(ra.w);
                    CoverItem it;
                    it.f0 = make_float4(ra.x, ra.y, lo2, 2.f * kLn2 * (lo2 + kLog2_255));  // Q = 2 ln(255 o)
                    it.f1 = make_float4(rb.x, rb.y, rb.z, __fdividef(1.f, rb.x));
                    nb = (int)(rc.x >> 16);
                    it.i0 = make_int4(c0, r0, (int)(rc.x & 0xFFFFu), nb);
                    it.i1 = make_int4((int)a.dbucket[item], V.W, V.H, V.tiles_x);
                    it.i2 = make_int4(V.tile_base, V.model, 0, 0);
                    s_item[warp][lane] = it;
                }
            }
        }
        int incl = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(full, incl, 31);
        if (total == 0) continue;
        __syncwarp();
        for (int b0 = 0; b0 < total; b0 += 32) {
            const int g = b0 + lane;
            const int own = segment_owner(g, incl);
            const int first = __shfl_sync(full, incl - nb, own);
            if (g < total) {
                const CoverItem& it = s_item[warp][own];
                const int ty = it.i0.z + (g - first);
                int st0, n;
                inner_tiles(make_float4(it.f0.x, it.f0.y, 0.f, 0.f), it.f1, it.f1.w, it.f0.w, it.i0.x, it.i0.y,
                            it.i1.y, it.i1.z, it.i1.w, it.i2.y, ty, a.tile_w, a.tile_h, st0, n);
                if (n > 0) s_run[warp][atomicAdd(&s_cnt[warp], 1)] = make_int4(ty, st0, n, own);
            }
            __syncwarp();
            if (s_cnt[warp] > kCoverSlots - 32) cover_flush(a, s_item[warp], s_run[warp], s_pre[warp], &s_cnt[warp], lane);
        }
        __syncwarp();
        if (s_cnt[warp] > 0) cover_flush(a, s_item[warp], s_run[warp], s_pre[warp], &s_cnt[warp], lane);
        __syncwarp();  // the next round overwrites the item list
    }
}

__global__ void __launch_bounds__(256) k_cut(const uint32_t* __restrict__ cover, uint8_t* __restrict__ cut,
                                             uint32_t total_tiles) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x) {
        // the bucket sums are each at most the true sum (a wrapped 32-bit sum only makes them
        // smaller), so the cut is never earlier than the bound allows
        uint32_t v[kCutBuckets];
#pragma unroll
        for (int b = 0; b < kCutBuckets; ++b) v[b] = cover[(size_t)b * total_tiles + t];
        unsigned long long cum = 0ull;
        uint8_t c = kCutNone;
#pragma unroll
        for (int b = 0; b < kCutBuckets; ++b) {
            cum += v[b];
            if (c == kCutNone && cum >= kCutThreshold) c = (uint8_t)b;
        }
        cut[t] = c;
    }
}

// One block per bucket: G[b][t] = #{t' < t : cut[t'] >= b}, t = 0 .. total_tiles.
__global__ void __launch_bounds__(1024) k_prefix(const uint8_t* __restrict__ cut, uint32_t* __restrict__ G,
                                                 uint32_t total_tiles) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int b = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* g = G + (size_t)b * (total_tiles + 1u);
    if (threadIdx.x == 0) s_carry = 0u;
    __syncthreads();
    for (uint32_t base = 0; base < total_tiles; base += 4096u) {
        uint32_t f[4], x = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t t = base + 4u * threadIdx.x + (uint32_t)k;
            f[k] = (t < total_tiles && cut[t] >= (uint8_t)b) ? 1u : 0u;
            x += f[k];
        }
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        uint32_t pre = s_carry, tot = 0u;
        for (int k = 0; k < 32; ++k) {
            const uint32_t v = s_warp[k];
            if (k < w) pre += v;
            tot += v;
        }
        pre += incl - x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t t = base + 4u * threadIdx.x + (uint32_t)k;
            if (t < total_tiles) g[t] = pre;
            pre += f[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) g[total_tiles] = s_carry;
}

cudaError_t launch_saturation(const SatArgs& a, int num_sms, cudaStream_t st, int* launches) {
    cudaError_t e;
    if (a.n_items == 0 || a.total_tiles == 0) {
        // no items: nothing is emitted either way; keep the per-item words defined
        return cudaSuccess;
    }
    if ((e = cudaMemsetAsync(a.cover, 0, sizeof(uint32_t) * kCutBuckets * (size_t)a.total_tiles, st)) != cudaSuccess)
        return e;
    const int items_blocks = (int)min((a.n_items + 255u) / 256u, (uint32_t)num_sms * 8u);
    k_cover<<<items_blocks, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int tile_blocks = (int)min((a.total_tiles + 255u) / 256u, (uint32_t)num_sms * 8u);
    k_cut<<<tile_blocks, 256, 0, st>>>(a.cover, a.cut, a.total_tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the prefix tables overwrite the bucket sums, which k_cut has consumed
    k_prefix<<<kCutBuckets, 1024, 0, st>>>(a.cut, a.cover, a.total_tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 3;
    return cudaSuccess;
}

}  // namespace odgs
