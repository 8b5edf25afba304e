// Truncation of the tile lists at saturated tiles (sm_103a). Runs in the binning, before the
// depth sort, on the preprocess's per-item records:
//   k_cover   per depth bucket and tile, the fixed-point sum of -log2(1 - a_c) over the items
//             whose alpha is at least a_c >= 1/255 at every pixel centre of the tile
//             (cover_weight); an item is examined only if its ellipse is wide enough to hold a
//             tile's pixel centres, by a whole warp, and only on the tiles of each of its tile
//             rows that lie within its ellipse (inner_tiles)
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
    // the pixel centres of a tile fit in the ellipse {q <= Qb} only if its minor axis is at least
    // the tile's smaller side minus one pixel: 2 sqrt(Qb lambda_min) >= min(tw, th) - 1, with
    // Sigma_2D from the slice form (C = 1 / gamma, B = beta C, A = 1 / a + beta B) and
    // lambda_min = det / lambda_max, det = 1 / (a gamma). A filter only (relaxed by 10 %, in the
    // hardware's approximate reciprocal and square root): the weights decide.
    const float C = __fdividef(1.f, rb.z), B = rb.y * C, A = __fdividef(1.f, rb.x) + rb.y * B;
    const float h = 0.5f * (A - C), h2 = h * h + B * B;
    const float lmax = 0.5f * (A + C) + h2 * rsqrtf(fmaxf(h2, 1e-30f));
    const float lmin = __fdividef(1.f, rb.x * rb.z * lmax);
    const float d = (float)(min(tw, th) - 1);
    return 4.f * rb.w * lmin >= 0.81f * d * d;
}

}  // namespace

// Tile columns [start, start + n) (mod tiles_x) of tile row ty whose four corner pixels all lie in
// the ellipse q <= Q of an item: the slice of the ellipse at a pixel row dy is the interval
// |dx - beta dy| <= sqrt((Q - gamma dy^2) / a), the box of the tile's pixel centres lies in the
// ellipse iff its corners do, so the columns are those within both of its rows' slices. Only a
// filter, in the hardware's approximate square root (cover_weight decides each tile; a tile missed
// here only weakens the bound). ia = 1 / a.
__device__ __forceinline__ void inner_tiles(float4 ra, float4 rb, float ia, float Q, int c0, int r0, const ViewDev& V,
                                            int ty, int tw, int th, int& start, int& n) {
    start = 0;
    n = 0;
    const int y0 = ty * th, y1 = min(y0 + th - 1, V.H - 1);
    const float dy0 = (float)(y0 - r0) - ra.y, dy1 = (float)(y1 - r0) - ra.y;
    const float h0 = (Q - rb.z * dy0 * dy0) * ia, h1 = (Q - rb.z * dy1 * dy1) * ia;
    if (!(h0 > 0.f && h1 > 0.f)) return;
    const float s0 = h0 * rsqrtf(h0), s1 = h1 * rsqrtf(h1);
    const float lo = fmaxf(rb.y * dy0 - s0, rb.y * dy1 - s1), hi = fminf(rb.y * dy0 + s0, rb.y * dy1 + s1);
    if (!(hi - lo >= (float)(tw - 1))) return;
    const float span = 4.f * (float)V.W;  // clamp before the conversions
    const float xl = fminf(fmaxf((float)c0 + ra.x + lo, -span), span);
    const float xh = fminf(fmaxf((float)c0 + ra.x + hi, -span), span);
    const float itw = 1.f / (float)tw;  // exact: tw is 8, 16 or 32
    const int tlo = (int)ceilf(xl * itw), thi = (int)floorf((xh - (float)(tw - 1)) * itw);
    if (thi < tlo) return;
    if (V.model == 0) {
        n = min(thi - tlo + 1, V.tiles_x);
        start = ((tlo % V.tiles_x) + V.tiles_x) % V.tiles_x;
    } else {
        const int a0 = max(tlo, 0), a1 = min(thi, V.tiles_x - 1);
        if (a1 >= a0) { start = a0; n = a1 - a0 + 1; }
    }
}

constexpr int kCoverSlots = 128;  // (item, tile row) runs a warp holds before it takes their tiles

// The per-lane item of a round of k_cover, as the lanes that take its tiles read it (shuffles).
struct CoverItem {
    float4 ra, rb;
    float lo2;
    int c0, r0, vi;
    uint32_t bucket;
};

// Takes the tiles of the warp's listed runs, 32 at a time: each lane finds its run by a binary
// search over the runs' prefix counts and the run's item by shuffles from the item's lane.
__device__ __forceinline__ void cover_flush(const SatArgs& a, const CoverItem& it, int4* run, int* pre, int* cnt,
                                            int lane) {
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
    for (int g0 = 0; g0 < tot; g0 += 32) {
        const int g = g0 + lane;
        int lo = 0, hi = nr - 1;  // the last run starting at or before g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const int4 R = run[lo];
        const int src = R.w;
        const float4 A = make_float4(__shfl_sync(full, it.ra.x, src), __shfl_sync(full, it.ra.y, src),
                                     __shfl_sync(full, it.ra.z, src), __shfl_sync(full, it.ra.w, src));
        const float4 Bq = make_float4(__shfl_sync(full, it.rb.x, src), __shfl_sync(full, it.rb.y, src),
                                      __shfl_sync(full, it.rb.z, src), 0.f);
        const float lo2 = __shfl_sync(full, it.lo2, src);
        const int c0 = __shfl_sync(full, it.c0, src), r0 = __shfl_sync(full, it.r0, src);
        const int vi = __shfl_sync(full, it.vi, src);
        const uint32_t bucket = __shfl_sync(full, it.bucket, src);
        if (g >= tot) continue;
        const ViewDev& V = a.views[vi];
        int tx = R.y + (g - pre[lo]);
        if (tx >= V.tiles_x) tx -= V.tiles_x;
        const int x0 = tx * a.tile_w, x1 = x0 + a.tile_w - 1;
        const int y0 = R.x * a.tile_h, y1 = min(y0 + a.tile_h - 1, V.H - 1);
        int sh = 0;
        if (V.model == 0) {  // a tile split by the seam (two images of the item) adds nothing
            sh = seam_shift(x0, c0, A.x, V.W);
            if (seam_shift(x1, c0, A.x, V.W) != sh) continue;
        }
        const uint32_t w = cover_weight(A, Bq, lo2, (float)(c0 + sh), r0, x0, x1, y0, y1);
        if (w) atomicAdd(a.cover + (size_t)bucket * a.total_tiles + (size_t)V.tile_base + (size_t)R.x * V.tiles_x + tx, w);
    }
    __syncwarp();
    if (lane == 0) *cnt = 0;
    __syncwarp();
}

// Every lane takes one item; candidates list the runs of inner tiles of their tile rows, one tile
// row per step for all lanes, in the warp's shared list, which the warp empties (cover_flush)
// whenever another step could overfill it.
__global__ void __launch_bounds__(256, 4) k_cover(SatArgs a) {
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
        uint4 rc = make_uint4(0u, 0u, 0u, 0u);
        CoverItem it;
        it.ra = make_float4(0.f, 0.f, 0.f, 0.f);
        it.rb = make_float4(1.f, 0.f, 1.f, 0.f);
        it.lo2 = 0.f;
        it.c0 = it.r0 = it.vi = 0;
        it.bucket = 0u;
        bool cand = false;
        if (item < a.n_items) {
            rc = a.rect[item];
            if (rc.y > 0u) {
                it.rb = a.rec_b[item];
                cand = cover_candidate(rc, it.rb, a.tile_w, a.tile_h);
            }
        }
        float Q = 0.f, ia = 0.f;
        const int nb = cand ? (int)(rc.x >> 16) : 0, ty0 = (int)(rc.x & 0xFFFFu);
        if (cand) {
            it.ra = a.rec_a[item];
            unpack_anchor(it.ra.z, it.c0, it.r0);
            it.vi = (int)(item / (uint32_t)a.n_per_view);
            it.lo2 = __log2f(it.ra.w);
            Q = 2.f * kLn2 * (it.lo2 + kLog2_255);  // 2 ln(255 o)
            ia = __fdividef(1.f, it.rb.x);
            it.bucket = (uint32_t)depth_bucket(a.dkey[item], a.base);
        }
        const int steps = __reduce_max_sync(full, (unsigned)nb);
        for (int b = 0; b < steps; ++b) {
            if (b < nb) {
                int st0, n;
                inner_tiles(it.ra, it.rb, ia, Q, it.c0, it.r0, a.views[it.vi], ty0 + b, a.tile_w, a.tile_h, st0, n);
                if (n > 0) s_run[warp][atomicAdd(&s_cnt[warp], 1)] = make_int4(ty0 + b, st0, n, lane);
            }
            __syncwarp();
            if (s_cnt[warp] > kCoverSlots - 32) cover_flush(a, it, s_run[warp], s_pre[warp], &s_cnt[warp], lane);
        }
        __syncwarp();
        if (s_cnt[warp] > 0) cover_flush(a, it, s_run[warp], s_pre[warp], &s_cnt[warp], lane);
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
