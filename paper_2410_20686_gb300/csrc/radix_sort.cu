// Stable LSD radix sort of 32-bit keys with 32-bit values (sm_103a), used twice per frame:
//   1. (view, Gaussian) items by the bits of their FP32 radial depth   ("sorting by depth",
//      Sec. 3.1), ties kept in item order;
//   2. the (tile, Gaussian) pairs, emitted in depth order, by tile id.
// Together they give every tile its Gaussians in (depth, index) order, the same order as one
// stable sort of 64-bit (tile | depth) keys, with far fewer bytes moved.
//
// One histogram kernel counts the digits of all passes in a single read of the keys; each
// pass is then one "onesweep" kernel (Adinets & Merrill 2022): a CTA ranks a 2048- or 4096-key
// tile in shared memory (warp-level ranking by ballots or a match keeps it stable), publishes its per-digit counts,
// obtains the exclusive prefix of all earlier tiles by decoupled look-back, and writes its keys
// digit-run by digit-run (coalesced). The CTAs are persistent (as many as fit on the GPU, each
// claiming tiles in order), so a sort sized for a capacity far above its keys launches no idle
// CTAs. Look-back waits are bounded: a CTA that has read the
// look-back words `wait_limit` times without reaching an inclusive prefix sets kStTimeout in the
// status word and finishes with a partial prefix; its out-of-range writes are skipped, and every
// consumer of the sorted arrays bounds the indices it reads.
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItemsMax = 16;  // 4096 keys per CTA for sorts of at least kLargeSort keys, else 2048
constexpr size_t kLargeSort = 1u << 19;  // measured: the 1M-item depth sort is faster with 4096-key tiles
constexpr int kRadix = 256;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;

__global__ void __launch_bounds__(256) k_radix_hist(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_ptr,
                                                    int begin_bit, int n_passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[4][kRadix];
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t n = *n_ptr;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    // warp-uniform trip count so every lane takes part in the match
    for (uint32_t base = gwarp * 32u; base < n; base += nwarps * 32u) {
        const uint32_t idx = base + lane;
        const bool valid = idx < n;
        const uint32_t k = valid ? keys[idx] : 0u;
        // the low digits of the keys (depths, tile ids) are spread over many bins: one shared
        // atomic per key; the top digit takes few values (the exponent byte of a positive float
        // depth), so equal digits of the warp are counted with one atomic
        for (int p = 0; p + 1 < n_passes; ++p) {
            const uint32_t d = (k >> (begin_bit + 8 * p)) & 0xFFu;
            if (valid) atomicAdd(&h[p][d], 1u);
        }
        {
            const int p = n_passes - 1;
            const uint32_t d = (k >> (begin_bit + 8 * p)) & 0xFFu;
            const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u);
            if (valid && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_passes * kRadix; i += blockDim.x) {
        uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kSortWarps; ++i) {
        uint32_t s = s_warp[i];
        if (i < w) wpre += s;
        tot += s;
    }
    total = tot;
    __syncthreads();
    return wpre + x - v;
}

template <int kSortItems>
__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         const uint32_t* __restrict__ n_ptr, int shift,
                                                         int bits, int use_match, const uint32_t* __restrict__ hist,
                                                         uint32_t* lookback, uint32_t* tile_ctr, uint32_t* status,
                                                         uint32_t wait_limit) {
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp_hist[kSortWarps][kRadix];
    __shared__ uint32_t s_digit_excl[kRadix];
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_keys[kSortThreads * kSortItems];
    __shared__ uint32_t s_vals[kSortThreads * kSortItems];
    __shared__ uint32_t s_scan[kSortWarps];
    __shared__ uint32_t s_gex[kRadix];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = *n_ptr;
    const uint32_t mask = (1u << bits) - 1u;
    const uint32_t lt = (1u << lane) - 1u;
    // global digit offset of this pass (exclusive scan of the global histogram), the same for
    // every tile
    uint32_t tot;
    s_gex[tid] = block_excl_scan_256(hist[tid], s_scan, tot);

    // Persistent: the grid holds at most the CTAs that fit on the GPU at once (the pair buffer's
    // capacity, which sizes the sort, is far above the pairs a frame keeps), and each CTA claims
    // tiles in order until they run out. A tile waits only on tiles claimed before it, by CTAs
    // that are running, so the look-back always progresses. When the grid has a CTA for every
    // tile, the CTAs' first claims take them all, and a CTA stops after its first tile.
    const uint32_t per_cta = (uint32_t)(kSortThreads * kSortItems);
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
        for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&s_warp_hist[0][0])[i] = 0u;
        __syncthreads();
        const uint32_t tile = s_tile;
        const uint32_t base = tile * per_cta;
        if (base >= n) break;  // CTA-uniform: every tile has been claimed

        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        const uint32_t wbase = base + (uint32_t)warp * (32u * kSortItems);
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const uint32_t idx = wbase + (uint32_t)i * 32u + (uint32_t)lane;
            const bool valid = idx < n;
            key[i] = valid ? kin[idx] : 0u;
            val[i] = valid ? vin[idx] : 0u;
        }
        // stable warp-level ranking: items are ordered by (warp, i, lane).
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const uint32_t idx = wbase + (uint32_t)i * 32u + (uint32_t)lane;
            const bool valid = idx < n;
            const uint32_t d = (key[i] >> shift) & mask;
            // lanes holding the same digit: a warp match costs more the more distinct digits the
            // warp holds, so it ranks the last (most significant) pass, where they are few; the
            // others take one ballot per digit bit (an invalid lane's peers are never used)
            uint32_t peers;
            if (use_match) {
                peers = __match_any_sync(0xffffffffu, valid ? d : (0x100u | (uint32_t)lane));
            } else {
                peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    if (b < bits) {
                        const bool bit = (d >> b) & 1u;
                        const uint32_t bb = __ballot_sync(0xffffffffu, bit);
                        peers &= bit ? bb : ~bb;
                    }
                }
            }
            const uint32_t before = valid ? s_warp_hist[warp][d] : 0u;
            __syncwarp();
            if (valid && lane == (uint32_t)(__ffs(peers) - 1)) s_warp_hist[warp][d] = before + (uint32_t)__popc(peers);
            __syncwarp();
            rank[i] = before + (uint32_t)__popc(peers & lt);
        }
        __syncthreads();
        // per digit (one thread each): exclusive prefix over warps, CTA count
        uint32_t cnt = 0;
        {
            const int d = tid;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t c = s_warp_hist[w][d];
                s_warp_hist[w][d] = cnt;
                cnt += c;
            }
        }
        // publish this tile's count for digit tid
        uint32_t* my = lookback + (size_t)tile * kRadix + tid;
        if (tile == 0) {
            atomicExch(my, kFlagPrefix | cnt);
        } else {
            atomicExch(my, kFlagAgg | cnt);
        }
        const uint32_t dex = block_excl_scan_256(cnt, s_scan, tot);
        s_digit_excl[tid] = dex;
        // decoupled look-back for digit tid
        uint32_t excl = 0;
        if (tile > 0) {
            int j = (int)tile - 1;
            uint32_t reads = 0;
            while (j >= 0) {
                if (reads++ >= wait_limit) {  // every read counts, so a limit of 0 gives up at once
                    atomicOr(status, kStTimeout);
                    break;
                }
                const uint32_t e = ld_volatile(lookback + (size_t)j * kRadix + tid);
                const uint32_t flag = e & ~kCountMask;
                if (flag == 0u) {
                    __nanosleep(32);
                    continue;
                }
                excl += e & kCountMask;
                if (flag == kFlagPrefix) break;
                --j;
            }
            atomicExch(my, kFlagPrefix | (excl + cnt));
        }
        s_base[tid] = s_gex[tid] + excl - dex;
        __syncthreads();
        // scatter into shared memory in sorted order within the tile
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const uint32_t idx = wbase + (uint32_t)i * 32u + (uint32_t)lane;
            if (idx < n) {
                const uint32_t d = (key[i] >> shift) & mask;
                const uint32_t pos = s_digit_excl[d] + s_warp_hist[warp][d] + rank[i];
                s_keys[pos] = key[i];
                s_vals[pos] = val[i];
            }
        }
        __syncthreads();
        const uint32_t count = min(per_cta, n - base);
        for (uint32_t p = tid; p < count; p += kSortThreads) {
            const uint32_t k = s_keys[p];
            const uint32_t d = (k >> shift) & mask;
            const uint32_t dst = s_base[d] + p;
            if (dst < n) {  // only false after a look-back that gave up (status already set)
                kout[dst] = k;
                vout[dst] = s_vals[p];
            }
        }
        if ((n + per_cta - 1) / per_cta <= gridDim.x) break;
        // the next tile's first barrier orders these reads of s_keys, s_vals and s_base before
        // its writes; s_tile and s_warp_hist are not read here
    }
}

int radix_passes(int bits) { return (bits + 7) / 8; }

// Look-back words for the smaller (2048-key) tile, which needs the most.
size_t radix_lookback_words(size_t max_items) {
    const size_t per = kSortThreads * (kSortItemsMax / 2);
    size_t tiles = (max_items + per - 1) / per;
    return (tiles ? tiles : 1) * kRadix;
}

// Sorts (k[0], v[0]) by key bits [0, bits); returns the buffer index (0 or 1) that holds the
// result. scratch: hist [4 * 256] + tile counters [4] + lookback [radix_lookback_words]. With
// hist_ready the digit histograms of all passes are already in hist (counted by the producer).
cudaError_t launch_radix_sort(uint32_t* k[2], uint32_t* v[2], const uint32_t* n_ptr, size_t max_items, int bits,
                              uint32_t* hist, uint32_t* tile_ctrs, uint32_t* lookback, uint32_t* status, int num_sms,
                              cudaStream_t st, int* result_buf, int* launches, bool hist_ready, uint32_t wait_limit,
                              int lb_regions) {
    const int passes = radix_passes(bits);
    *result_buf = 0;
    if (passes == 0 || max_items == 0) return cudaSuccess;
    cudaError_t e;
    // tile counters placed kCtrBytes before the look-back regions are cleared with them
    const bool ctr_with_lb = lb_regions >= passes &&
                             reinterpret_cast<uint8_t*>(lookback) == reinterpret_cast<uint8_t*>(tile_ctrs) + kCtrBytes;
    if (!ctr_with_lb && (e = cudaMemsetAsync(tile_ctrs, 0, sizeof(uint32_t) * 4, st)) != cudaSuccess) return e;
    if (!hist_ready) {
        if ((e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 4 * kRadix, st)) != cudaSuccess) return e;
        int hblocks = (int)min((max_items + 255) / 256, (size_t)num_sms * 8);
        hblocks = max(hblocks, 1);
        k_radix_hist<<<hblocks, 256, 0, st>>>(k[0], n_ptr, 0, passes, hist);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 1;
    }
    static bool carveout_set = false;  // all of the SM's shared memory for the onesweep CTAs
    if (!carveout_set) {
        cudaFuncSetAttribute(k_onesweep<kSortItemsMax>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_onesweep<kSortItemsMax / 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        carveout_set = true;
    }
    const bool large = max_items >= kLargeSort;
    const int per_cta = kSortThreads * (large ? kSortItemsMax : kSortItemsMax / 2);
    const size_t lb_words = radix_lookback_words(max_items);
    const int tiles = (int)((max_items + per_cta - 1) / per_cta);
    // persistent CTAs: as many as fit at once, at most one per tile
    static int resident[2] = {0, 0};
    int& res = resident[large ? 1 : 0];
    if (res == 0) {
        int per_sm = 0;
        if (large)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<kSortItemsMax>, kSortThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<kSortItemsMax / 2>, kSortThreads, 0);
        res = max(per_sm, 1);
    }
    const int grid = max(min(tiles, res * num_sms), 1);
    int cur = 0;
    // with a look-back region per pass, one memset clears them all; else the one region is
    // cleared before every pass
    const bool regions = lb_regions >= passes;
    if (regions && (e = cudaMemsetAsync(ctr_with_lb ? static_cast<void*>(tile_ctrs) : static_cast<void*>(lookback), 0,
                                        (ctr_with_lb ? kCtrBytes : 0) + sizeof(uint32_t) * lb_words * passes, st)) !=
                       cudaSuccess)
        return e;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const int pbits = min(8, bits - shift);
        uint32_t* lb = regions ? lookback + (size_t)p * lb_words : lookback;
        if (!regions && (e = cudaMemsetAsync(lb, 0, sizeof(uint32_t) * lb_words, st)) != cudaSuccess) return e;
        if (large)
            k_onesweep<kSortItemsMax><<<grid, kSortThreads, 0, st>>>(
                k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], n_ptr, shift, pbits, p == passes - 1 ? 1 : 0,
                hist + p * kRadix, lb, tile_ctrs + p, status, wait_limit);
        else
            k_onesweep<kSortItemsMax / 2><<<grid, kSortThreads, 0, st>>>(
                k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], n_ptr, shift, pbits, p == passes - 1 ? 1 : 0,
                hist + p * kRadix, lb, tile_ctrs + p, status, wait_limit);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 1;
        cur ^= 1;
    }
    *result_buf = cur;
    return cudaSuccess;
}

}  // namespace odgs
