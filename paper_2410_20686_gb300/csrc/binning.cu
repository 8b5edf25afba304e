// Tile binning of the depth-sorted items (sm_103a):
//   k_count_blocks  per block of 2048 depth-sorted items: number of (tile, item) pairs
//   k_scan_blocks   exclusive scan of the block totals (one CTA) + capacity check
//   k_emit          each item writes one (tile id, item) pair per tile of its rectangle, in
//                   depth order, at its exclusive-scan offset; pairs beyond the capacity are
//                   dropped (status bit kStCapacity set by k_scan_blocks)
//   k_tile_ranges   [start, end) of every tile's run in the tile-sorted pair list
// A rectangle is tx0 | ntx << 16, ty0 | nty << 16; its columns wrap around the longitude seam
// (tile column (tx0 + k) mod tiles_x).
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t rect_tiles(uint2 r) { return (r.x >> 16) * (r.y >> 16); }

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* s) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kScanThreads) k_count_blocks(const uint32_t* __restrict__ sorted_idx,
                                                              const uint2* __restrict__ rect, uint32_t n_items,
                                                              unsigned long long* __restrict__ block_sums) {
    __shared__ unsigned long long s[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kScanTile;
    unsigned long long c = 0ull;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        uint32_t k = base + i;
        if (k < n_items) c += rect_tiles(rect[sorted_idx[k]]);
    }
    c = block_sum_u64(c, s);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = c;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(unsigned long long* __restrict__ block_sums, int nblocks,
                                                      Header* hdr, unsigned long long capacity) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0ull;
    __syncthreads();
    for (int base = 0; base < nblocks; base += 1024) {
        int i = base + threadIdx.x;
        unsigned long long v = i < nblocks ? block_sums[i] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        unsigned long long wpre = 0ull, tot = 0ull;
        for (int k = 0; k < 32; ++k) {
            unsigned long long sv = s_warp[k];
            if (k < w) wpre += sv;
            tot += sv;
        }
        unsigned long long carry = s_carry;
        if (i < nblocks) block_sums[i] = carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        unsigned long long total = s_carry;
        unsigned long long used = total < capacity ? total : capacity;
        hdr->pairs_emitted = used;
        hdr->n_pairs_sort = (uint32_t)used;
        if (total > capacity) atomicOr(&hdr->status, kStCapacity);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_emit(const uint32_t* __restrict__ sorted_idx,
                                                      const uint2* __restrict__ rect,
                                                      const ViewDev* __restrict__ views, int n_per_view,
                                                      uint32_t n_items,
                                                      const unsigned long long* __restrict__ block_offsets,
                                                      unsigned long long capacity, uint32_t* __restrict__ keys,
                                                      uint32_t* __restrict__ vals) {
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t idx[kScanItems];
    uint2 rc[kScanItems];
    unsigned long long cnt = 0ull;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        uint32_t k = base + j;
        idx[j] = k < n_items ? sorted_idx[k] : 0u;
        rc[j] = k < n_items ? rect[idx[j]] : make_uint2(0u, 0u);
        cnt += rect_tiles(rc[j]);
    }
    // block exclusive scan of the per-thread counts
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    unsigned long long off = block_offsets[blockIdx.x] + x - cnt;
    for (int k = 0; k < w; ++k) off += s_warp[k];
#pragma unroll 1
    for (int j = 0; j < kScanItems; ++j) {
        const uint2 r = rc[j];
        const uint32_t ntx = r.x >> 16, nty = r.y >> 16;
        if (ntx == 0u || nty == 0u) continue;
        const uint32_t tx0 = r.x & 0xFFFFu, ty0 = r.y & 0xFFFFu;
        const int v = (int)(idx[j] / (uint32_t)n_per_view);
        const ViewDev& V = views[v];
        for (uint32_t ty = 0; ty < nty; ++ty) {
            const uint32_t row = (uint32_t)V.tile_base + (ty0 + ty) * (uint32_t)V.tiles_x;
            uint32_t tx = tx0;
            for (uint32_t k = 0; k < ntx; ++k) {
                if (off < capacity) {
                    keys[off] = row + tx;
                    vals[off] = idx[j];
                }
                ++off;
                if (++tx == (uint32_t)V.tiles_x) tx = 0u;
            }
        }
    }
}

__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, const Header* __restrict__ hdr,
                              uint2* __restrict__ ranges, uint32_t total_tiles) {
    const uint32_t n = hdr->n_pairs_sort;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (k >= total_tiles) continue;  // only after a failed sort (status already set)
        if (i == 0u || keys[i - 1] != k) ranges[k].x = i;
        if (i + 1u == n || keys[i + 1] != k) ranges[k].y = i + 1u;
    }
}

int scan_blocks_for(uint32_t n_items) { return (int)((n_items + kScanTile - 1) / kScanTile); }

cudaError_t launch_binning(const BinArgs& a, cudaStream_t st, int* launches) {
    cudaError_t e;
    const int nb = scan_blocks_for(a.n_items);
    if (nb > 0) {
        k_count_blocks<<<nb, kScanThreads, 0, st>>>(a.sorted_idx, a.rect, a.n_items, a.block_sums);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 1;
    }
    k_scan_blocks<<<1, 1024, 0, st>>>(a.block_sums, nb, a.hdr, a.capacity);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 1;
    if (nb > 0) {
        k_emit<<<nb, kScanThreads, 0, st>>>(a.sorted_idx, a.rect, a.views, a.n_per_view, a.n_items, a.block_sums,
                                            a.capacity, a.keys, a.vals);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 1;
    }
    return cudaSuccess;
}

cudaError_t launch_tile_ranges(const uint32_t* keys, const Header* hdr, uint2* ranges, int total_tiles,
                               size_t max_pairs, int num_sms, cudaStream_t st, int* launches) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, st);
    if (e != cudaSuccess) return e;
    if (max_pairs == 0) return cudaSuccess;
    int blocks = (int)min((max_pairs + 255) / 256, (size_t)num_sms * 16);
    k_tile_ranges<<<max(blocks, 1), 256, 0, st>>>(keys, hdr, ranges, (uint32_t)total_tiles);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace odgs
