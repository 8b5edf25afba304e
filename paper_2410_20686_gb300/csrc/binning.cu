// Tile binning of the depth-sorted items (sm_103a):
//   k_count_blocks  per block of 512 depth-sorted items: number of (tile, item) pairs
//   k_scan_blocks   exclusive scan of the block totals (one CTA) + capacity check
//   k_emit          each item writes one (tile id, item) pair per tile its footprint meets, in
//                   depth order, at its exclusive-scan offset, and counts the tile sort's digits;
//                   items with more than 32 pairs are queued for k_emit_big; pairs beyond the
//                   capacity are dropped (status bit kStCapacity set by k_scan_blocks)
//   k_emit_big      the queued items, one warp each
//   k_tile_ranges   [start, end) of every tile's run in the tile-sorted pair list
// An item's rect is (ty0 | bands << 16, number of tiles, spans of bands 0 and 1), rect2 the spans
// of bands 2..5; the columns of further bands are recomputed from its records by band_columns
// (odgs_common.cuh), exactly as the preprocess counted them. A big item's pairs over its stored
// bands are one flat range that the warp writes 32 at a time; pole-stretched Gaussians can cover
// hundreds of tiles. With truncated lists (saturation.cu) an item writes only the pairs of the
// tiles that keep its depth bucket, compacted in its tile order; the scan uses the kept counts,
// and items keep the thread or warp emission that their whole footprint would take.
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 2;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t rect_tiles(uint4 r) { return r.y; }

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* s) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    __syncthreads();
    return t;
}

// Tiles t of one row run [row + s, row + s + c) (mod tiles_x) with cut[t] >= b, from bucket b's
// prefix counts G over the tiles.
__device__ __forceinline__ uint32_t kept_in_run(const uint32_t* G, uint32_t row, int s, int c, int tiles_x) {
    const int first = min(c, tiles_x - s);
    uint32_t n = G[row + (uint32_t)(s + first)] - G[row + (uint32_t)s];
    if (c > first) n += G[row + (uint32_t)(c - first)] - G[row];
    return n;
}

// Span (start | count << 16) of stored band b < 6, without a dynamically indexed array.
__device__ __forceinline__ uint32_t stored_span(uint4 rc, const uint4* rect2, uint32_t idx, int b) {
    if (b == 0) return rc.z;
    if (b == 1) return rc.w;
    const uint4 r2 = rect2[idx];
    return b == 2 ? r2.x : (b == 3 ? r2.y : (b == 4 ? r2.z : r2.w));
}

// Pairs per block of 512 depth-sorted items. With truncated lists, the kept pairs of each item
// (its tiles whose cut keeps its depth bucket), stored per position for the emission: per row
// band two prefix-count loads, the bands of items with more than six (whose columns are not
// stored) computed by the warp, one band per lane.
__global__ void __launch_bounds__(kScanThreads) k_count_blocks(BinArgs a) {
    __shared__ unsigned long long s[kScanThreads / 32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t base = blockIdx.x * kScanTile;
    // the tile ranges of this binning start from 0 (k_tile_ranges writes the non-empty ones)
    if (a.ranges_zero)
        for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < a.n_ranges; t += gridDim.x * blockDim.x)
            a.ranges_zero[t] = make_uint2(0u, 0u);
    unsigned long long c = 0ull;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        const uint32_t k = base + i;
        uint4 rc = make_uint4(0u, 0u, 0u, 0u);
        uint32_t idx = 0u;
        if (k < a.n_items) {
            idx = a.sorted_idx[k];
            // idx >= n_items only after a depth sort that gave up (status already set)
            if (idx < a.n_items) rc = a.rect[idx];
        }
        if (!a.G) {
            c += rc.y;
            continue;
        }
        const int nb = (int)(rc.x >> 16), ty0 = (int)(rc.x & 0xFFFFu);
        const int bk = k < a.n_items ? depth_bucket(a.sorted_keys[k], a.base) : 0;
        const uint32_t* G = a.G + (size_t)bk * (a.total_tiles + 1u);
        // every tile of the frame keeps this bucket (the items in front of the first cut, among
        // them the near, large ones with many bands): the whole footprint
        const bool all = rc.y > 0u && G[a.total_tiles] == a.total_tiles;
        uint32_t kept = all ? rc.y : 0u;
        if (rc.y > 0u && !all && nb <= 6) {
            const ViewDev& V = a.views[idx / (uint32_t)a.n_per_view];
            const uint4 r2 = nb > 2 ? a.rect2[idx] : make_uint4(0u, 0u, 0u, 0u);
            for (int b = 0; b < nb; ++b) {
                const uint32_t sp = b == 0 ? rc.z : (b == 1 ? rc.w : (b == 2 ? r2.x : (b == 3 ? r2.y : (b == 4 ? r2.z : r2.w))));
                const uint32_t row = (uint32_t)V.tile_base + (uint32_t)(ty0 + b) * (uint32_t)V.tiles_x;
                if (sp >> 16) kept += kept_in_run(G, row, (int)(sp & 0xFFFFu), (int)(sp >> 16), V.tiles_x);
            }
        }
        // items of more bands (near, large Gaussians, which cluster at the front of the depth
        // order): queued for k_count_big, which spreads them over all warps
        const bool many = rc.y > 0u && !all && nb > 6;
        const unsigned m = __ballot_sync(full, many);
        if (m) {
            uint32_t slot = 0u;
            if (lane == __ffs(m) - 1) slot = atomicAdd(&a.hdr->n_count_big, (uint32_t)__popc(m));
            slot = __shfl_sync(full, slot, __ffs(m) - 1);
            if (many) a.big[slot + __popc(m & ((1u << lane) - 1u))] = make_uint2(k, 0u);
        }
        if (many) continue;  // k_count_big writes its word and adds its pairs to the block's sum
        if (k < a.n_items) a.kcount[k] = kept | ((uint32_t)bk << 26);
        c += kept;
    }
    c = block_sum_u64(c, s);
    if (threadIdx.x == 0) a.block_sums[blockIdx.x] = c;
}

// Kept pairs of the queued items of more than six bands, one warp per item (static round robin),
// added to their block's sum.
__global__ void __launch_bounds__(256) k_count_big(BinArgs a) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t nq = a.hdr->n_count_big;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nq; i += nwarps) {
        const uint32_t k = a.big[i].x;
        const uint32_t idx = a.sorted_idx[k];
        const uint4 rc = a.rect[idx];
        const int bk = depth_bucket(a.sorted_keys[k], a.base);
        const ViewDev& V = a.views[idx / (uint32_t)a.n_per_view];
        const Footprint fp = make_footprint(a.rec_a[idx], a.rec_b[idx]);
        int jlo, jhi;
        footprint_rows(fp, V.H, jlo, jhi);
        const uint32_t* G = a.G + (size_t)bk * (a.total_tiles + 1u);
        const int nb = (int)(rc.x >> 16), ty0 = (int)(rc.x & 0xFFFFu);
        uint32_t tot = 0u;
        for (int gb = 0; gb < nb; gb += 32) {
            const int b = gb + lane;
            int start = 0, cnt = 0;
            if (b < 6) {
                const uint32_t sp = stored_span(rc, a.rect2, idx, b);
                start = (int)(sp & 0xFFFFu);
                cnt = (int)(sp >> 16);
            } else if (b < nb) {
                const int ty = ty0 + b, th = a.tile_h;
                band_columns(fp, max(jlo, ty * th), min(jhi, ty * th + th - 1), V.W, a.tile_w, V.tiles_x, V.model == 0,
                             start, cnt);
            }
            const uint32_t row = (uint32_t)V.tile_base + (uint32_t)(ty0 + b) * (uint32_t)V.tiles_x;
            tot += cnt > 0 ? kept_in_run(G, row, start, cnt, V.tiles_x) : 0u;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(full, tot, o);
        if (lane == 0) {
            a.kcount[k] = tot | ((uint32_t)bk << 26);
            if (tot) atomicAdd(a.block_sums + k / kScanTile, (unsigned long long)tot);
        }
    }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(unsigned long long* __restrict__ block_sums, int nblocks,
                                                      Header* hdr, unsigned long long capacity,
                                                      uint32_t* __restrict__ key_hist) {
    // the tile sort's digit counts, which the emission adds up, start from 0
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) key_hist[i] = 0u;
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
        hdr->n_big = 0u;
        hdr->n_count_big = 0u;
        if (total > capacity) atomicOr(&hdr->status, kStCapacity);
    }
}

// Counts the tile-sort digits of the keys key0 .. key0 + cnt - 1 (a contiguous run) in the block's
// shared histogram. Lanes [lane0, lane0 + nlanes) share the low digit (distinct bins, one atomic
// per key); the first lane adds the higher digits one constant-digit segment at a time, so a row
// of consecutive tiles costs one atomic per higher digit instead of one per key.
// Higher digits (passes 1 and up) of the run of consecutive keys key0 .. key0 + cnt - 1.
__device__ __forceinline__ void count_high(uint32_t key0, int cnt, uint32_t (*s_hist)[256], int passes) {
    if (cnt <= 0) return;
    const uint32_t end = key0 + (uint32_t)cnt;
    for (int p = 1; p < passes; ++p) {
        const int sh = 8 * p;
        uint32_t k = key0;
        while (k < end) {
            const uint32_t seg_end = min(end, ((k >> sh) + 1u) << sh);
            atomicAdd(&s_hist[p][(k >> sh) & 0xFFu], seg_end - k);
            k = seg_end;
        }
    }
}

__device__ __forceinline__ void count_run(uint32_t key0, int cnt, uint32_t (*s_hist)[256], int passes, int lane0,
                                          int nlanes) {
    if (cnt <= 0) return;
    for (int k = lane0; k < cnt; k += nlanes) atomicAdd(&s_hist[0][(key0 + (uint32_t)k) & 0xFFu], 1u);
    if (lane0 != 0) return;
    const uint32_t end = key0 + (uint32_t)cnt;
    for (int p = 1; p < passes; ++p) {
        const int sh = 8 * p;
        uint32_t k = key0;
        while (k < end) {
            const uint32_t seg_end = min(end, ((k >> sh) + 1u) << sh);
            atomicAdd(&s_hist[p][(k >> sh) & 0xFFu], seg_end - k);
            k = seg_end;
        }
    }
}

// Writes the pairs of one row band: columns start .. start + cnt - 1 (mod tiles_x), lanes
// [lane0, lane0 + nlanes) sharing the work, and counts their tile-sort digits. Pairs at or
// beyond the capacity are neither written nor counted.
__device__ __forceinline__ void write_band(uint32_t row, int start, int cnt, int tiles_x, uint32_t idx,
                                           unsigned long long off, unsigned long long capacity, int lane0,
                                           int nlanes, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                           uint32_t (*s_hist)[256], int passes) {
    if (off >= capacity) return;
    if ((unsigned long long)cnt > capacity - off) cnt = (int)(capacity - off);
    for (int k = lane0; k < cnt; k += nlanes) {
        const unsigned long long o = off + (unsigned long long)k;
        int tx = start + k;
        if (tx >= tiles_x) tx -= tiles_x;
        keys[o] = row + (uint32_t)tx;
        vals[o] = idx;
    }
    // digit counts of the (at most two, seam-wrapped) runs of consecutive keys
    const int first = min(cnt, tiles_x - start);
    count_run(row + (uint32_t)start, first, s_hist, passes, lane0, nlanes);
    count_run(row, cnt - first, s_hist, passes, lane0, nlanes);
}

// Spans of the item's first kStoredBands row bands, as the preprocess stored them.
constexpr int kStoredBands = 6;
__device__ __forceinline__ void stored_spans(uint32_t idx, uint4 rc, const EmitArgs& a, uint32_t spans[kStoredBands]) {
    spans[0] = rc.z;
    spans[1] = rc.w;
    if ((rc.x >> 16) > 2u) {
        const uint4 r2 = a.rect2[idx];
        spans[2] = r2.x; spans[3] = r2.y; spans[4] = r2.z; spans[5] = r2.w;
    } else {
        spans[2] = spans[3] = spans[4] = spans[5] = 0u;
    }
}

// Writes the pairs of one row band that keep bucket bk (cut[tile] >= bk), compacted from offset
// off by one thread, and counts their digits; returns the offset after them.
__device__ __forceinline__ unsigned long long write_band_kept(uint32_t row, int start, int cnt, int tiles_x,
                                                              uint32_t idx, int bk, unsigned long long off,
                                                              const EmitArgs& a, uint32_t (*s_hist)[256]) {
    for (int k = 0; k < cnt; ++k) {
        int tx = start + k;
        if (tx >= tiles_x) tx -= tiles_x;
        const uint32_t key = row + (uint32_t)tx;
        if ((int)__ldg(a.cut + key) < bk) continue;
        if (off < a.capacity) {
            a.keys[off] = key;
            a.vals[off] = idx;
            for (int p = 0; p < a.key_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 0xFFu], 1u);
        }
        ++off;
    }
    return off;
}

// Emits all pairs of one item from offset off, by one thread. The spans of the item's first
// kStoredBands row bands were stored by the preprocess; further bands are recomputed (same
// functions). bk >= 0: only the pairs of tiles that keep depth bucket bk.
__device__ __forceinline__ void emit_item_thread(uint32_t idx, uint4 rc, unsigned long long off, const EmitArgs& a,
                                                 uint32_t (*s_hist)[256], int bk) {
    const ViewDev& V = a.views[idx / (uint32_t)a.n_per_view];
    const int ty0 = (int)(rc.x & 0xFFFFu), nb = (int)(rc.x >> 16);
    const int th = a.tile_h;
    uint32_t spans[kStoredBands];
    stored_spans(idx, rc, a, spans);
#pragma unroll
    for (int b = 0; b < kStoredBands; ++b) {  // constant indices: the spans stay in registers
        if (b >= nb) break;
        const uint32_t row = (uint32_t)V.tile_base + (uint32_t)(ty0 + b) * (uint32_t)V.tiles_x;
        const int cnt = (int)(spans[b] >> 16);
        if (bk >= 0) {
            off = write_band_kept(row, (int)(spans[b] & 0xFFFFu), cnt, V.tiles_x, idx, bk, off, a, s_hist);
            continue;
        }
        write_band(row, (int)(spans[b] & 0xFFFFu), cnt, V.tiles_x, idx, off, a.capacity, 0, 1, a.keys, a.vals,
                   s_hist, a.key_passes);
        off += (unsigned long long)cnt;
    }
    if (nb <= kStoredBands) return;
    Footprint fp = make_footprint(a.rec_a[idx], a.rec_b[idx]);
    int jlo, jhi;
    footprint_rows(fp, V.H, jlo, jhi);
    for (int ty = ty0 + kStoredBands; ty < ty0 + nb; ++ty) {
        int start, cnt;
        band_columns(fp, max(jlo, ty * th), min(jhi, ty * th + th - 1), V.W, a.tile_w, V.tiles_x, V.model == 0, start,
                         cnt);
        const uint32_t row = (uint32_t)V.tile_base + (uint32_t)ty * (uint32_t)V.tiles_x;
        if (bk >= 0) {
            off = write_band_kept(row, start, cnt, V.tiles_x, idx, bk, off, a, s_hist);
            continue;
        }
        write_band(row, start, cnt, V.tiles_x, idx, off, a.capacity, 0, 1, a.keys, a.vals, s_hist, a.key_passes);
        off += (unsigned long long)cnt;
    }
}

// The kept pairs of one item (tiles that keep depth bucket bk), by a whole warp: lanes compute the
// spans of 32 row bands at a time, then the warp takes band after band 32 columns per step and
// writes the kept ones compacted (ballot order = column order).
__device__ __forceinline__ void emit_item_warp_kept(uint32_t idx, uint4 rc, unsigned long long off, int bk,
                                                    const EmitArgs& a, int lane, uint32_t (*s_hist)[256]) {
    const unsigned full = 0xffffffffu;
    const ViewDev& V = a.views[idx / (uint32_t)a.n_per_view];
    const int th = a.tile_h, ty0 = (int)(rc.x & 0xFFFFu), nb = (int)(rc.x >> 16);
    const uint4 r2 = nb > 2 ? a.rect2[idx] : make_uint4(0u, 0u, 0u, 0u);
    Footprint fp{};
    int jlo = 0, jhi = -1;
    if (nb > kStoredBands) {
        fp = make_footprint(a.rec_a[idx], a.rec_b[idx]);
        footprint_rows(fp, V.H, jlo, jhi);
    }
    const unsigned lt = (1u << lane) - 1u;
    for (int gb = 0; gb < nb; gb += 32) {
        const int b = gb + lane;
        int start = 0, cnt = 0;
        if (b < nb) {
            if (b < kStoredBands) {
                const uint32_t sp = b == 0 ? rc.z : (b == 1 ? rc.w : (b == 2 ? r2.x : (b == 3 ? r2.y : (b == 4 ? r2.z : r2.w))));
                start = (int)(sp & 0xFFFFu);
                cnt = (int)(sp >> 16);
            } else {
                const int ty = ty0 + b;
                band_columns(fp, max(jlo, ty * th), min(jhi, ty * th + th - 1), V.W, a.tile_w, V.tiles_x, V.model == 0,
                             start, cnt);
            }
        }
        unsigned nz = __ballot_sync(full, cnt > 0);
        while (nz) {
            const int l = __ffs(nz) - 1;
            nz &= nz - 1u;
            const int c = __shfl_sync(full, cnt, l), s0 = __shfl_sync(full, start, l);
            const uint32_t row = (uint32_t)V.tile_base + (uint32_t)(ty0 + gb + l) * (uint32_t)V.tiles_x;
            for (int k0 = 0; k0 < c; k0 += 32) {
                const int k = k0 + lane;
                uint32_t key = 0u;
                bool kept = false;
                if (k < c) {
                    int tx = s0 + k;
                    if (tx >= V.tiles_x) tx -= V.tiles_x;
                    key = row + (uint32_t)tx;
                    kept = (int)__ldg(a.cut + key) >= bk;
                }
                const unsigned km = __ballot_sync(full, kept);
                if (kept) {
                    const unsigned long long o = off + (unsigned long long)__popc(km & lt);
                    if (o < a.capacity) {
                        a.keys[o] = key;
                        a.vals[o] = idx;
                        for (int p = 0; p < a.key_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 0xFFu], 1u);
                    }
                }
                off += (unsigned long long)__popc(km);
            }
        }
    }
}

// Emits all pairs of one item from offset off, by a whole warp: lanes compute the spans of 32
// row bands at a time, then the warp writes band after band, 32 columns per step.
__device__ __forceinline__ void emit_item_warp(uint32_t idx, unsigned long long off, const EmitArgs& a, int lane,
                                               uint32_t (*s_hist)[256]) {
    const ViewDev& V = a.views[idx / (uint32_t)a.n_per_view];
    const uint4 rc = a.rect[idx];
    const int th = a.tile_h;
    if ((rc.x >> 16) <= (uint32_t)kStoredBands) {  // spans stored by the preprocess
        const int ty0 = (int)(rc.x & 0xFFFFu), nb = (int)(rc.x >> 16);
        uint32_t spans[kStoredBands];
        stored_spans(idx, rc, a, spans);
        // the item's pairs as one range: pair t lies in the band b with cum[b] <= t < cum[b + 1]
        int cum[kStoredBands + 1];
        cum[0] = 0;
#pragma unroll
        for (int b = 0; b < kStoredBands; ++b) cum[b + 1] = cum[b] + (b < nb ? (int)(spans[b] >> 16) : 0);
        if (off >= a.capacity) return;  // pairs beyond the capacity are neither written nor counted
        const int avail = (int)min((unsigned long long)cum[kStoredBands], a.capacity - off);
        const int tiles_x = V.tiles_x;
        for (int t = lane; t < avail; t += 32) {
            int b = 0;
#pragma unroll
            for (int q = 1; q < kStoredBands; ++q) b += t >= cum[q] ? 1 : 0;
            uint32_t sp = spans[0];
            int c0 = 0;
#pragma unroll
            for (int q = 1; q < kStoredBands; ++q) {  // selects: the arrays stay in registers
                sp = b == q ? spans[q] : sp;
                c0 = b == q ? cum[q] : c0;
            }
            int col = (int)(sp & 0xFFFFu) + (t - c0);
            if (col >= tiles_x) col -= tiles_x;
            const uint32_t key = (uint32_t)V.tile_base + (uint32_t)(ty0 + b) * (uint32_t)tiles_x + (uint32_t)col;
            a.keys[off + (unsigned long long)t] = key;
            a.vals[off + (unsigned long long)t] = idx;
            atomicAdd(&s_hist[0][key & 0xFFu], 1u);
        }
        if (a.key_passes > 1 && lane < nb) {  // higher digits: lane b counts the runs of band b
            uint32_t sp = spans[0];
            int c0 = 0;
#pragma unroll
            for (int q = 1; q < kStoredBands; ++q) {
                sp = lane == q ? spans[q] : sp;
                c0 = lane == q ? cum[q] : c0;
            }
            const int c = min(max(avail - c0, 0), (int)(sp >> 16));
            const int start = (int)(sp & 0xFFFFu);
            const uint32_t row = (uint32_t)V.tile_base + (uint32_t)(ty0 + lane) * (uint32_t)tiles_x;
            const int first = min(c, tiles_x - start);
            count_high(row + (uint32_t)start, first, s_hist, a.key_passes);
            count_high(row, c - first, s_hist, a.key_passes);
        }
        return;
    }
    Footprint fp = make_footprint(a.rec_a[idx], a.rec_b[idx]);
    int jlo, jhi;
    footprint_rows(fp, V.H, jlo, jhi);
    if (jlo > jhi) return;
    const int ty0 = jlo / th, ty1 = jhi / th;
    for (int gq = ty0; gq <= ty1; gq += 32) {
        const int ty = gq + lane;
        int start = 0, cnt = 0;
        if (ty <= ty1)
            band_columns(fp, max(jlo, ty * th), min(jhi, ty * th + th - 1), V.W, a.tile_w, V.tiles_x, V.model == 0, start,
                         cnt);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - cnt;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned nz = __ballot_sync(0xffffffffu, cnt > 0);
        while (nz) {
            const int l = __ffs(nz) - 1;
            nz &= nz - 1u;
            const int c = __shfl_sync(0xffffffffu, cnt, l);
            const int s0 = __shfl_sync(0xffffffffu, start, l);
            const int e0 = __shfl_sync(0xffffffffu, excl, l);
            const uint32_t row = (uint32_t)V.tile_base + (uint32_t)(gq + l) * (uint32_t)V.tiles_x;
            write_band(row, s0, c, V.tiles_x, idx, off + (unsigned long long)e0, a.capacity, lane, 32, a.keys, a.vals,
                       s_hist, a.key_passes);
        }
        off += (unsigned long long)total;
    }
}

__device__ __forceinline__ void flush_digits(uint32_t (*s_hist)[256], uint32_t* key_hist, int passes) {
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = s_hist[i >> 8][i & 255];
        if (c) atomicAdd(key_hist + i, c);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_emit(EmitArgs a) {
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_carry;
    __shared__ uint32_t s_hist[4][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t base = blockIdx.x * kScanTile;
    for (int i = tid; i < 4 * 256; i += kScanThreads) s_hist[i >> 8][i & 255] = 0u;
    if (tid == 0) s_carry = a.block_offsets[blockIdx.x];
    __syncthreads();
    for (int round = 0; round < kScanItems; ++round) {
        const uint32_t k = base + (uint32_t)(round * kScanThreads + tid);
        const uint32_t idx = k < a.n_items ? a.sorted_idx[k] : 0u;
        // an index past the end (only after a depth sort that gave up) emits nothing, as in
        // k_count_blocks, so that the offsets of the two kernels agree
        const uint4 rc = (k < a.n_items && idx < a.n_items) ? a.rect[idx] : make_uint4(0u, 0u, 0u, 0u);
        // kept pairs (the scan) and the item's whole footprint (thread or warp emission)
        const uint32_t kw = (a.kcount && k < a.n_items) ? a.kcount[k] : rc.y;
        const uint32_t cnt = a.kcount ? (kw & 0x3FFFFFFu) : rc.y;
        const int bk = (a.kcount && cnt < rc.y) ? (int)(kw >> 26) : -1;
        // block-wide exclusive scan of the counts of this round (items in depth order)
        unsigned long long x = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        unsigned long long off = s_carry + x - cnt, tot = 0ull;
        for (int j = 0; j < kScanThreads / 32; ++j) {
            const unsigned long long v = s_warp[j];
            if (j < w) off += v;
            tot += v;
        }
        __syncthreads();
        if (tid == 0) s_carry += tot;
        // small items: one lane each
        if (cnt > 0u && rc.y <= 32u) emit_item_thread(idx, rc, off, a, s_hist, bk);
        // large items: queued for k_emit_big (whole warps, dynamically scheduled). Depth order
        // clusters the nearest, largest Gaussians into the first blocks, so serving them here
        // would leave a few warps writing most of the pairs.
        const bool big = cnt > 0u && rc.y > 32u;
        const unsigned bigm = __ballot_sync(0xffffffffu, big);
        if (bigm) {  // one queue reservation per warp
            uint32_t base_slot = 0u;
            if (lane == __ffs(bigm) - 1) base_slot = atomicAdd(&a.hdr->n_big, (uint32_t)__popc(bigm));
            base_slot = __shfl_sync(0xffffffffu, base_slot, __ffs(bigm) - 1);
            if (big) a.big[base_slot + __popc(bigm & ((1u << lane) - 1u))] = make_uint2(k, (uint32_t)off);
        }
    }
    flush_digits(s_hist, a.key_hist, a.key_passes);
}

__global__ void __launch_bounds__(256, 4) k_emit_big(EmitArgs a) {
    __shared__ uint32_t s_hist[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) s_hist[i >> 8][i & 255] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t n_big = a.hdr->n_big;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    // static round-robin over the queue: no shared counter to contend on
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_big; i += nwarps) {
        const uint2 e = a.big[i];
        const uint32_t idx = a.sorted_idx[e.x];
        if (a.kcount) {
            const uint4 rc = a.rect[idx];
            const uint32_t kw = a.kcount[e.x];
            if ((kw & 0x3FFFFFFu) < rc.y) {
                emit_item_warp_kept(idx, rc, (unsigned long long)e.y, (int)(kw >> 26), a, lane, s_hist);
                continue;
            }
        }
        emit_item_warp(idx, (unsigned long long)e.y, a, lane, s_hist);
    }
    flush_digits(s_hist, a.key_hist, a.key_passes);
}

// [start, end) of every tile's run. A thread takes 4 consecutive keys (one 16-byte load when the
// array is 16-byte aligned) plus the keys on either side.
__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t* __restrict__ keys, const Header* __restrict__ hdr,
                                                     uint2* __restrict__ ranges, uint32_t total_tiles) {
    const uint32_t n = hdr->n_pairs_sort;
    const uint32_t nq = (n + 3u) / 4u;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0u;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4u * t;
        uint32_t k[4];
        if (vec && i0 + 4u <= n) {
            const uint4 q = *reinterpret_cast<const uint4*>(keys + i0);
            k[0] = q.x; k[1] = q.y; k[2] = q.z; k[3] = q.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) k[r] = (i0 + (uint32_t)r < n) ? keys[i0 + r] : 0xFFFFFFFFu;
        }
        uint32_t prev = i0 > 0u ? keys[i0 - 1u] : 0xFFFFFFFFu;
        const uint32_t next = (i0 + 4u < n) ? keys[i0 + 4u] : 0xFFFFFFFFu;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t i = i0 + (uint32_t)r;
            if (i >= n) break;
            const uint32_t kk = k[r];
            const uint32_t kn = r < 3 ? k[r + 1] : next;
            if (kk < total_tiles) {  // false only after a failed sort (status already set)
                if (i == 0u || prev != kk) ranges[kk].x = i;
                if (i + 1u == n || kn != kk) ranges[kk].y = i + 1u;
            }
            prev = kk;
        }
    }
}

int scan_blocks_for(uint32_t n_items) { return (int)((n_items + kScanTile - 1) / kScanTile); }

cudaError_t launch_binning(const BinArgs& a, cudaStream_t st, int* launches) {
    cudaError_t e;
    const int nb = scan_blocks_for(a.n_items);
    if (a.emit_only) {
        if ((e = cudaMemsetAsync(&a.hdr->n_big, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    } else if (nb > 0) {
        // the kept-count queue counter is 0: cleared by the preprocess's setup and by every scan
        k_count_blocks<<<nb, kScanThreads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 1;
        if (a.G) {
            k_count_big<<<a.num_sms * 8, 256, 0, st>>>(a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            *launches += 1;
        }
    }
    if (!a.emit_only) {
        k_scan_blocks<<<1, 1024, 0, st>>>(a.block_sums, nb, a.hdr, a.capacity, a.key_hist);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 1;
    }
    if (nb == 0 && (e = cudaMemsetAsync(a.key_hist, 0, sizeof(uint32_t) * 4 * 256, st)) != cudaSuccess) return e;
    if (nb > 0) {
        EmitArgs ea{};
        ea.sorted_idx = a.sorted_idx; ea.rect = a.rect; ea.rect2 = a.rect2; ea.rec_a = a.rec_a; ea.rec_b = a.rec_b; ea.views = a.views;
        ea.n_per_view = a.n_per_view; ea.n_items = a.n_items; ea.tile_w = a.tile_w; ea.tile_h = a.tile_h;
        ea.block_offsets = a.block_sums; ea.capacity = a.capacity; ea.keys = a.keys; ea.vals = a.vals;
        ea.big = a.big; ea.hdr = a.hdr;
        ea.key_hist = a.key_hist; ea.key_passes = a.key_passes;
        ea.kcount = a.G ? a.kcount : nullptr;
        ea.cut = a.cut;
        // zeroed by the scan, except when the scan does not run
        if (a.emit_only && (e = cudaMemsetAsync(a.key_hist, 0, sizeof(uint32_t) * 4 * 256, st)) != cudaSuccess) return e;
        k_emit<<<nb, kScanThreads, 0, st>>>(ea);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_emit_big<<<a.num_sms * 8, 256, 0, st>>>(ea);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 2;
    }
    return cudaSuccess;
}

cudaError_t launch_tile_ranges(const uint32_t* keys, const Header* hdr, uint2* ranges, int total_tiles,
                               size_t max_pairs, int num_sms, cudaStream_t st, int* launches, bool zeroed) {
    cudaError_t e;
    if (!zeroed && (e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, st)) != cudaSuccess) return e;
    if (max_pairs == 0) return cudaSuccess;
    int blocks = (int)min((max_pairs / 4 + 255) / 256, (size_t)num_sms * 16);
    k_tile_ranges<<<max(blocks, 1), 256, 0, st>>>(keys, hdr, ranges, (uint32_t)total_tiles);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace odgs
