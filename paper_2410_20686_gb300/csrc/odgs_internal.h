// Launcher interfaces between the C-ABI host code (api.cu) and the kernel files.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "odgs.h"
#include "odgs_common.cuh"

namespace odgs {

// Camera model fields of a ViewDev from the caller's view (false: invalid model or focal).
inline bool fill_camera(const odgs_view& w, ViewDev& d) {
    for (int i = 0; i < 9; ++i) d.R[i] = w.R_wc[i];
    for (int i = 0; i < 3; ++i) d.t[i] = w.t_wc[i];
    // camera centre -R^T t (double accumulation, then rounded)
    for (int j = 0; j < 3; ++j)
        d.cam[j] = (float)-((double)w.R_wc[j] * w.t_wc[0] + (double)w.R_wc[3 + j] * w.t_wc[1] +
                            (double)w.R_wc[6 + j] * w.t_wc[2]);
    d.model = w.model;
    if (w.model == 0) {
        d.fx = (float)((double)w.width / (2.0 * 3.14159265358979323846));
        d.fy = (float)((double)w.height / 3.14159265358979323846);
        d.cx = d.cy = 0.f;
        return true;
    }
    if (w.model != 1) return false;
    const bool fin = std::isfinite(w.fx) && std::isfinite(w.fy) && std::isfinite(w.cx) && std::isfinite(w.cy);
    if (!fin || !(w.fx > 0.f) || !(w.fy > 0.f)) return false;
    d.fx = w.fx; d.fy = w.fy; d.cx = w.cx; d.cy = w.cy;
    return true;
}

struct ViewTable {
    ViewDev v[kMaxViews];
    int n_views;
    uint32_t n_items;
};

struct Geometry {
    int total_tiles = 0, total_pixels = 0, total_trig = 0, key_bits = 1;
    size_t n_items = 0;
};

// Argument checks shared by every entry point that takes these structs (api.cu): the settings
// with their defaults filled in, the Gaussian arrays (pointers, 16-byte alignment where the
// kernels load 16 bytes), and the views (sizes, finite poses, camera model) with the per-view
// device constants and the frame's tile / pixel totals. ODGS_ERR_INVALID_ARG on any violation.
odgs_status check_settings(const odgs_settings* s, odgs_settings* out);
odgs_status check_gaussians(const odgs_gaussians* g, const odgs_settings& st);
odgs_status build_geometry(const odgs_view* views, int n_views, const odgs_settings& s, int n, Geometry* g,
                           ViewTable* tab);

struct PreArgs {
    const float *means, *scales, *quats, *opacity, *sh;
    int n, n_views, sh_coeffs;
    const ViewDev* views;
    const float4* trig;
    Settings st;
    float4 *rec_a, *rec_b, *rec_c;
    uint4* rect;   // (ty0 | bands << 16, tiles, span of band 0, span of band 1); span = start | count << 16
    uint4* rect2;  // spans of bands 2..5 (items with more than 2 bands)
    uint32_t *dkey, *dval;
    uint32_t* dhist;  // [4][256] digit histograms of dkey (zeroed by k_setup), for the depth sort
    uint8_t* dbucket;  // per item its depth bucket (saturation.cu), or null
    uint32_t cut_base;  // depth_bucket's origin
    Header* hdr;
};

struct PreBwdArgs {
    const float *means, *scales, *quats, *opacity, *sh;
    int n, n_views, sh_coeffs;
    const ViewDev* views;
    float dilation;
    const float4* acc;
    float *g_means, *g_scales, *g_quats, *g_opacity, *g_sh;
    int accumulate;
    int raw;                         // gradients w.r.t. log-scales and opacity logits
    const uint4* rect;               // footprint words: tile count > 0 <=> visible in that view
    float *d_grad, *d_elev;          // densification statistics (all three or none)
    uint32_t* d_count;
};

struct BinArgs {
    const uint32_t* sorted_idx;
    const uint4* rect;
    const uint4* rect2;
    const float4 *rec_a, *rec_b;
    int tile_w, tile_h;
    const ViewDev* views;
    int n_per_view;
    uint32_t n_items;
    unsigned long long* block_sums;
    Header* hdr;
    unsigned long long capacity;
    uint32_t *keys, *vals;
    uint2* big;  // [n_items] queue of (depth-order position, offset) of items with more than 32 pairs
    int num_sms;
    uint32_t* key_hist;  // [passes][256] digit histograms of the emitted tile ids (zeroed here)
    int key_passes;
    // truncated lists (saturation.cu), or null: per tile the last depth bucket it keeps and per
    // bucket the prefix counts over the tiles of cut >= bucket; the depth-sorted keys (buckets);
    // per depth-order position the kept pairs | bucket << 26 (written by k_count_blocks)
    const uint8_t* cut;
    const uint32_t* G;
    const uint32_t* sorted_keys;
    uint2* ranges_zero;  // the tile ranges, cleared by the pair count (or null)
    uint32_t n_ranges;
    uint32_t base, total_tiles;
    uint32_t* kcount;
    // the pair counts, their scan and the kept-pair words of this depth order are in place from an
    // earlier binning of the same frame: emit only (a rebuild of the lists for the backward pass)
    bool emit_only;
};

struct EmitArgs {
    const uint32_t* sorted_idx;
    const uint4* rect;
    const uint4* rect2;
    const float4 *rec_a, *rec_b;
    const ViewDev* views;
    int n_per_view;
    uint32_t n_items;
    int tile_w, tile_h;
    const unsigned long long* block_offsets;
    unsigned long long capacity;
    uint32_t *keys, *vals;
    uint2* big;
    Header* hdr;
    uint32_t* key_hist;
    int key_passes;
    const uint32_t* kcount;  // by depth-order position, or null
    const uint8_t* cut;
};

struct SatArgs {
    const uint4* rect;
    const float4 *rec_a, *rec_b;
    const uint8_t* dbucket;  // depth bucket by item (the geometry kernel's)
    const ViewDev* views;
    int n_per_view;
    uint32_t n_items, total_tiles;
    int tile_w, tile_h;
    uint32_t* cover;   // [kCutBuckets][total_tiles] bucket sums, then [kCutBuckets][total_tiles + 1] prefixes
    uint8_t* cut;      // [total_tiles]
};
// Frames of more tiles keep their whole lists (the bucket tables take 128 bytes per tile).
constexpr uint32_t kCutMaxTiles = 1u << 19;
cudaError_t launch_saturation(const SatArgs& a, int num_sms, cudaStream_t st, int* launches);

struct FwdArgs {
    const ViewDev* views;
    int n_views, total_tiles, tile_w, tile_h, batch, ppt;
    uint32_t n_items;
    const uint2* ranges;
    const uint32_t* pair_vals;
    const float4 *rec_a, *rec_b, *rec_c;
    float* images[kMaxViews];
    float* user_T[kMaxViews];
    float* T_final;
    uint32_t* n_last;
    float bg[3];
    Header* hdr;
};

struct BwdArgs {
    const ViewDev* views;
    int n_views, total_tiles, tile_w, tile_h, batch, ppt;
    uint32_t n_items;
    const uint2* ranges;
    const uint32_t* pair_vals;
    const float4 *rec_a, *rec_b, *rec_c;
    const float* dL_dimages[kMaxViews];
    const float* T_final;
    const uint32_t* n_last;
    float bg[3];
    float4* acc;
    Header* hdr;
    int checked;  // flag non-finite dL/dimage values and take them as 0
};

cudaError_t launch_setup(const ViewTable& tab, ViewDev* views, float4* trig, Header* hdr, int total_trig,
                         uint32_t* dhist, cudaStream_t st);
cudaError_t launch_preprocess(const PreArgs& a, int sh_degree, cudaStream_t st);
cudaError_t launch_preprocess_bwd(const PreBwdArgs& a, int sh_degree, cudaStream_t st);

int radix_passes(int bits);
size_t radix_lookback_words(size_t max_items);
// Look-back reads a sort CTA makes before it gives up and sets kStTimeout (odgs_set_wait_limit).
constexpr uint32_t kDefaultWaitLimit = 1u << 22;
cudaError_t launch_radix_sort(uint32_t* k[2], uint32_t* v[2], const uint32_t* n_ptr, size_t max_items, int bits,
                              uint32_t* hist, uint32_t* tile_ctrs, uint32_t* lookback, uint32_t* status, int num_sms,
                              cudaStream_t st, int* result_buf, int* launches, bool hist_ready, uint32_t wait_limit,
                              int lb_regions = 1);  // look-back regions of radix_lookback_words each
// A sort whose four tile counters lie kCtrBytes before its look-back regions (one per pass) clears
// both with one memset.
constexpr size_t kCtrBytes = 256;

int scan_blocks_for(uint32_t n_items);
cudaError_t launch_binning(const BinArgs& a, cudaStream_t st, int* launches);
// zeroed: the ranges are already 0 (cleared by the pair count of the same binning)
cudaError_t launch_tile_ranges(const uint32_t* keys, const Header* hdr, uint2* ranges, int total_tiles,
                               size_t max_pairs, int num_sms, cudaStream_t st, int* launches, bool zeroed = false);

size_t render_fwd_smem(int batch);
size_t render_bwd_smem(int batch, int threads);
// Pixels per thread of a blend kernel: want if valid (0 if not), or for want = 0 `prefer` if it
// fits the tile, else the largest of 4, 2, 1 that does. The forward prefers 2, the backward 4.
int pixels_per_thread(int tile_w, int tile_h, int want, int prefer);
int render_fwd_occupancy(int tile_w, int tile_h, int batch, int ppt);
int render_bwd_occupancy(int tile_w, int tile_h, int batch, int ppt);
cudaError_t launch_render_fwd(const FwdArgs& a, int grid, cudaStream_t st);
cudaError_t launch_render_bwd(const BwdArgs& a, int grid, cudaStream_t st);

}  // namespace odgs
