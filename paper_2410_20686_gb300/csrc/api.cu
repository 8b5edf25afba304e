// C ABI of the ODGS ERP rasterizer: argument validation, workspace layout, launch sequences.
// The declarations and the contract of every entry point are in include/odgs.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "odgs.h"
#include "odgs_internal.h"

using namespace odgs;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t hdr, views, trig, rec_a, rec_b, rec_c, rect, rect2, dkey0, dkey1, dval0, dval1, block_sums, ranges, T_final,
        n_last, acc, sort_hist, sort_ctr, sort_lb, big, cover, cut, kcount, dbucket, total;
    bool truncate;  // the lists are truncated at saturated tiles (the tables below are present)
};

struct PairLayout {
    size_t keys0, keys1, vals0, vals1, hist, ctr, lb, total;
};


// Truncated lists unless the caller asks for the whole lists or the frame has too many tiles.
bool truncates(const odgs_settings& s, const Geometry& g) { return !s.full_lists && (uint32_t)g.total_tiles <= kCutMaxTiles; }

// Look-back regions of the two sorts: one per pass, so that one memset clears them (the depth
// sort's four passes; the tile sort's passes when the tile ids take at most 16 bits).
constexpr int kDepthLbRegions = 4;
constexpr int kPairLbRegions = 2;

Layout make_layout(size_t items, const Geometry& g, bool truncate) {
    Layout L{};
    L.truncate = truncate;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    L.hdr = take(sizeof(Header));
    L.views = take(sizeof(ViewDev) * kMaxViews);
    L.trig = take(sizeof(float4) * (size_t)g.total_trig);
    L.rec_a = take(sizeof(float4) * items);
    L.rec_b = take(sizeof(float4) * items);
    L.rec_c = take(sizeof(float4) * items);
    L.rect = take(sizeof(uint4) * items);
    L.rect2 = take(sizeof(uint4) * items);
    L.dkey0 = take(sizeof(uint32_t) * items);
    L.dkey1 = take(sizeof(uint32_t) * items);
    L.dval0 = take(sizeof(uint32_t) * items);
    L.dval1 = take(sizeof(uint32_t) * items);
    L.block_sums = take(sizeof(unsigned long long) * ((size_t)scan_blocks_for((uint32_t)items) + 1));
    L.ranges = take(sizeof(uint2) * (size_t)g.total_tiles);
    L.T_final = take(sizeof(float) * (size_t)g.total_pixels);
    L.n_last = take(sizeof(uint32_t) * (size_t)g.total_pixels);
    L.acc = take(3 * sizeof(float4) * items);
    L.sort_hist = take(sizeof(uint32_t) * 4 * 256);
    // the tile counters kCtrBytes before the look-back regions: one memset clears both
    L.sort_ctr = take(kCtrBytes + sizeof(uint32_t) * radix_lookback_words(items) * kDepthLbRegions);
    L.sort_lb = L.sort_ctr + kCtrBytes;
    L.big = take(sizeof(uint2) * items);
    const size_t tt = truncate ? (size_t)g.total_tiles : 0;
    L.cover = take(sizeof(uint32_t) * (size_t)kCutBuckets * (truncate ? tt + 1 : 0));
    L.cut = take(tt);
    L.kcount = take(truncate ? sizeof(uint32_t) * items : 0);
    L.dbucket = take(truncate ? items : 0);
    L.total = o;
    return L;
}

PairLayout make_pair_layout(size_t cap) {
    PairLayout P{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    P.keys0 = take(sizeof(uint32_t) * cap);
    P.keys1 = take(sizeof(uint32_t) * cap);
    P.vals0 = take(sizeof(uint32_t) * cap);
    P.vals1 = take(sizeof(uint32_t) * cap);
    P.hist = take(sizeof(uint32_t) * 4 * 256);
    P.ctr = take(kCtrBytes + sizeof(uint32_t) * radix_lookback_words(cap) * kPairLbRegions);
    P.lb = P.ctr + kCtrBytes;
    P.total = o;
    return P;
}

}  // namespace

odgs_status odgs::check_settings(const odgs_settings* s, odgs_settings* out) {
    if (!s) return ODGS_ERR_INVALID_ARG;
    odgs_settings t = *s;
    if (t.sh_degree < 0 || t.sh_degree > 3) return ODGS_ERR_INVALID_ARG;
    const int K = (t.sh_degree + 1) * (t.sh_degree + 1);
    if (t.sh_coeffs < K || t.sh_coeffs > 64) return ODGS_ERR_INVALID_ARG;
    if (t.tile_w == 0 && t.tile_h == 0) { t.tile_w = 16; t.tile_h = 16; }
    if (!(t.tile_w == 8 || t.tile_w == 16 || t.tile_w == 32)) return ODGS_ERR_INVALID_ARG;
    const int area = t.tile_w * t.tile_h;
    if (t.tile_h < 1 || area < 32 || area > 1024 || area % 32 != 0) return ODGS_ERR_INVALID_ARG;
    t.pixels_per_thread = pixels_per_thread(t.tile_w, t.tile_h, t.pixels_per_thread, 2);
    t.pixels_per_thread_bwd = pixels_per_thread(t.tile_w, t.tile_h, t.pixels_per_thread_bwd, 4);
    if (t.pixels_per_thread == 0 || t.pixels_per_thread_bwd == 0) return ODGS_ERR_INVALID_ARG;
    if (t.batch == 0) t.batch = 128;
    if (t.batch < 1 || t.batch > 256) return ODGS_ERR_INVALID_ARG;
    if (!std::isfinite(t.cov_dilation) || t.cov_dilation < 0.f) return ODGS_ERR_INVALID_ARG;
    if (!std::isfinite(t.r_near) || !(t.r_far > t.r_near) || t.r_near < 0.f) return ODGS_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(t.bg[c])) return ODGS_ERR_INVALID_ARG;
    if (t.raw_params != 0 && t.raw_params != 1) return ODGS_ERR_INVALID_ARG;
    if (t.checked != 0 && t.checked != 1) return ODGS_ERR_INVALID_ARG;
    if (t.full_lists != 0 && t.full_lists != 1) return ODGS_ERR_INVALID_ARG;
    *out = t;
    return ODGS_OK;
}

odgs_status odgs::build_geometry(const odgs_view* views, int n_views, const odgs_settings& s, int n, Geometry* g,
                                 ViewTable* tab) {
    if (!views || n_views < 1 || n_views > kMaxViews || n < 0) return ODGS_ERR_INVALID_ARG;
    long long tiles = 0, pixels = 0, trig = 0;
    for (int v = 0; v < n_views; ++v) {
        const odgs_view& w = views[v];
        if (w.width < s.tile_w || w.height < 1 || w.width > 16384 || w.height > 16384) return ODGS_ERR_INVALID_ARG;
        if (w.width % s.tile_w != 0) return ODGS_ERR_INVALID_ARG;
        for (int i = 0; i < 9; ++i)
            if (!std::isfinite(w.R_wc[i])) return ODGS_ERR_INVALID_ARG;
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(w.t_wc[i])) return ODGS_ERR_INVALID_ARG;
        const int tx = w.width / s.tile_w, ty = (w.height + s.tile_h - 1) / s.tile_h;
        ViewDev scratch_view{};
        ViewDev& d = tab ? tab->v[v] : scratch_view;
        memset(&d, 0, sizeof(d));
        if (!fill_camera(w, d)) return ODGS_ERR_INVALID_ARG;
        d.W = w.width; d.H = w.height; d.tiles_x = tx; d.tiles_y = ty;
        d.tile_base = (int)tiles; d.pix_base = (int)pixels;
        d.trig_u = (int)trig; d.trig_v = (int)(trig + w.width);
        tiles += (long long)tx * ty;
        pixels += (long long)w.width * w.height;
        trig += (long long)w.width + w.height;
    }
    const long long items = (long long)n * n_views;
    if (tiles >= (1ll << 30) || pixels >= (1ll << 31) || items >= (1ll << 31)) return ODGS_ERR_INVALID_ARG;
    g->total_tiles = (int)tiles;
    g->total_pixels = (int)pixels;
    g->total_trig = (int)trig;
    g->n_items = (size_t)items;
    int bits = 1;
    while ((1ll << bits) < tiles) ++bits;
    g->key_bits = bits;
    if (tab) {
        tab->n_views = n_views;
        tab->n_items = (uint32_t)items;
    }
    return ODGS_OK;
}

odgs_status odgs::check_gaussians(const odgs_gaussians* g, const odgs_settings& st) {
    if (!g || g->n < 0) return ODGS_ERR_INVALID_ARG;
    if (g->n == 0) return ODGS_OK;
    if (!g->means || !g->scales || !g->quats || !g->opacity || !g->sh) return ODGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(g->quats) % 16 != 0) return ODGS_ERR_INVALID_ARG;
    if ((st.sh_coeffs * 3) % 4 == 0 && reinterpret_cast<uintptr_t>(g->sh) % 16 != 0) return ODGS_ERR_INVALID_ARG;
    return ODGS_OK;
}

struct odgs_ctx {
    int device = 0, num_sms = 1;
    int n = 0, V = 0;
    odgs_settings s{};
    ViewTable tab{};
    odgs_view views[kMaxViews];
    Geometry geo{};
    Layout L{};
    odgs_gaussians g{};
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;
    uint8_t* pb = nullptr;
    size_t pb_cap = 0;
    PairLayout P{};
    uint32_t* sorted_vals = nullptr;
    int stage = 0;
    int launches = 0;
    int bwd_batch = 64;
    uint32_t wait_limit = kDefaultWaitLimit;
    int depth_buf = 0, pair_buf = 0;  // which buffer of each double-buffered sort holds its result
    // the cut per tile and the kept counts per item of the current preprocess are in the
    // workspace (they are computed from the depth keys by item, which the depth sort overwrites,
    // so a second odgs_bin_sort or a rebuild of the lists reuses them)
    bool cut_ready = false;
    // a second stream on which the binning computes the cuts while the depth sort runs (forked
    // from and joined back to the caller's stream by events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~odgs_ctx() {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
    }
};

extern "C" {

const char* odgs_status_string(odgs_status st) {
    switch (st) {
        case ODGS_OK: return "ok";
        case ODGS_ERR_INVALID_ARG: return "invalid argument";
        case ODGS_ERR_CAPACITY: return "pair capacity exceeded";
        case ODGS_ERR_CUDA: return "CUDA error";
        case ODGS_ERR_TIMEOUT: return "device wait timed out";
        case ODGS_ERR_NONFINITE: return "non-finite input";
        case ODGS_ERR_STATE: return "call out of order";
        case ODGS_ERR_WORKSPACE: return "workspace too small";
    }
    return "unknown status";
}

odgs_status odgs_create(odgs_ctx** out) {
    if (!out) return ODGS_ERR_INVALID_ARG;
    *out = nullptr;
    odgs_ctx* c = new (std::nothrow) odgs_ctx();
    if (!c) return ODGS_ERR_INVALID_ARG;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return ODGS_ERR_CUDA;
    }
    *out = c;
    return ODGS_OK;
}

void odgs_destroy(odgs_ctx* ctx) { delete ctx; }

odgs_status odgs_workspace_size(int n, const odgs_view* views, int n_views, const odgs_settings* s, size_t* bytes) {
    if (!bytes) return ODGS_ERR_INVALID_ARG;
    odgs_settings st;
    odgs_status r = check_settings(s, &st);
    if (r != ODGS_OK) return r;
    Geometry g;
    r = build_geometry(views, n_views, st, n, &g, nullptr);
    if (r != ODGS_OK) return r;
    *bytes = make_layout(g.n_items, g, truncates(st, g)).total;
    return ODGS_OK;
}

odgs_status odgs_pair_buffer_size(size_t cap, size_t* bytes) {
    if (!bytes || cap >= (1ull << 30)) return ODGS_ERR_INVALID_ARG;
    *bytes = make_pair_layout(cap).total;
    return ODGS_OK;
}

static odgs_status run_preprocess(odgs_ctx* c, cudaStream_t st) {
    uint8_t* w = c->ws;
    Header* hdr = reinterpret_cast<Header*>(w + c->L.hdr);
    ViewDev* vd = reinterpret_cast<ViewDev*>(w + c->L.views);
    float4* trig = reinterpret_cast<float4*>(w + c->L.trig);
    uint32_t* dhist = reinterpret_cast<uint32_t*>(w + c->L.sort_hist);
    if (launch_setup(c->tab, vd, trig, hdr, c->geo.total_trig, dhist, st) != cudaSuccess) return ODGS_ERR_CUDA;
    c->launches += 1;
    PreArgs a{};
    a.means = c->g.means; a.scales = c->g.scales; a.quats = c->g.quats; a.opacity = c->g.opacity; a.sh = c->g.sh;
    a.n = c->n; a.n_views = c->V; a.sh_coeffs = c->s.sh_coeffs;
    a.views = vd; a.trig = trig;
    a.st.sh_degree = c->s.sh_degree; a.st.sh_coeffs = c->s.sh_coeffs;
    a.st.tile_w = c->s.tile_w; a.st.tile_h = c->s.tile_h;
    a.st.dilation = c->s.cov_dilation; a.st.r_near = c->s.r_near; a.st.r_far = c->s.r_far;
    for (int i = 0; i < 3; ++i) a.st.bg[i] = c->s.bg[i];
    a.st.raw = c->s.raw_params;
    a.st.checked = c->s.checked;
    a.rec_a = reinterpret_cast<float4*>(w + c->L.rec_a);
    a.rec_b = reinterpret_cast<float4*>(w + c->L.rec_b);
    a.rec_c = reinterpret_cast<float4*>(w + c->L.rec_c);
    a.rect = reinterpret_cast<uint4*>(w + c->L.rect);
    a.rect2 = reinterpret_cast<uint4*>(w + c->L.rect2);
    a.dkey = reinterpret_cast<uint32_t*>(w + c->L.dkey0);
    a.dval = reinterpret_cast<uint32_t*>(w + c->L.dval0);
    a.dhist = dhist;
    if (c->L.truncate) {
        a.dbucket = w + c->L.dbucket;
        uint32_t rn;
        std::memcpy(&rn, &c->s.r_near, sizeof(rn));
        a.cut_base = rn >> kCutShift;
    }
    a.hdr = hdr;
    if (launch_preprocess(a, c->s.sh_degree, st) != cudaSuccess) return ODGS_ERR_CUDA;
    if (c->n > 0) c->launches += 2;
    return ODGS_OK;
}

odgs_status odgs_preprocess(odgs_ctx* c, const odgs_gaussians* g, const odgs_view* views, int n_views,
                            const odgs_settings* s, void* workspace, size_t ws_bytes, void* stream) {
    if (!c || !g) return ODGS_ERR_INVALID_ARG;
    odgs_settings st;
    odgs_status r = check_settings(s, &st);
    if (r != ODGS_OK) return r;
    r = check_gaussians(g, st);
    if (r != ODGS_OK) return r;
    ViewTable tab{};
    Geometry geo;
    r = build_geometry(views, n_views, st, g->n, &geo, &tab);
    if (r != ODGS_OK) return r;
    Layout L = make_layout(geo.n_items, geo, truncates(st, geo));
    if (!workspace) return ODGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0) return ODGS_ERR_INVALID_ARG;
    if (ws_bytes < L.total) return ODGS_ERR_WORKSPACE;
    c->s = st;
    c->tab = tab;
    for (int v = 0; v < n_views; ++v) c->views[v] = views[v];
    c->geo = geo;
    c->L = L;
    c->g = *g;
    c->n = g->n;
    c->V = n_views;
    c->ws = static_cast<uint8_t*>(workspace);
    c->ws_bytes = ws_bytes;
    c->stage = 0;
    c->launches = 0;
    c->cut_ready = false;
    c->bwd_batch = std::min(st.batch, 64);
    const int bwd_threads = st.tile_w * st.tile_h / st.pixels_per_thread_bwd;
    while (c->bwd_batch > 8 && render_bwd_smem(c->bwd_batch, bwd_threads) > 48 * 1024) c->bwd_batch /= 2;
    r = run_preprocess(c, static_cast<cudaStream_t>(stream));
    if (r != ODGS_OK) return r;
    c->stage = 1;
    return ODGS_OK;
}

odgs_status odgs_query_pairs(odgs_ctx* c, size_t* pairs, void* stream) {
    if (!c || !pairs) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 1) return ODGS_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    if (cudaMemcpyAsync(&h, c->ws + c->L.hdr, sizeof(Header), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ODGS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ODGS_ERR_CUDA;
    *pairs = (size_t)h.pairs;
    if (h.status & kStTimeout) return ODGS_ERR_TIMEOUT;
    if (h.status & kStCapacity) return ODGS_ERR_CAPACITY;
    if (h.status & kStNonfinite) return ODGS_ERR_NONFINITE;
    return ODGS_OK;
}

odgs_status odgs_get_status(odgs_ctx* c, uint32_t* bits, void* stream) {
    if (!c || !bits) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 1) return ODGS_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    if (cudaMemcpyAsync(&h, c->ws + c->L.hdr, sizeof(Header), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ODGS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ODGS_ERR_CUDA;
    *bits = h.status;
    return ODGS_OK;
}

// rebuild: the lists of the frame's own earlier binning are rebuilt in the pair buffer (which
// other frames may have used since); the depth order, the pair counts and their scan are still in
// the workspace, so only the emission, the tile sort and the ranges run again.
static odgs_status run_bin_sort(odgs_ctx* c, cudaStream_t st, bool rebuild = false) {
    uint8_t* w = c->ws;
    Header* hdr = reinterpret_cast<Header*>(w + c->L.hdr);
    bool joined = true;  // no side-stream work to wait for
    // 0. which tiles saturate, and from which depth on (before the depth sort reorders the keys)
    if (c->L.truncate && !c->cut_ready) {
        SatArgs sa{};
        sa.rect = reinterpret_cast<const uint4*>(w + c->L.rect);
        sa.rec_a = reinterpret_cast<const float4*>(w + c->L.rec_a);
        sa.rec_b = reinterpret_cast<const float4*>(w + c->L.rec_b);
        sa.dbucket = w + c->L.dbucket;
        sa.views = reinterpret_cast<const ViewDev*>(w + c->L.views);
        sa.n_per_view = c->n > 0 ? c->n : 1;
        sa.n_items = (uint32_t)c->geo.n_items;
        sa.total_tiles = (uint32_t)c->geo.total_tiles;
        sa.tile_w = c->s.tile_w;
        sa.tile_h = c->s.tile_h;
        sa.cover = reinterpret_cast<uint32_t*>(w + c->L.cover);
        sa.cut = w + c->L.cut;
        // on the side stream, beside the depth sort (they share no data; the depth sort's
        // passes fill only part of the GPU)
        if (!c->side && (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess))
            return ODGS_ERR_CUDA;
        if (cudaEventRecord(c->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(c->side, c->ev_fork, 0) != cudaSuccess)
            return ODGS_ERR_CUDA;
        if (launch_saturation(sa, c->num_sms, c->side, &c->launches) != cudaSuccess) return ODGS_ERR_CUDA;
        if (cudaEventRecord(c->ev_join, c->side) != cudaSuccess) return ODGS_ERR_CUDA;
        joined = false;
        c->cut_ready = true;
    }
    // 1. depth sort of all (view, Gaussian) items (digit histograms counted by the preprocess)
    uint32_t* dk[2] = {reinterpret_cast<uint32_t*>(w + c->L.dkey0), reinterpret_cast<uint32_t*>(w + c->L.dkey1)};
    uint32_t* dv[2] = {reinterpret_cast<uint32_t*>(w + c->L.dval0), reinterpret_cast<uint32_t*>(w + c->L.dval1)};
    int rb = c->depth_buf;
    if (!rebuild) {
        if (launch_radix_sort(dk, dv, &hdr->n_items, c->geo.n_items, 32, reinterpret_cast<uint32_t*>(w + c->L.sort_hist),
                              reinterpret_cast<uint32_t*>(w + c->L.sort_ctr), reinterpret_cast<uint32_t*>(w + c->L.sort_lb),
                              &hdr->status, c->num_sms, st, &rb, &c->launches, /*hist_ready=*/true,
                              c->wait_limit, kDepthLbRegions) != cudaSuccess)
            return ODGS_ERR_CUDA;
        c->depth_buf = rb;
    }
    // 2. emit (tile, item) pairs in depth order
    uint8_t* p = c->pb;
    uint32_t* pk[2] = {reinterpret_cast<uint32_t*>(p + c->P.keys0), reinterpret_cast<uint32_t*>(p + c->P.keys1)};
    uint32_t* pv[2] = {reinterpret_cast<uint32_t*>(p + c->P.vals0), reinterpret_cast<uint32_t*>(p + c->P.vals1)};
    BinArgs b{};
    b.sorted_idx = dv[rb];
    b.rect = reinterpret_cast<const uint4*>(w + c->L.rect);
    b.rect2 = reinterpret_cast<const uint4*>(w + c->L.rect2);
    b.rec_a = reinterpret_cast<const float4*>(w + c->L.rec_a);
    b.rec_b = reinterpret_cast<const float4*>(w + c->L.rec_b);
    b.tile_w = c->s.tile_w;
    b.tile_h = c->s.tile_h;
    b.views = reinterpret_cast<const ViewDev*>(w + c->L.views);
    b.n_per_view = c->n > 0 ? c->n : 1;
    b.n_items = (uint32_t)c->geo.n_items;
    b.block_sums = reinterpret_cast<unsigned long long*>(w + c->L.block_sums);
    b.hdr = hdr;
    b.capacity = c->pb_cap;
    b.keys = pk[0];
    b.vals = pv[0];
    b.big = reinterpret_cast<uint2*>(w + c->L.big);
    b.num_sms = c->num_sms;
    b.key_hist = reinterpret_cast<uint32_t*>(p + c->P.hist);
    b.key_passes = radix_passes(c->geo.key_bits);
    if (c->L.truncate && c->geo.n_items > 0) {
        b.cut = w + c->L.cut;
        b.G = reinterpret_cast<const uint32_t*>(w + c->L.cover);
        b.sorted_keys = dk[rb];
        uint32_t rn;
        std::memcpy(&rn, &c->s.r_near, sizeof(rn));
        b.base = rn >> kCutShift;
        b.total_tiles = (uint32_t)c->geo.total_tiles;
        b.kcount = reinterpret_cast<uint32_t*>(w + c->L.kcount);
    }
    b.emit_only = rebuild;
    if (!rebuild && c->geo.n_items > 0) {  // the pair count clears the ranges
        b.ranges_zero = reinterpret_cast<uint2*>(w + c->L.ranges);
        b.n_ranges = (uint32_t)c->geo.total_tiles;
    }
    if (!joined && cudaStreamWaitEvent(st, c->ev_join, 0) != cudaSuccess) return ODGS_ERR_CUDA;
    if (launch_binning(b, st, &c->launches) != cudaSuccess) return ODGS_ERR_CUDA;
    // 3. stable sort of the pairs by tile id
    int rp = 0;
    if (launch_radix_sort(pk, pv, &hdr->n_pairs_sort, c->pb_cap, c->geo.key_bits, reinterpret_cast<uint32_t*>(p + c->P.hist),
                          reinterpret_cast<uint32_t*>(p + c->P.ctr), reinterpret_cast<uint32_t*>(p + c->P.lb),
                          &hdr->status, c->num_sms, st, &rp, &c->launches, /*hist_ready=*/true,
                          c->wait_limit, kPairLbRegions) != cudaSuccess)
        return ODGS_ERR_CUDA;
    c->sorted_vals = pv[rp];
    c->pair_buf = rp;
    // 4. per-tile ranges
    if (launch_tile_ranges(pk[rp], hdr, reinterpret_cast<uint2*>(w + c->L.ranges), c->geo.total_tiles, c->pb_cap,
                           c->num_sms, st, &c->launches, /*zeroed=*/b.ranges_zero != nullptr) != cudaSuccess)
        return ODGS_ERR_CUDA;
    return ODGS_OK;
}

odgs_status odgs_bin_sort(odgs_ctx* c, void* pair_buffer, size_t cap, void* stream) {
    if (!c) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 1) return ODGS_ERR_STATE;
    if (cap >= (1ull << 30)) return ODGS_ERR_INVALID_ARG;
    if (cap > 0 && !pair_buffer) return ODGS_ERR_INVALID_ARG;
    if (pair_buffer && reinterpret_cast<uintptr_t>(pair_buffer) % kAlign != 0) return ODGS_ERR_INVALID_ARG;
    c->pb = static_cast<uint8_t*>(pair_buffer);
    c->pb_cap = cap;
    c->P = make_pair_layout(cap);
    odgs_status r = run_bin_sort(c, static_cast<cudaStream_t>(stream));
    if (r != ODGS_OK) return r;
    c->stage = 2;
    return ODGS_OK;
}

static int persistent_grid(odgs_ctx* c, int per_sm) {
    long long g = (long long)c->num_sms * per_sm;
    if (g > c->geo.total_tiles) g = c->geo.total_tiles;
    return (int)(g < 1 ? 1 : g);
}

odgs_status odgs_render_fwd(odgs_ctx* c, float* const* images, float* const* final_T, void* stream) {
    if (!c || !images) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 2) return ODGS_ERR_STATE;
    for (int v = 0; v < c->V; ++v)
        if (!images[v]) return ODGS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* w = c->ws;
    Header* hdr = reinterpret_cast<Header*>(w + c->L.hdr);
    FwdArgs a{};
    a.views = reinterpret_cast<const ViewDev*>(w + c->L.views);
    a.n_views = c->V; a.total_tiles = c->geo.total_tiles;
    a.tile_w = c->s.tile_w; a.tile_h = c->s.tile_h; a.batch = c->s.batch;
    a.ppt = c->s.pixels_per_thread;
    a.n_items = (uint32_t)c->geo.n_items;
    a.ranges = reinterpret_cast<const uint2*>(w + c->L.ranges);
    a.pair_vals = c->sorted_vals;
    a.rec_a = reinterpret_cast<const float4*>(w + c->L.rec_a);
    a.rec_b = reinterpret_cast<const float4*>(w + c->L.rec_b);
    a.rec_c = reinterpret_cast<const float4*>(w + c->L.rec_c);
    for (int v = 0; v < c->V; ++v) {
        a.images[v] = images[v];
        a.user_T[v] = final_T ? final_T[v] : nullptr;
    }
    a.T_final = reinterpret_cast<float*>(w + c->L.T_final);
    a.n_last = reinterpret_cast<uint32_t*>(w + c->L.n_last);
    for (int i = 0; i < 3; ++i) a.bg[i] = c->s.bg[i];
    a.hdr = hdr;
    // the work counter and the forward counters: one memset
    if (cudaMemsetAsync(&hdr->evals_fwd, 0, reinterpret_cast<uint8_t*>(&hdr->pad1 + 1) - reinterpret_cast<uint8_t*>(&hdr->evals_fwd),
                        st) != cudaSuccess)
        return ODGS_ERR_CUDA;
    const int grid = persistent_grid(c, render_fwd_occupancy(c->s.tile_w, c->s.tile_h, a.batch, a.ppt));
    if (launch_render_fwd(a, grid, st) != cudaSuccess) return ODGS_ERR_CUDA;
    c->launches += 1;
    c->stage = 3;
    return ODGS_OK;
}

odgs_status odgs_render_bwd(odgs_ctx* c, const float* const* dL, void* stream) {
    if (!c || !dL) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 3) return ODGS_ERR_STATE;
    for (int v = 0; v < c->V; ++v)
        if (!dL[v]) return ODGS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (c->s.recompute_lists) {
        // the tile lists were not kept (the pair buffer may have served other frames since
        // odgs_render_fwd): rebuild them from the depth order, the pair counts and the per-item
        // records, which the workspace still holds (emission, tile sort and ranges only). The
        // binning is deterministic, so the lists are identical to the forward's.
        odgs_status r = run_bin_sort(c, st, /*rebuild=*/true);
        if (r != ODGS_OK) return r;
    }
    uint8_t* w = c->ws;
    Header* hdr = reinterpret_cast<Header*>(w + c->L.hdr);
    float4* acc = reinterpret_cast<float4*>(w + c->L.acc);
    if (cudaMemsetAsync(acc, 0, 3 * sizeof(float4) * c->geo.n_items, st) != cudaSuccess) return ODGS_ERR_CUDA;
    // the work counter and the evaluation counter: one memset
    if (cudaMemsetAsync(&hdr->evals_bwd, 0, reinterpret_cast<uint8_t*>(&hdr->pad0 + 1) - reinterpret_cast<uint8_t*>(&hdr->evals_bwd),
                        st) != cudaSuccess)
        return ODGS_ERR_CUDA;
    BwdArgs a{};
    a.views = reinterpret_cast<const ViewDev*>(w + c->L.views);
    a.n_views = c->V; a.total_tiles = c->geo.total_tiles;
    a.tile_w = c->s.tile_w; a.tile_h = c->s.tile_h; a.batch = c->bwd_batch;
    a.ppt = c->s.pixels_per_thread_bwd;
    a.n_items = (uint32_t)c->geo.n_items;
    a.ranges = reinterpret_cast<const uint2*>(w + c->L.ranges);
    a.pair_vals = c->sorted_vals;
    a.rec_a = reinterpret_cast<const float4*>(w + c->L.rec_a);
    a.rec_b = reinterpret_cast<const float4*>(w + c->L.rec_b);
    a.rec_c = reinterpret_cast<const float4*>(w + c->L.rec_c);
    for (int v = 0; v < c->V; ++v) a.dL_dimages[v] = dL[v];
    a.T_final = reinterpret_cast<const float*>(w + c->L.T_final);
    a.n_last = reinterpret_cast<const uint32_t*>(w + c->L.n_last);
    for (int i = 0; i < 3; ++i) a.bg[i] = c->s.bg[i];
    a.acc = acc;
    a.hdr = hdr;
    a.checked = c->s.checked;
    const int grid = persistent_grid(c, render_bwd_occupancy(c->s.tile_w, c->s.tile_h, a.batch, a.ppt));
    if (launch_render_bwd(a, grid, st) != cudaSuccess) return ODGS_ERR_CUDA;
    c->launches += 1;
    c->stage = 4;
    return ODGS_OK;
}

odgs_status odgs_preprocess_bwd(odgs_ctx* c, const odgs_grads* grads, void* stream) {
    if (!c || !grads) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 4) return ODGS_ERR_STATE;
    if (c->n > 0 && (!grads->means || !grads->scales || !grads->quats || !grads->opacity || !grads->sh))
        return ODGS_ERR_INVALID_ARG;
    if (c->n > 0 && reinterpret_cast<uintptr_t>(grads->quats) % 16 != 0) return ODGS_ERR_INVALID_ARG;
    if (c->n > 0 && (c->s.sh_coeffs * 3) % 4 == 0 && reinterpret_cast<uintptr_t>(grads->sh) % 16 != 0)
        return ODGS_ERR_INVALID_ARG;
    const int dens = (grads->densify_grad != nullptr) + (grads->densify_elev != nullptr) +
                     (grads->densify_count != nullptr);
    if (dens != 0 && dens != 3) return ODGS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* w = c->ws;
    PreBwdArgs b{};
    b.rect = reinterpret_cast<const uint4*>(w + c->L.rect);
    if (dens == 3) {
        b.d_grad = grads->densify_grad;
        b.d_elev = grads->densify_elev;
        b.d_count = grads->densify_count;
    }
    b.means = c->g.means; b.scales = c->g.scales; b.quats = c->g.quats; b.opacity = c->g.opacity; b.sh = c->g.sh;
    b.n = c->n; b.n_views = c->V; b.sh_coeffs = c->s.sh_coeffs;
    b.views = reinterpret_cast<const ViewDev*>(w + c->L.views);
    b.dilation = c->s.cov_dilation;
    b.acc = reinterpret_cast<const float4*>(w + c->L.acc);
    b.g_means = grads->means; b.g_scales = grads->scales; b.g_quats = grads->quats;
    b.g_opacity = grads->opacity; b.g_sh = grads->sh;
    b.accumulate = c->s.grad_accumulate;
    b.raw = c->s.raw_params;
    if (launch_preprocess_bwd(b, c->s.sh_degree, st) != cudaSuccess) return ODGS_ERR_CUDA;
    if (c->n > 0) c->launches += 1;
    return ODGS_OK;
}

odgs_status odgs_frame_stats(odgs_ctx* c, odgs_stats* out, void* stream) {
    if (!c || !out) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 1) return ODGS_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    if (cudaMemcpyAsync(&h, c->ws + c->L.hdr, sizeof(Header), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ODGS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ODGS_ERR_CUDA;
    out->pairs = h.pairs;
    out->pairs_sorted = h.pairs_emitted;
    out->evals_fwd = h.evals_fwd;
    out->evals_bwd = h.evals_bwd;
    out->blended = h.blended;
    out->entries_tile = h.entries_tile;
    out->visible = h.visible;
    out->status = h.status;
    return ODGS_OK;
}

int odgs_last_launch_count(const odgs_ctx* c) { return c ? c->launches : 0; }

odgs_status odgs_set_wait_limit(odgs_ctx* c, uint32_t reads) {
    if (!c) return ODGS_ERR_INVALID_ARG;
    c->wait_limit = reads;
    return ODGS_OK;
}

odgs_status odgs_debug_screen_grads(odgs_ctx* c, float* out, size_t n_items, void* stream) {
    if (!c || !out) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 4) return ODGS_ERR_STATE;
    if (n_items != c->geo.n_items) return ODGS_ERR_INVALID_ARG;
    if (n_items == 0) return ODGS_OK;
    if (cudaMemcpyAsync(out, c->ws + c->L.acc, 3 * sizeof(float4) * n_items, cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return ODGS_ERR_CUDA;
    return ODGS_OK;
}

odgs_status odgs_debug_lists(odgs_ctx* c, uint32_t* depth_keys, uint32_t* depth_items, size_t n_items,
                             uint32_t* pair_tiles, uint32_t* pair_items, size_t n_pairs, uint32_t* ranges,
                             size_t n_tiles, void* stream) {
    if (!c) return ODGS_ERR_INVALID_ARG;
    if (c->stage < 2) return ODGS_ERR_STATE;
    if ((depth_keys || depth_items) && n_items != c->geo.n_items) return ODGS_ERR_INVALID_ARG;
    if ((pair_tiles || pair_items) && n_pairs > c->pb_cap) return ODGS_ERR_INVALID_ARG;
    if (ranges && n_tiles != (size_t)c->geo.total_tiles) return ODGS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint8_t* w = c->ws;
    const uint8_t* p = c->pb;
    const size_t dk = c->depth_buf ? c->L.dkey1 : c->L.dkey0, dv = c->depth_buf ? c->L.dval1 : c->L.dval0;
    const size_t pk = c->pair_buf ? c->P.keys1 : c->P.keys0, pv = c->pair_buf ? c->P.vals1 : c->P.vals0;
    struct Copy {
        void* dst;
        const void* src;
        size_t bytes;
    } copies[5] = {{depth_keys, w + dk, 4 * n_items},
                   {depth_items, w + dv, 4 * n_items},
                   {pair_tiles, p ? p + pk : nullptr, 4 * n_pairs},
                   {pair_items, p ? p + pv : nullptr, 4 * n_pairs},
                   {ranges, w + c->L.ranges, 8 * n_tiles}};
    for (const Copy& k : copies) {
        if (!k.dst || k.bytes == 0) continue;
        if (!k.src) return ODGS_ERR_STATE;
        if (cudaMemcpyAsync(k.dst, k.src, k.bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return ODGS_ERR_CUDA;
    }
    return ODGS_OK;
}

}  // extern "C"
