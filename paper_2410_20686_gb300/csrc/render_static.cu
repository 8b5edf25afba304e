// odgs_render_fwd_static: the single-view forward render for callers that cannot allocate
// device memory. Some callers cannot call cudaMalloc: code running inside a host application's
// frame callback or plugin that owns a fixed device-memory budget (an allocation there can fail
// or is not allowed), and real-time loops in which cudaMalloc / cudaFree would synchronize the
// device and stall the frame. This entry point takes only the inputs and the outputs; every
// intermediate buffer (per-Gaussian records, depth and tile sorts, tile ranges, per-pixel state)
// is carved from one file-scope device array that each GPU holds from the moment the library is
// loaded until the process exits.
//
// It runs the same kernels as odgs_preprocess + odgs_bin_sort + odgs_render_fwd, so its image is
// the same as that path's. Limits: n <= kStaticMaxGaussians, one view of at most
// kStaticMaxPixels pixels, and as many (tile, Gaussian) pairs as fit in the rest of the array.
// Calls share the array: two calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on it and give wrong images. Every call resets
// the parts that must start at zero (header counters, sort histograms and look-back words, tile
// ranges) before use; everything else is fully written before it is read.
#include <mutex>

#include "odgs.h"
#include "odgs_internal.h"

using namespace odgs;

namespace {

constexpr size_t kStaticBytes = 32ull << 20;  // 32 MiB per GPU
constexpr int kStaticMaxGaussians = 32768;
constexpr long long kStaticMaxPixels = 524288;  // e.g. 1024 x 512
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch per device. In host code the symbol name is only a
// host-side stand-in, so the address is fetched once per device, with that device current.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

odgs_status scratch_for_current_device(uint8_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ODGS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ODGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return ODGS_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<uint8_t*>(g_scratch_addr[dev]);
    return ODGS_OK;
}

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" odgs_status odgs_render_fwd_static(const odgs_gaussians* g, const odgs_view* view,
                                              const odgs_settings* s, float* image, float* final_T,
                                              uint32_t* status_out, void* stream) {
    // ---- arguments (nothing is launched when one is rejected): the checks of the workspace
    // entry points, then this entry point's own size limits
    if (!view || !image || !status_out) return ODGS_ERR_INVALID_ARG;
    odgs_settings st;
    odgs_status r = check_settings(s, &st);
    if (r != ODGS_OK) return r;
    r = check_gaussians(g, st);
    if (r != ODGS_OK) return r;
    if (g->n > kStaticMaxGaussians) return ODGS_ERR_INVALID_ARG;
    if ((long long)view->width * view->height > kStaticMaxPixels) return ODGS_ERR_INVALID_ARG;
    ViewTable tab{};
    Geometry geo;
    r = build_geometry(view, 1, st, g->n, &geo, &tab);
    if (r != ODGS_OK) return r;
    const int W = view->width, H = view->height;

    uint8_t* base = nullptr;
    r = scratch_for_current_device(&base);
    if (r != ODGS_OK) return r;
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    int num_sms = 1, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ODGS_ERR_CUDA;
    const int tiles = geo.total_tiles;
    const int key_bits = geo.key_bits;
    const size_t n = (size_t)g->n, pixels = (size_t)W * H;

    // ---- carve the static array
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = up256(o + bytes);
        return base + at;
    };
    Header* hdr = reinterpret_cast<Header*>(take(sizeof(Header)));
    ViewDev* vd = reinterpret_cast<ViewDev*>(take(sizeof(ViewDev)));
    float4* trig = reinterpret_cast<float4*>(take(sizeof(float4) * (size_t)(W + H)));
    float4* rec_a = reinterpret_cast<float4*>(take(sizeof(float4) * n));
    float4* rec_b = reinterpret_cast<float4*>(take(sizeof(float4) * n));
    float4* rec_c = reinterpret_cast<float4*>(take(sizeof(float4) * n));
    uint4* rect = reinterpret_cast<uint4*>(take(sizeof(uint4) * n));
    uint4* rect2 = reinterpret_cast<uint4*>(take(sizeof(uint4) * n));
    uint32_t* dk[2] = {reinterpret_cast<uint32_t*>(take(4 * n)), reinterpret_cast<uint32_t*>(take(4 * n))};
    uint32_t* dv[2] = {reinterpret_cast<uint32_t*>(take(4 * n)), reinterpret_cast<uint32_t*>(take(4 * n))};
    unsigned long long* block_sums =
        reinterpret_cast<unsigned long long*>(take(8 * ((size_t)scan_blocks_for((uint32_t)n) + 1)));
    uint2* ranges = reinterpret_cast<uint2*>(take(sizeof(uint2) * (size_t)tiles));
    float* T_final = reinterpret_cast<float*>(take(4 * pixels));
    uint32_t* n_last = reinterpret_cast<uint32_t*>(take(4 * pixels));
    uint32_t* d_hist = reinterpret_cast<uint32_t*>(take(4 * 4 * 256));
    uint32_t* d_ctr = reinterpret_cast<uint32_t*>(take(4 * 4));
    uint32_t* d_lb = reinterpret_cast<uint32_t*>(take(4 * radix_lookback_words(n)));
    uint32_t* p_hist = reinterpret_cast<uint32_t*>(take(4 * 4 * 256));
    uint32_t* p_ctr = reinterpret_cast<uint32_t*>(take(4 * 4));
    uint2* big = reinterpret_cast<uint2*>(take(sizeof(uint2) * n));
    if (o >= kStaticBytes) return ODGS_ERR_WORKSPACE;
    // the rest holds the pairs: two key and two value buffers plus the sort look-back words
    const size_t rem = kStaticBytes - o;
    auto pair_bytes = [](size_t c) { return 4 * up256(4 * c) + up256(4 * radix_lookback_words(c)); };
    size_t cap = rem / 17;  // at least 16.25 bytes per pair
    while (cap > 0 && pair_bytes(cap) > rem) cap -= (cap < 4096 ? cap : 4096);
    uint32_t* pk[2] = {reinterpret_cast<uint32_t*>(take(4 * cap)), reinterpret_cast<uint32_t*>(take(4 * cap))};
    uint32_t* pv[2] = {reinterpret_cast<uint32_t*>(take(4 * cap)), reinterpret_cast<uint32_t*>(take(4 * cap))};
    uint32_t* p_lb = reinterpret_cast<uint32_t*>(take(4 * radix_lookback_words(cap)));
    if (o > kStaticBytes) return ODGS_ERR_WORKSPACE;

    // ---- the forward path (same kernels as the workspace entry points)
    int launches = 0;
    if (launch_setup(tab, vd, trig, hdr, geo.total_trig, d_hist, strm) != cudaSuccess) return ODGS_ERR_CUDA;
    PreArgs a{};
    a.means = g->means; a.scales = g->scales; a.quats = g->quats; a.opacity = g->opacity; a.sh = g->sh;
    a.n = g->n; a.n_views = 1; a.sh_coeffs = st.sh_coeffs;
    a.views = vd; a.trig = trig;
    a.st.sh_degree = st.sh_degree; a.st.sh_coeffs = st.sh_coeffs;
    a.st.tile_w = st.tile_w; a.st.tile_h = st.tile_h;
    a.st.dilation = st.cov_dilation; a.st.r_near = st.r_near; a.st.r_far = st.r_far;
    for (int i = 0; i < 3; ++i) a.st.bg[i] = st.bg[i];
    a.st.raw = st.raw_params;
    a.st.checked = st.checked;
    a.rec_a = rec_a; a.rec_b = rec_b; a.rec_c = rec_c; a.rect = rect; a.rect2 = rect2; a.dkey = dk[0]; a.dval = dv[0];
    a.dhist = d_hist;
    a.hdr = hdr;
    if (launch_preprocess(a, st.sh_degree, strm) != cudaSuccess) return ODGS_ERR_CUDA;
    int rb = 0;
    if (launch_radix_sort(dk, dv, &hdr->n_items, n, 32, d_hist, d_ctr, d_lb, &hdr->status, num_sms, strm, &rb,
                          &launches, /*hist_ready=*/true, kDefaultWaitLimit) != cudaSuccess)
        return ODGS_ERR_CUDA;
    BinArgs b{};
    b.sorted_idx = dv[rb]; b.rect = rect; b.rect2 = rect2; b.views = vd; b.n_per_view = g->n > 0 ? g->n : 1;
    b.rec_a = rec_a; b.rec_b = rec_b; b.tile_w = st.tile_w; b.tile_h = st.tile_h;
    b.n_items = (uint32_t)n; b.block_sums = block_sums; b.hdr = hdr; b.capacity = cap;
    b.keys = pk[0]; b.vals = pv[0];
    b.big = big; b.num_sms = num_sms;
    b.key_hist = p_hist; b.key_passes = radix_passes(key_bits);
    if (launch_binning(b, strm, &launches) != cudaSuccess) return ODGS_ERR_CUDA;
    int rp = 0;
    if (launch_radix_sort(pk, pv, &hdr->n_pairs_sort, cap, key_bits, p_hist, p_ctr, p_lb, &hdr->status, num_sms,
                          strm, &rp, &launches, /*hist_ready=*/true, kDefaultWaitLimit) != cudaSuccess)
        return ODGS_ERR_CUDA;
    if (launch_tile_ranges(pk[rp], hdr, ranges, tiles, cap, num_sms, strm, &launches) != cudaSuccess)
        return ODGS_ERR_CUDA;
    FwdArgs f{};
    f.views = vd; f.n_views = 1; f.total_tiles = tiles; f.tile_w = st.tile_w; f.tile_h = st.tile_h;
    f.batch = st.batch; f.ppt = st.pixels_per_thread; f.n_items = (uint32_t)n; f.ranges = ranges; f.pair_vals = pv[rp];
    f.rec_a = rec_a; f.rec_b = rec_b; f.rec_c = rec_c;
    f.images[0] = image; f.user_T[0] = final_T;
    f.T_final = T_final; f.n_last = n_last;
    for (int i = 0; i < 3; ++i) f.bg[i] = st.bg[i];
    f.hdr = hdr;
    // the work counter and the evaluation counters were zeroed by k_setup in this call
    const int per_sm = render_fwd_occupancy(st.tile_w, st.tile_h, st.batch, st.pixels_per_thread);
    long long grid = (long long)num_sms * per_sm;
    if (grid > tiles) grid = tiles;
    if (launch_render_fwd(f, (int)(grid < 1 ? 1 : grid), strm) != cudaSuccess) return ODGS_ERR_CUDA;
    // device status bits (ODGS_DEV_*) for the caller, without a host synchronization
    if (cudaMemcpyAsync(status_out, &hdr->status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, strm) != cudaSuccess)
        return ODGS_ERR_CUDA;
    return ODGS_OK;
}
