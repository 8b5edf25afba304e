// Forward alpha blending (Sec. 3.1, Eq. 2-3) on ERP tiles (sm_103a).
//
// A persistent grid pulls (view, tile) work items from an atomic counter, so one launch renders
// any number of views of mixed resolution. For each tile the CTA (one thread per pixel) walks
// the tile's depth-ordered list in batches: the threads gather a batch of records with 16-byte
// loads, convert them to the tile's staged form (seam shift, base-2 conic, log2 opacity) in
// shared memory, then every pixel evaluates the batch from shared memory (broadcast reads).
// A pixel stops before the Gaussian that would take its transmittance below 1e-4; the tile
// stops when all its pixels have stopped (__syncthreads_count).
//
// Per pixel the result depends only on the pixel, the Gaussians' records and their global
// order, never on the tile shape or batch size: the offset to a Gaussian is formed from integer
// pixel indices, and list entries with alpha < 1/255 leave the state untouched.
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

template <int MAXT>
__global__ void __launch_bounds__(MAXT) k_render_fwd(FwdArgs a) {
    extern __shared__ float4 smem[];
    const int B = a.batch;
    float4* s_pos = smem;
    float4* s_con = smem + B;
    float4* s_col = smem + 2 * B;
    float* s_fc2 = reinterpret_cast<float*>(smem + 3 * B);
    __shared__ int s_item;

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tw = a.tile_w;
    const int lx = tid % tw, ly = tid / tw;
    uint32_t evals = 0u, blended = 0u;  // (pixel, entry) evaluations / blends by this thread

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(&a.hdr->work_fwd, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= a.total_tiles) break;
        int v = 0;
        while (v + 1 < a.n_views && a.views[v + 1].tile_base <= item) ++v;
        const ViewDev& V = a.views[v];
        const int lt = item - V.tile_base;
        const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
        const int x0 = tx * tw;
        const int x = x0 + lx, y = ty * a.tile_h + ly;
        const bool inside = y < V.H;
        const float fi = (float)x, fj = (float)y;
        const uint2 rg = a.ranges[item];
        const int n = (int)(rg.y - rg.x);

        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int last = 0, tested = inside ? n : 0;
        bool done = !inside;
        for (int b0 = 0; b0 < n; b0 += B) {
            const int cnt = min(B, n - b0);
            int split = 0;
            for (int j = tid; j < cnt; j += nthr) {
                const uint32_t idx = a.pair_vals[rg.x + b0 + j];
                float4 ra, rb, rc;
                gather_records(a.rec_a, a.rec_b, a.rec_c, idx, a.n_items, ra, rb, rc);
                Staged s = stage_entry(ra, rb, rc, x0, tw, V.W);
                s_pos[j] = s.pos;
                s_con[j] = s.con;
                s_col[j] = s.col;
                s_fc2[j] = s.fc2;
                split |= (s.col.w <= 1e30f);
            }
            const int any_split = __syncthreads_or(split);
            if (!done) {
                if (!any_split) {
                    for (int j = 0; j < cnt; ++j) {
                        const float4 P = s_pos[j];
                        float dx, dy;
                        pixel_offset(fi, fj, P.x, P, dx, dy);
                        const float p = gauss_exponent(s_con[j], dx, dy);
                        if (p < kLog2AlphaMin) continue;
                        const float alpha = fminf(kAlphaMax, exp2f(p));
                        const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
                        if (Tn < kTMin) { done = true; tested = b0 + j + 1; break; }
                        const float w = __fmul_rn(alpha, T);
                        const float4 c = s_col[j];
                        C0 = __fmaf_rn(c.x, w, C0);
                        C1 = __fmaf_rn(c.y, w, C1);
                        C2 = __fmaf_rn(c.z, w, C2);
                        T = Tn;
                        last = b0 + j + 1;
                        ++blended;
                    }
                } else {
                    for (int j = 0; j < cnt; ++j) {
                        const float4 P = s_pos[j];
                        const float4 c = s_col[j];
                        const float fc = (fi >= c.w) ? s_fc2[j] : P.x;
                        float dx, dy;
                        pixel_offset(fi, fj, fc, P, dx, dy);
                        const float p = gauss_exponent(s_con[j], dx, dy);
                        if (p < kLog2AlphaMin) continue;
                        const float alpha = fminf(kAlphaMax, exp2f(p));
                        const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
                        if (Tn < kTMin) { done = true; tested = b0 + j + 1; break; }
                        const float w = __fmul_rn(alpha, T);
                        C0 = __fmaf_rn(c.x, w, C0);
                        C1 = __fmaf_rn(c.y, w, C1);
                        C2 = __fmaf_rn(c.z, w, C2);
                        T = Tn;
                        last = b0 + j + 1;
                        ++blended;
                    }
                }
            }
            if (__syncthreads_count(!done) == 0) break;
        }
        if (inside) {
            const int HW = V.W * V.H;
            const int pix = y * V.W + x;
            float* img = a.images[v];
            img[pix] = __fmaf_rn(T, a.bg[0], C0);
            img[HW + pix] = __fmaf_rn(T, a.bg[1], C1);
            img[2 * HW + pix] = __fmaf_rn(T, a.bg[2], C2);
            a.T_final[V.pix_base + pix] = T;
            a.n_last[V.pix_base + pix] = (uint32_t)last;
            if (a.user_T[v]) a.user_T[v][pix] = T;
        }
        evals += (uint32_t)tested;
    }
    unsigned long long ev = evals;
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if ((tid & 31) == 0 && ev) atomicAdd(&a.hdr->evals_fwd, ev);
    unsigned long long bl = blended;
    for (int o = 16; o > 0; o >>= 1) bl += __shfl_xor_sync(0xffffffffu, bl, o);
    if ((tid & 31) == 0 && bl) atomicAdd(&a.hdr->blended, bl);
}

size_t render_fwd_smem(int batch) { return (size_t)batch * (3 * sizeof(float4) + sizeof(float)); }

template <int MAXT>
static cudaError_t launch_fwd_t(const FwdArgs& a, int grid, cudaStream_t st) {
    size_t sm = render_fwd_smem(a.batch);
    k_render_fwd<MAXT><<<grid, a.tile_w * a.tile_h, sm, st>>>(a);
    return cudaGetLastError();
}

int render_fwd_occupancy(int threads, int batch) {
    int nb = 0;
    size_t sm = render_fwd_smem(batch);
    cudaError_t e;
    if (threads <= 64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<64>, threads, sm);
    else if (threads <= 128) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<128>, threads, sm);
    else if (threads <= 256) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<256>, threads, sm);
    else if (threads <= 512) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<512>, threads, sm);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<1024>, threads, sm);
    return e == cudaSuccess ? max(nb, 1) : 1;
}

cudaError_t launch_render_fwd(const FwdArgs& a, int grid, cudaStream_t st) {
    const int threads = a.tile_w * a.tile_h;
    if (threads <= 64) return launch_fwd_t<64>(a, grid, st);
    if (threads <= 128) return launch_fwd_t<128>(a, grid, st);
    if (threads <= 256) return launch_fwd_t<256>(a, grid, st);
    if (threads <= 512) return launch_fwd_t<512>(a, grid, st);
    return launch_fwd_t<1024>(a, grid, st);
}

}  // namespace odgs
