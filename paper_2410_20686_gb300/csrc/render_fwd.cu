// Forward alpha blending (Sec. 3.1, Eq. 2-3) on ERP tiles (sm_103a).
//
// A persistent grid pulls (view, tile) work items from an atomic counter, so one launch renders
// any number of views of mixed resolution. For each tile the CTA walks the tile's depth-ordered
// list in batches: the threads gather a batch of records with 16-byte loads, convert them to the
// tile's staged form (seam shift, base-2 slice-form conic, log2 opacity) in shared memory, then
// evaluate the batch from shared memory (broadcast reads).
//
// Each thread owns PPT pixels of one row, tile_w / PPT columns apart. The row-constant part of
// Eq. 2's quadratic form (the slice centre du + beta dy and gamma dy^2 + log2 o) and the
// shared-memory loads are paid once per thread and entry, not once per pixel; per pixel the
// exponent is (a t) t + row term with t the offset from the slice centre. The kernel is bound by
// instruction issue, so this is where its time goes.
// A pixel stops before the Gaussian that would take its transmittance below 1e-4; a thread stops
// when its pixels have; the tile stops when all threads have (__syncthreads_count).
//
// Per pixel the result depends only on the pixel, the Gaussians' records and their global
// order, never on the tile shape, the batch size or PPT: the offset to a Gaussian is formed from
// integer pixel indices, every pixel evaluates the same fixed sequence of round-to-nearest
// operations, and list entries with alpha < 1/255 leave the state untouched.
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

template <int PPT>
__global__ void __launch_bounds__(256) k_render_fwd(FwdArgs a) {
    extern __shared__ float4 smem[];
    const int B = a.batch;
    float4* s_pos = smem;
    float4* s_con = smem + B;
    float4* s_col = smem + 2 * B;
    float* s_fc2 = reinterpret_cast<float*>(smem + 3 * B);
    __shared__ int s_item;
    __shared__ uint32_t s_etile;  // entries the current tile processed until its pixels stopped

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tw = a.tile_w;
    const int tpr = tw / PPT;  // threads per pixel row
    // a thread's PPT pixels are tpr columns apart (interleaved), so a footprint a few pixels wide
    // falls in one of each lane's pixel slots rather than in several
    const int lx0 = tid % tpr, ly = tid / tpr;
    uint32_t evals = 0u, blended = 0u;  // (pixel, entry) evaluations / blends by this thread
    unsigned long long etile = 0ull;    // thread 0: sum of s_etile over this CTA's tiles
    if (tid == 0) s_etile = 0u;

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            etile += s_etile;
            s_etile = 0u;
            s_item = (int)atomicAdd(&a.hdr->work_fwd, 1u);
        }
        __syncthreads();
        const int item = s_item;
        if (item >= a.total_tiles) break;
        int v = 0;
        while (v + 1 < a.n_views && a.views[v + 1].tile_base <= item) ++v;
        const ViewDev& V = a.views[v];
        const int lt = item - V.tile_base;
        const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
        const int x0 = tx * tw;
        const int xp = x0 + lx0, y = ty * a.tile_h + ly;
        const bool inside = y < V.H;
        const float fj = (float)y;
        float fik[PPT];  // column coordinates of the thread's pixels
#pragma unroll
        for (int k = 0; k < PPT; ++k) fik[k] = (float)(xp + k * tpr);
        const uint2 rg = a.ranges[item];
        const int n = (int)(rg.y - rg.x);

        float T[PPT], C0[PPT], C1[PPT], C2[PPT];
        int last[PPT], tested[PPT];
        bool done[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            T[k] = 1.f; C0[k] = C1[k] = C2[k] = 0.f;
            last[k] = 0; tested[k] = inside ? n : 0; done[k] = !inside;
        }
        int alive = inside ? PPT : 0;
        for (int b0 = 0; b0 < n; b0 += B) {
            const int cnt = min(B, n - b0);
            int split = 0;
            for (int j = tid; j < cnt; j += nthr) {
                const uint32_t idx = a.pair_vals[rg.x + b0 + j];
                float4 ra, rb, rc;
                gather_records(a.rec_a, a.rec_b, a.rec_c, idx, a.n_items, ra, rb, rc);
                Staged s = stage_entry(ra, rb, rc, x0, tw, V.W, V.model == 0);
                s_pos[j] = s.pos;
                s_con[j] = s.con;
                s_col[j] = s.col;
                s_fc2[j] = s.fc2;
                split |= (s.col.w <= 1e30f);
            }
            const int any_split = __syncthreads_or(split);
#pragma unroll 4  // measured: 0.408 -> 0.389 ms (the backward's loop is slower unrolled)
            for (int j = 0; j < cnt && alive > 0; ++j) {
                const float4 P = s_pos[j];
                const float4 K = s_con[j];
                const float dy = __fsub_rn(__fsub_rn(fj, P.y), P.w);
                float centre, rowt;
                row_terms(K, P.z, dy, centre, rowt);
                // exponents of all PPT pixels first: independent chains, no branches
                float pk[PPT];
                if (!any_split) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const float t = __fsub_rn(__fsub_rn(fik[k], P.x), centre);
                        pk[k] = slice_exponent(K, t, rowt);
                    }
                } else {
                    const float fsplit = s_col[j].w, fc2 = s_fc2[j];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const float t = __fsub_rn(__fsub_rn(fik[k], (fik[k] >= fsplit) ? fc2 : P.x), centre);
                        pk[k] = slice_exponent(K, t, rowt);
                    }
                }
                bool any = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) any |= (!done[k]) & (pk[k] >= kLog2AlphaMin);
                if (!any) continue;
                const float4 c = s_col[j];
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (done[k] || pk[k] < kLog2AlphaMin) continue;
                    const float alpha = fminf(kAlphaMax, alpha_exp2(pk[k]));
                    const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                    if (Tn < kTMin) {
                        done[k] = true;
                        tested[k] = b0 + j + 1;
                        --alive;
                        continue;
                    }
                    const float w = __fmul_rn(alpha, T[k]);
                    C0[k] = __fmaf_rn(c.x, w, C0[k]);
                    C1[k] = __fmaf_rn(c.y, w, C1[k]);
                    C2[k] = __fmaf_rn(c.z, w, C2[k]);
                    T[k] = Tn;
                    last[k] = b0 + j + 1;
                    ++blended;
                }
            }
            if (__syncthreads_count(alive > 0) == 0) break;
        }
        int tmax = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) tmax = max(tmax, tested[k]);
        tmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)tmax);
        if ((tid & 31) == 0 && tmax > 0) atomicMax(&s_etile, (uint32_t)tmax);
        if (inside) {
            const int HW = V.W * V.H;
            float* img = a.images[v];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int pix = y * V.W + xp + k * tpr;
                img[pix] = __fmaf_rn(T[k], a.bg[0], C0[k]);
                img[HW + pix] = __fmaf_rn(T[k], a.bg[1], C1[k]);
                img[2 * HW + pix] = __fmaf_rn(T[k], a.bg[2], C2[k]);
                a.T_final[V.pix_base + pix] = T[k];
                a.n_last[V.pix_base + pix] = (uint32_t)last[k];
                if (a.user_T[v]) a.user_T[v][pix] = T[k];
                evals += (uint32_t)tested[k];
            }
        }
    }
    unsigned long long ev = evals;
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if ((tid & 31) == 0 && ev) atomicAdd(&a.hdr->evals_fwd, ev);
    unsigned long long bl = blended;
    for (int o = 16; o > 0; o >>= 1) bl += __shfl_xor_sync(0xffffffffu, bl, o);
    if ((tid & 31) == 0 && bl) atomicAdd(&a.hdr->blended, bl);
    if (tid == 0 && etile) atomicAdd(&a.hdr->entries_tile, etile);
}

size_t render_fwd_smem(int batch) { return (size_t)batch * (3 * sizeof(float4) + sizeof(float)); }

int pixels_per_thread(int tile_w, int tile_h, int want, int prefer) {
    const int area = tile_w * tile_h;
    auto fits = [&](int p) { return tile_w % p == 0 && (area / p) % 32 == 0 && area / p <= 256; };
    if (want != 0) return (want == 1 || want == 2 || want == 4 || want == 8) && fits(want) ? want : 0;
    if (fits(prefer)) return prefer;
    for (int p = 4; p >= 1; p >>= 1)
        if (fits(p)) return p;
    return 0;
}

int render_fwd_occupancy(int tile_w, int tile_h, int batch, int ppt) {
    if (ppt == 0) return 1;
    const int threads = tile_w * tile_h / ppt;
    const size_t sm = render_fwd_smem(batch);
    int nb = 0;
    cudaError_t e;
    switch (ppt) {
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<8>, threads, sm); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<4>, threads, sm); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<2>, threads, sm); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<1>, threads, sm); break;
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t launch_render_fwd(const FwdArgs& a, int grid, cudaStream_t st) {
    const int ppt = a.ppt;
    if (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 8) return cudaErrorInvalidValue;
    const int threads = a.tile_w * a.tile_h / ppt;
    const size_t sm = render_fwd_smem(a.batch);
    switch (ppt) {
        case 8: k_render_fwd<8><<<grid, threads, sm, st>>>(a); break;
        case 4: k_render_fwd<4><<<grid, threads, sm, st>>>(a); break;
        case 2: k_render_fwd<2><<<grid, threads, sm, st>>>(a); break;
        default: k_render_fwd<1><<<grid, threads, sm, st>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace odgs
