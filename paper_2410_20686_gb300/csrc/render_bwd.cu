// Backward alpha blending (reverse of Eq. 3) on ERP tiles (sm_103a).
//
// Same persistent (view, tile) schedule and layout as the forward kernel: PPT pixels of one row per
// thread, tile_w / PPT columns apart.
// Each pixel starts from its final transmittance and the index after its last blended Gaussian,
// and walks its tile list back to front, recovering T_j = T_{j+1} / (1 - alpha_j). Per blended
// Gaussian it forms
//   dL/drgb = alpha T g,   dL/dalpha = T (rgb . g) - (B . g) / (1 - alpha),
// with g = dL/dC and B the colour blended behind the Gaussian (background included), and from
// dL/dalpha the gradients w.r.t. opacity, the slice-form conic (a, beta, gamma) and ERP mean
// (u, v) through Eq. 2 (zero when alpha was clamped at 0.99). The skip / clamp decisions and alpha are recomputed
// with the forward kernel's exact operation sequence, so they match it bit for bit.
//
// A thread first sums over its PPT pixels, with dp = dL/d(power) and t the pixel's offset from the
// slice centre (the exponent's own variable), dp, dp t and dp t^2 and dL/drgb; with dy the same
// for all of a thread's pixels, these and dy times the first two and dy^2 times the first are the
// nine values (sum dp t gives the mean terms free of the cancellation an image-axis form suffers
// for needle-like Gaussians). The warp sums them over its lanes with a transpose
// reduction (12 shuffles for 9 values), the CTA over its warps in shared memory; then one thread
// per entry forms dL/d(u, v, conic, opacity), which are linear in these sums, and adds them to the
// per-(view, Gaussian) accumulator with three 16-byte vector atomics. A warp whose pixels all stopped before an entry skips it, and so does a warp
// none of whose pixel rows lies within the entry's footprint rows (the rows the binning lists the
// Gaussian in; outside them no pixel reaches alpha = 1/255); a warp with a single contributing
// lane skips the reduction.
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

// Sum v[0..8] over the warp. Returns the lane's share: value index *vi (valid iff *ok).
__device__ __forceinline__ float warp_reduce9(const float v[9], int lane, int* vi, bool* ok) {
    const unsigned full = 0xffffffffu;
    bool up = lane & 16;
    float w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float hi = (k + 5 < 9) ? v[k + 5] : 0.f;
        const float keep = up ? hi : v[k];
        const float send = up ? v[k] : hi;
        w[k] = keep + __shfl_xor_sync(full, send, 16);
    }
    up = lane & 8;
    float x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float hi = (k + 3 < 5) ? w[k + 3] : 0.f;
        const float keep = up ? hi : w[k];
        const float send = up ? w[k] : hi;
        x[k] = keep + __shfl_xor_sync(full, send, 8);
    }
    up = lane & 4;
    float y[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float hi = (k + 2 < 3) ? x[k + 2] : 0.f;
        const float keep = up ? hi : x[k];
        const float send = up ? x[k] : hi;
        y[k] = keep + __shfl_xor_sync(full, send, 4);
    }
    up = lane & 2;
    float z = (up ? y[1] : y[0]) + __shfl_xor_sync(full, up ? y[0] : y[1], 2);
    z += __shfl_xor_sync(full, z, 1);
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
    const int idx = 5 * b4 + 3 * b3 + 2 * b2 + b1;
    *vi = idx;
    *ok = ((lane & 1) == 0) && (2 * b2 + b1 < 3 - b3) && (idx < 9);
    return z;
}

template <int PPT>
__global__ void __launch_bounds__(256) k_render_bwd(BwdArgs a) {
    extern __shared__ float4 smem[];
    const int B = a.batch;
    const int nwarps = blockDim.x >> 5;
    float4* s_pos = smem;
    float4* s_con = smem + B;
    float4* s_col = smem + 2 * B;
    float4* s_raw = smem + 3 * B;  // a, beta, gamma (slice-form conic), 1 / opacity
    int2* s_rows = reinterpret_cast<int2*>(smem + 4 * B);  // pixel rows the footprint reaches
    float* s_fc2 = reinterpret_cast<float*>(s_rows + B);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_fc2 + B);
    float* s_red = reinterpret_cast<float*>(s_idx + B);  // [B][nwarps][9]
    __shared__ int s_item;
    __shared__ int s_maxn;

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int tw = a.tile_w;
    const int tpr = tw / PPT;
    // a thread's PPT pixels are tpr columns apart (interleaved), so a footprint a few pixels wide
    // falls in one of each lane's pixel slots rather than in several
    const int lx0 = tid % tpr, ly = tid / tpr;
    const int wy0 = (warp << 5) / tpr, wy1 = ((warp << 5) + 31) / tpr;  // the warp's tile rows
    uint32_t evals = 0u;

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_item = (int)atomicAdd(&a.hdr->work_bwd, 1u);
            s_maxn = 0;
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
        // entries past the tile's range (possible only when the lists were rebuilt after a sort
        // that gave up, so that they differ from the forward's) stage as never-blending entries
        const uint32_t rlen = rg.y > rg.x ? rg.y - rg.x : 0u;
        const int wr0 = ty * a.tile_h + wy0, wr1 = ty * a.tile_h + wy1;

        float T[PPT], Bg[PPT], g0[PPT], g1[PPT], g2[PPT];
        int nl[PPT];
        int tmax = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            T[k] = 1.f; Bg[k] = 0.f; g0[k] = g1[k] = g2[k] = 0.f; nl[k] = 0;
            if (inside) {
                const int pix = y * V.W + xp + k * tpr;
                const int HW = V.W * V.H;
                T[k] = a.T_final[V.pix_base + pix];
                nl[k] = (int)a.n_last[V.pix_base + pix];
                const float* gi = a.dL_dimages[v];
                g0[k] = gi[pix]; g1[k] = gi[HW + pix]; g2[k] = gi[2 * HW + pix];
                if (a.checked) {  // a non-finite gradient value counts as 0 and is reported
                    const bool f0 = isfinite(g0[k]), f1 = isfinite(g1[k]), f2 = isfinite(g2[k]);
                    if (!(f0 && f1 && f2)) {
                        atomicOr(&a.hdr->status, kStNonfinite);
                        g0[k] = f0 ? g0[k] : 0.f; g1[k] = f1 ? g1[k] : 0.f; g2[k] = f2 ? g2[k] : 0.f;
                    }
                }
                Bg[k] = T[k] * (a.bg[0] * g0[k] + a.bg[1] * g1[k] + a.bg[2] * g2[k]);
                tmax = max(tmax, nl[k]);
                evals += (uint32_t)nl[k];
            }
        }
        if (tmax > 0) atomicMax(&s_maxn, tmax);
        __syncthreads();
        const int maxn = s_maxn;
        const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)tmax);  // warp-uniform bound

        for (int hi = maxn; hi > 0; hi -= B) {
            const int lo = max(0, hi - B);
            const int cnt = hi - lo;
            int split = 0;
            for (int j = tid; j < cnt; j += nthr) {
                const uint32_t idx = (uint32_t)(lo + j) < rlen ? a.pair_vals[rg.x + lo + j] : 0xFFFFFFFFu;
                float4 ra, rb, rc;
                gather_records(a.rec_a, a.rec_b, a.rec_c, idx, a.n_items, ra, rb, rc);
                Staged s = stage_entry(ra, rb, rc, x0, tw, V.W, V.model == 0);
                s_pos[j] = s.pos;
                s_con[j] = s.con;
                s_col[j] = s.col;
                s_fc2[j] = s.fc2;
                s_raw[j] = make_float4(rb.x, rb.y, rb.z, ra.w > 0.f ? 1.f / ra.w : 0.f);
                s_idx[j] = idx < a.n_items ? idx : 0u;
                s_rows[j] = footprint_row_range(ra, rb, V.H);
                split |= (s.col.w <= 1e30f);
            }
            const int any_split = __syncthreads_or(split);
            for (int j = cnt - 1; j >= 0; --j) {
                const int e = lo + j;
                float* red = s_red + ((size_t)j * nwarps + warp) * 9;
                const int2 rows = s_rows[j];
                // no pixel of this warp reached entry e in the forward pass, or none of its rows is
                // within the footprint's rows
                if (e >= wmax || rows.y < wr0 || rows.x > wr1) {
                    if (lane < 9) red[lane] = 0.f;
                    continue;
                }
                // sums over this thread's pixels of dp, dp t and dp t^2 (dp = dL/d power) and of
                // dL/drgb; the conic, opacity and mean terms are linear in these and in dy times them,
                // so the warp reduces them and the CTA pass after the batch forms the terms
                float S0 = 0.f, S1 = 0.f, S2 = 0.f, V0 = 0.f, V1 = 0.f, V2 = 0.f, dy = 0.f;
                bool contrib = false;
                if (e < tmax) {
                    const float4 P = s_pos[j];
                    const float4 K = s_con[j];
                    dy = __fsub_rn(__fsub_rn(fj, P.y), P.w);
                    float centre, rowt;
                    row_terms(K, P.z, dy, centre, rowt);
                    // exponents of all PPT pixels first (the forward kernel's exact sequence); t is
                    // the pixel's offset from the slice centre, dx = t + (centre - du)
                    float pk[PPT], tk[PPT];
                    if (!any_split) {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            tk[k] = __fsub_rn(__fsub_rn(fik[k], P.x), centre);
                            pk[k] = slice_exponent(K, tk[k], rowt);
                        }
                    } else {
                        const float fsplit = s_col[j].w, fc2 = s_fc2[j];
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            tk[k] = __fsub_rn(__fsub_rn(fik[k], (fik[k] >= fsplit) ? fc2 : P.x), centre);
                            pk[k] = slice_exponent(K, tk[k], rowt);
                        }
                    }
                    const float4 c = s_col[j];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (e >= nl[k] || pk[k] < kLog2AlphaMin) continue;
                        contrib = true;
                        const float t = tk[k];
                        const float ar = alpha_exp2(pk[k]);
                        const float alpha = fminf(kAlphaMax, ar);
                        const float inv = __fdividef(1.f, __fsub_rn(1.f, alpha));
                        const float Tj = T[k] * inv;
                        const float w = alpha * Tj;
                        const float cg = c.x * g0[k] + c.y * g1[k] + c.z * g2[k];
                        V0 = fmaf(w, g0[k], V0);
                        V1 = fmaf(w, g1[k], V1);
                        V2 = fmaf(w, g2[k], V2);
                        const float dLda = Tj * cg - Bg[k] * inv;
                        Bg[k] = fmaf(cg, w, Bg[k]);
                        T[k] = Tj;
                        if (ar < kAlphaMax) {  // no gradient through the 0.99 clamp
                            const float dp = dLda * alpha;  // dL/d(power), power = ln G
                            const float dpt = dp * t;
                            S0 += dp;
                            S1 += dpt;
                            S2 = fmaf(dpt, t, S2);
                        }
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, contrib);
                if (m == 0u) {
                    if (lane < 9) red[lane] = 0.f;
                    continue;
                }
                // sum dp, sum dp t, sum dp t^2, sum dp t dy, sum dp dy, sum dp dy^2, dL/drgb
                const float dyS0 = dy * S0;
                const float vals[9] = {S0, S1, S2, dy * S1, dyS0, dy * dyS0, V0, V1, V2};
                if ((m & (m - 1u)) == 0u) {  // one contributing lane: no reduction needed
                    if (contrib) {
#pragma unroll
                        for (int q = 0; q < 9; ++q) red[q] = vals[q];
                    }
                } else {
                    int vi;
                    bool ok;
                    const float sm = warp_reduce9(vals, lane, &vi, &ok);
                    if (ok) red[vi] = sm;
                }
            }
            __syncthreads();
            // per entry: the warps' sums added, then the screen-space gradient terms. With (dx, dy) =
            // pixel - mean and power = ln o - (a t^2 + gamma dy^2) / 2, t = dx - beta dy (the conic in
            // slice form), the gradients w.r.t. the mean, the slice-form conic and the opacity are
            //   dL/du = a sum(dp t), dL/dv = -a beta sum(dp t) + gamma sum(dp dy),
            //   dL/da = -sum(dp t^2) / 2, dL/dbeta = a sum(dp t dy), dL/dgamma = -sum(dp dy^2) / 2,
            //   dL/do = sum(dp) / o.
            // Each sum is dominated by its own scale (t across the ellipse, dy along it), so even for a
            // needle-like Gaussian the thin direction's information is not a small difference of the
            // long direction's sums, as the conic's image-axis entries would make it.
            for (int jj = tid; jj < cnt; jj += nthr) {
                float q[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) q[k] = 0.f;
                for (int w = 0; w < nwarps; ++w) {
                    const float* r = s_red + ((size_t)jj * nwarps + w) * 9;
#pragma unroll
                    for (int k = 0; k < 9; ++k) q[k] += r[k];
                }
                const float4 R = s_raw[jj];  // a, beta, gamma, 1 / o
                const float du_ = R.x * q[1];
                const float4 p0 = make_float4(du_, fmaf(R.z, q[4], -R.y * du_), -0.5f * q[2], R.x * q[3]);
                const float4 p1 = make_float4(-0.5f * q[5], R.w * q[0], q[6], q[7]);
                float4* dst = a.acc + 3 * (size_t)s_idx[jj];
                if (p0.x != 0.f || p0.y != 0.f || p0.z != 0.f || p0.w != 0.f) red_add_v4(dst, p0);
                if (p1.x != 0.f || p1.y != 0.f || p1.z != 0.f || p1.w != 0.f) red_add_v4(dst + 1, p1);
                if (q[8] != 0.f) red_add_v4(dst + 2, make_float4(q[8], 0.f, 0.f, 0.f));
            }
            __syncthreads();  // the next batch overwrites the staged entries and s_red
        }
    }
    unsigned long long ev = evals;
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if (lane == 0 && ev) atomicAdd(&a.hdr->evals_bwd, ev);
}

size_t render_bwd_smem(int batch, int threads) {
    return (size_t)batch * (4 * sizeof(float4) + sizeof(int2) + sizeof(float) + sizeof(uint32_t)) +
           (size_t)batch * (threads / 32) * 9 * sizeof(float);
}

int render_bwd_occupancy(int tile_w, int tile_h, int batch, int ppt) {
    if (ppt == 0) return 1;
    const int threads = tile_w * tile_h / ppt;
    const size_t sm = render_bwd_smem(batch, threads);
    int nb = 0;
    cudaError_t e;
    switch (ppt) {
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<8>, threads, sm); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<4>, threads, sm); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<2>, threads, sm); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<1>, threads, sm); break;
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t launch_render_bwd(const BwdArgs& a, int grid, cudaStream_t st) {
    const int ppt = a.ppt;
    if (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 8) return cudaErrorInvalidValue;
    const int threads = a.tile_w * a.tile_h / ppt;
    const size_t sm = render_bwd_smem(a.batch, threads);
    switch (ppt) {
        case 8: k_render_bwd<8><<<grid, threads, sm, st>>>(a); break;
        case 4: k_render_bwd<4><<<grid, threads, sm, st>>>(a); break;
        case 2: k_render_bwd<2><<<grid, threads, sm, st>>>(a); break;
        default: k_render_bwd<1><<<grid, threads, sm, st>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace odgs
