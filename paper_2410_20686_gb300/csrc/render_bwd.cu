// Backward alpha blending (reverse of Eq. 3) on ERP tiles (sm_103a).
//
// Same persistent (view, tile) schedule as the forward kernel. Each pixel starts from its final
// transmittance and the index after its last blended Gaussian, and walks its tile list back to
// front, recovering T_j = T_{j+1} / (1 - alpha_j). Per blended Gaussian it forms
//   dL/drgb = alpha T g,   dL/dalpha = T (rgb . g) - (B . g) / (1 - alpha),
// with g = dL/dC and B the colour blended behind the Gaussian (background included), and from
// dL/dalpha the gradients w.r.t. opacity, conic (a, b, c) and ERP mean (u, v) through Eq. 2
// (zero when alpha was clamped at 0.99).
//
// The nine per-Gaussian values are summed over the 32 pixels of a warp with a transpose
// reduction (12 shuffles instead of 45), over the warps of the CTA in shared memory, and then
// added to the per-(view, Gaussian) accumulator with three 16-byte vector atomics.
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

template <int MAXT>
__global__ void __launch_bounds__(MAXT) k_render_bwd(BwdArgs a) {
    extern __shared__ float4 smem[];
    const int B = a.batch;
    const int nwarps = blockDim.x >> 5;
    float4* s_pos = smem;
    float4* s_con = smem + B;
    float4* s_col = smem + 2 * B;
    float4* s_raw = smem + 3 * B;  // conic a, b, c, 1 / opacity
    float* s_fc2 = reinterpret_cast<float*>(smem + 4 * B);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_fc2 + B);
    float* s_red = reinterpret_cast<float*>(s_idx + B);  // [B][nwarps][9]
    __shared__ int s_item;
    __shared__ int s_maxn;

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int tw = a.tile_w;
    const int lx = tid % tw, ly = tid / tw;
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
        const int x = x0 + lx, y = ty * a.tile_h + ly;
        const bool inside = y < V.H;
        const float fi = (float)x, fj = (float)y;
        const uint2 rg = a.ranges[item];

        float T = 1.f, Bg = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        int nl = 0;
        if (inside) {
            const int pix = y * V.W + x;
            const int HW = V.W * V.H;
            T = a.T_final[V.pix_base + pix];
            nl = (int)a.n_last[V.pix_base + pix];
            const float* gi = a.dL_dimages[v];
            g0 = gi[pix]; g1 = gi[HW + pix]; g2 = gi[2 * HW + pix];
            Bg = T * (a.bg[0] * g0 + a.bg[1] * g1 + a.bg[2] * g2);
            if (nl > 0) atomicMax(&s_maxn, nl);
        }
        __syncthreads();
        const int maxn = s_maxn;
        const int wmax = __reduce_max_sync(0xffffffffu, (unsigned)nl);  // warp-uniform bound
        evals += (uint32_t)nl;

        for (int hi = maxn; hi > 0; hi -= B) {
            const int lo = max(0, hi - B);
            const int cnt = hi - lo;
            int split = 0;
            for (int j = tid; j < cnt; j += nthr) {
                const uint32_t idx = a.pair_vals[rg.x + lo + j];
                float4 ra, rb, rc;
                gather_records(a.rec_a, a.rec_b, a.rec_c, idx, a.n_items, ra, rb, rc);
                Staged s = stage_entry(ra, rb, rc, x0, tw, V.W);
                s_pos[j] = s.pos;
                s_con[j] = s.con;
                s_col[j] = s.col;
                s_fc2[j] = s.fc2;
                s_raw[j] = make_float4(rb.x, rb.y, rb.z, ra.w > 0.f ? 1.f / ra.w : 0.f);
                s_idx[j] = idx < a.n_items ? idx : 0u;
                split |= (s.col.w <= 1e30f);
            }
            const int any_split = __syncthreads_or(split);
            for (int j = cnt - 1; j >= 0; --j) {
                const int e = lo + j;
                float* red = s_red + ((size_t)j * nwarps + warp) * 9;
                if (e >= wmax) {  // no pixel of this warp reached entry e in the forward pass
                    if (lane < 9) red[lane] = 0.f;
                    continue;
                }
                float vals[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) vals[k] = 0.f;
                bool contrib = false;
                if (e < nl) {
                    const float4 P = s_pos[j];
                    const float4 c = s_col[j];
                    const float fc = (any_split && fi >= c.w) ? s_fc2[j] : P.x;
                    float dx, dy;
                    pixel_offset(fi, fj, fc, P, dx, dy);
                    const float p = gauss_exponent(s_con[j], dx, dy);
                    if (p >= kLog2AlphaMin) {
                        contrib = true;
                        const float ar = exp2f(p);
                        const float alpha = fminf(kAlphaMax, ar);
                        const float om = __fsub_rn(1.f, alpha);
                        const float Tj = __fdiv_rn(T, om);
                        const float w = alpha * Tj;
                        const float cg = c.x * g0 + c.y * g1 + c.z * g2;
                        vals[6] = w * g0;
                        vals[7] = w * g1;
                        vals[8] = w * g2;
                        const float dLda = Tj * cg - Bg / om;
                        Bg = fmaf(cg, w, Bg);
                        T = Tj;
                        if (ar < kAlphaMax) {
                            const float4 R = s_raw[j];
                            const float dp = dLda * alpha;  // dL/d(power), power = ln G
                            vals[5] = dp * R.w;
                            vals[2] = dp * (-0.5f * dx * dx);
                            vals[3] = dp * (-dx * dy);
                            vals[4] = dp * (-0.5f * dy * dy);
                            vals[0] = dp * (R.x * dx + R.y * dy);
                            vals[1] = dp * (R.y * dx + R.z * dy);
                        }
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, contrib);
                if (m == 0u) {
                    if (lane < 9) red[lane] = 0.f;
                } else if ((m & (m - 1u)) == 0u) {  // one contributing pixel: no reduction needed
                    if (contrib) {
#pragma unroll
                        for (int k = 0; k < 9; ++k) red[k] = vals[k];
                    }
                } else {
                    int vi;
                    bool ok;
                    const float sm = warp_reduce9(vals, lane, &vi, &ok);
                    if (ok) red[vi] = sm;
                }
            }
            __syncthreads();
            for (int q = tid; q < cnt * 3; q += nthr) {
                const int jj = q / 3, part = q - 3 * jj;
                const int nv = part < 2 ? 4 : 1;
                float sum[4] = {0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < nwarps; ++w) {
                    const float* r = s_red + ((size_t)jj * nwarps + w) * 9 + 4 * part;
                    for (int k = 0; k < nv; ++k) sum[k] += r[k];
                }
                if (sum[0] != 0.f || sum[1] != 0.f || sum[2] != 0.f || sum[3] != 0.f)
                    red_add_v4(a.acc + 3 * (size_t)s_idx[jj] + part, make_float4(sum[0], sum[1], sum[2], sum[3]));
            }
            __syncthreads();  // the next batch overwrites the staged entries and s_red
        }
    }
    unsigned long long ev = evals;
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if (lane == 0 && ev) atomicAdd(&a.hdr->evals_bwd, ev);
}

size_t render_bwd_smem(int batch, int threads) {
    return (size_t)batch * (4 * sizeof(float4) + sizeof(float) + sizeof(uint32_t)) +
           (size_t)batch * (threads / 32) * 9 * sizeof(float);
}

int render_bwd_occupancy(int threads, int batch) {
    int nb = 0;
    size_t sm = render_bwd_smem(batch, threads);
    cudaError_t e;
    if (threads <= 64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<64>, threads, sm);
    else if (threads <= 128) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<128>, threads, sm);
    else if (threads <= 256) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<256>, threads, sm);
    else if (threads <= 512) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<512>, threads, sm);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<1024>, threads, sm);
    return e == cudaSuccess ? max(nb, 1) : 1;
}

template <int MAXT>
static cudaError_t launch_bwd_t(const BwdArgs& a, int grid, cudaStream_t st) {
    const int threads = a.tile_w * a.tile_h;
    size_t sm = render_bwd_smem(a.batch, threads);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_render_bwd<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_render_bwd<MAXT><<<grid, threads, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const BwdArgs& a, int grid, cudaStream_t st) {
    const int threads = a.tile_w * a.tile_h;
    if (threads <= 64) return launch_bwd_t<64>(a, grid, st);
    if (threads <= 128) return launch_bwd_t<128>(a, grid, st);
    if (threads <= 256) return launch_bwd_t<256>(a, grid, st);
    if (threads <= 512) return launch_bwd_t<512>(a, grid, st);
    return launch_bwd_t<1024>(a, grid, st);
}

}  // namespace odgs
