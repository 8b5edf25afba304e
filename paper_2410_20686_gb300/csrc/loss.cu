// L1 + D-SSIM loss of 3DGS training on ERP images, forward and gradient (sm_103a).
//
// SSIM_mean = sum_q c_q s_q with c_q the pixel's weight (cos(theta) of its row, or 1) over the
// weight of all 3 W H values, and s_q = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sxx + syy + C2))
// from window moments mx = g * x, sxx = g * x^2 - mx^2, sxy = g * xy - mx my (g: the separable
// 11-tap Gaussian). Because every moment is a correlation with g, which is symmetric,
//   dSSIM_mean / dx_p = (g * A)_p + 2 x_p (g * B)_p + y_p (g * C)_p,
//   A = c (ds/dmx - 2 mx ds/dsxx - my ds/dsxy),  B = c ds/dsxx,  C = c ds/dsxy.
//   k_ssim_fwd    per 32 x 32 tile and channel: the image and target with a 5-pixel halo in shared
//                 memory (cp.async, double-buffered: the next channel loads while this one computes), a horizontal then a vertical 11-tap pass for the five moments (each thread
//                 computes 4 outputs from the 14 inputs it loads once), then s, the loss partial
//                 and the maps A, B, C (scratch)
//   k_ssim_bwd    the same tiling over A, B, C: two passes, then the gradient with the L1 term
//   k_l1          lambda = 0: the L1 term alone, one pass
//   k_loss_reduce one CTA: the CTAs' partials in a fixed order (deterministic)
// Rows outside the image are zero (zero padding); columns wrap around the seam or are zero.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "odgs_train.h"

namespace {

constexpr int kR = 5;
constexpr int kWin = 2 * kR + 1;
constexpr int kTX = 32, kTY = 32;
constexpr int kInW = kTX + 2 * kR, kInH = kTY + 2 * kR;
constexpr int kLd = kInW + 1;  // odd row stride of the input tiles: rows of a warp hit distinct banks
constexpr int kHd = kTX + 1;   // row stride of the horizontal pass's output
constexpr int kCB = 4;         // outputs per thread in each pass (register blocking)
constexpr int kThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct LossArgs {
    const float* x;
    const float* y;
    float* grad;
    float* maps;     // [3 channels][3 maps A, B, C][H][W]
    float* partial;  // [CTAs]
    int W, H, wrap, area;
    float lam, inv_wsum;
    float g[kWin];
};

__device__ __forceinline__ float row_weight(const LossArgs& a, int j) {
    // cos of the row centre's elevation pi (1/2 - (j + 1/2) / H) = sin(pi (j + 1/2) / H)
    return a.area ? sinpif(((float)j + 0.5f) / (float)a.H) : 1.f;
}

// Copies rows [y0 - kR, y0 + kTY + kR) x columns [x0 - kR, x0 + kTX + kR) of src into dst with
// asynchronous 4-byte copies (cp.async; zero-filled outside the image): the caller commits the
// group and waits for it later, so the copy overlaps the previous channel's passes.
__device__ __forceinline__ void load_halo_async(const LossArgs& a, const float* __restrict__ src, float (*dst)[kLd],
                                                int x0, int y0) {
    for (int i = threadIdx.x; i < kInH * kInW; i += kThreads) {
        const int r = i / kInW, q = i - r * kInW;
        const int gy = y0 + r - kR;
        int gx = x0 + q - kR;
        bool ok = gy >= 0 && gy < a.H;
        if (a.wrap) {  // gx lies in [-5, W + 36]: one wrap unless the image is narrower than that
            if (gx < 0) gx += a.W;
            else if (gx >= a.W) gx -= a.W;
            if (gx < 0 || gx >= a.W) gx = ((gx % a.W) + a.W) % a.W;
        } else {
            ok = ok && gx >= 0 && gx < a.W;
        }
        const float* g = ok ? src + (size_t)gy * a.W + gx : src;
        const unsigned d = (unsigned)__cvta_generic_to_shared(&dst[r][q]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(g), "r"(ok ? 4 : 0) : "memory");
    }
}

__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ float block_sum(float v, float* s_red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
    return t;
}

// Forward: per channel, the 11-tap passes with register blocking (a thread computes kCB outputs
// from the kCB + 10 inputs it loads once), then SSIM, the loss partial and the maps A, B, C.
__global__ void __launch_bounds__(kThreads) k_ssim_fwd(LossArgs a) {
    // dynamic shared memory (above the 48 KB static limit): input tiles double-buffered over the
    // channels, then the horizontal pass's five moments
    extern __shared__ float s_dyn[];
    float (*s_xb)[kInH][kLd] = reinterpret_cast<float (*)[kInH][kLd]>(s_dyn);
    float (*s_yb)[kInH][kLd] = s_xb + 2;
    float (*s_h)[kInH][kHd] = reinterpret_cast<float (*)[kInH][kHd]>(s_yb + 2);
    __shared__ float s_red[kThreads / 32];
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const size_t HW = (size_t)a.W * a.H;
    float part = 0.f;
    load_halo_async(a, a.x, s_xb[0], x0, y0);
    load_halo_async(a, a.y, s_yb[0], x0, y0);
    async_commit();
    for (int c = 0; c < 3; ++c) {
        if (c < 2) {  // the next channel's tiles load while this one computes
            load_halo_async(a, a.x + (c + 1) * HW, s_xb[(c + 1) & 1], x0, y0);
            load_halo_async(a, a.y + (c + 1) * HW, s_yb[(c + 1) & 1], x0, y0);
            async_commit();
            async_wait<1>();
        } else {
            async_wait<0>();
        }
        __syncthreads();
        float (*s_x)[kLd] = s_xb[c & 1];
        float (*s_y)[kLd] = s_yb[c & 1];
        // horizontal: rows [0, kInH) x output columns [0, kTX); lanes take consecutive rows
        for (int it = threadIdx.x; it < kInH * (kTX / kCB); it += kThreads) {
            const int r = it % kInH, q0 = (it / kInH) * kCB;
            float o[5][kCB];
#pragma unroll
            for (int m = 0; m < 5; ++m)
#pragma unroll
                for (int j = 0; j < kCB; ++j) o[m][j] = 0.f;
#pragma unroll
            for (int i = 0; i < kCB + 2 * kR; ++i) {
                const float xv = s_x[r][q0 + i], yv = s_y[r][q0 + i];
                const float xx = xv * xv, yy = yv * yv, xy = xv * yv;
#pragma unroll
                for (int j = 0; j < kCB; ++j) {
                    const int k = i - j;
                    if (k < 0 || k >= kWin) continue;
                    const float gk = a.g[k];
                    o[0][j] = fmaf(gk, xv, o[0][j]);
                    o[1][j] = fmaf(gk, yv, o[1][j]);
                    o[2][j] = fmaf(gk, xx, o[2][j]);
                    o[3][j] = fmaf(gk, yy, o[3][j]);
                    o[4][j] = fmaf(gk, xy, o[4][j]);
                }
            }
#pragma unroll
            for (int m = 0; m < 5; ++m)
#pragma unroll
                for (int j = 0; j < kCB; ++j) s_h[m][r][q0 + j] = o[m][j];
        }
        __syncthreads();
        // vertical: output rows [r0, r0 + kCB) of column q; lanes take consecutive columns
        for (int it = threadIdx.x; it < kTX * (kTY / kCB); it += kThreads) {
            const int q = it % kTX, r0 = (it / kTX) * kCB;
            float o[5][kCB];
#pragma unroll
            for (int m = 0; m < 5; ++m)
#pragma unroll
                for (int j = 0; j < kCB; ++j) o[m][j] = 0.f;
#pragma unroll
            for (int i = 0; i < kCB + 2 * kR; ++i) {
                float h[5];
#pragma unroll
                for (int m = 0; m < 5; ++m) h[m] = s_h[m][r0 + i][q];
#pragma unroll
                for (int j = 0; j < kCB; ++j) {
                    const int k = i - j;
                    if (k < 0 || k >= kWin) continue;
                    const float gk = a.g[k];
#pragma unroll
                    for (int m = 0; m < 5; ++m) o[m][j] = fmaf(gk, h[m], o[m][j]);
                }
            }
            const int gx = x0 + q;
#pragma unroll
            for (int j = 0; j < kCB; ++j) {
                const int gy = y0 + r0 + j;
                if (gy >= a.H || gx >= a.W) continue;
                const float mx = o[0][j], my = o[1][j];
                const float sxx = o[2][j] - mx * mx, syy = o[3][j] - my * my, sxy = o[4][j] - mx * my;
                const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
                const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
                const float iB1 = 1.f / B1, iB2 = 1.f / B2;
                const float sv = A1 * A2 * iB1 * iB2;
                const float ds_dmx = 2.f * A2 * (my * B1 - mx * A1) * iB1 * iB1 * iB2;
                const float ds_dsxx = -sv * iB2;
                const float ds_dsxy = 2.f * A1 * iB1 * iB2;
                const float xv = s_x[r0 + j + kR][q + kR], yv = s_y[r0 + j + kR][q + kR];
                const float w = row_weight(a, gy) * a.inv_wsum;
                part = fmaf(w, (1.f - a.lam) * fabsf(xv - yv) + a.lam * (1.f - sv), part);
                float* mp = a.maps + (size_t)(3 * c) * HW + (size_t)gy * a.W + gx;
                mp[0] = w * (ds_dmx - 2.f * mx * ds_dsxx - my * ds_dsxy);
                mp[HW] = w * ds_dsxx;
                mp[2 * HW] = w * ds_dsxy;
            }
        }
        __syncthreads();  // the next channel overwrites the tiles
    }
    const float t = block_sum(part, s_red);
    if (threadIdx.x == 0) a.partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Backward: the same blocked passes over the maps A, B, C, then the gradient with the L1 term.
__global__ void __launch_bounds__(kThreads) k_ssim_bwd(LossArgs a) {
    // dynamic shared memory: the three maps' tiles double-buffered over the channels, then the
    // horizontal pass's outputs
    extern __shared__ float s_dyn[];
    float (*s_mb)[3][kInH][kLd] = reinterpret_cast<float (*)[3][kInH][kLd]>(s_dyn);
    float (*s_h)[kInH][kHd] = reinterpret_cast<float (*)[kInH][kHd]>(s_mb + 2);
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const size_t HW = (size_t)a.W * a.H;
    for (int k = 0; k < 3; ++k) load_halo_async(a, a.maps + (size_t)k * HW, s_mb[0][k], x0, y0);
    async_commit();
    for (int c = 0; c < 3; ++c) {
        if (c < 2) {  // the next channel's maps load while this one computes
            for (int k = 0; k < 3; ++k)
                load_halo_async(a, a.maps + (size_t)(3 * (c + 1) + k) * HW, s_mb[(c + 1) & 1][k], x0, y0);
            async_commit();
            async_wait<1>();
        } else {
            async_wait<0>();
        }
        __syncthreads();
        float (*s_m)[kInH][kLd] = s_mb[c & 1];
        for (int it = threadIdx.x; it < kInH * (kTX / kCB); it += kThreads) {
            const int r = it % kInH, q0 = (it / kInH) * kCB;
            float o[3][kCB];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int j = 0; j < kCB; ++j) o[m][j] = 0.f;
#pragma unroll
            for (int i = 0; i < kCB + 2 * kR; ++i) {
                float v[3];
#pragma unroll
                for (int m = 0; m < 3; ++m) v[m] = s_m[m][r][q0 + i];
#pragma unroll
                for (int j = 0; j < kCB; ++j) {
                    const int k = i - j;
                    if (k < 0 || k >= kWin) continue;
                    const float gk = a.g[k];
#pragma unroll
                    for (int m = 0; m < 3; ++m) o[m][j] = fmaf(gk, v[m], o[m][j]);
                }
            }
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int j = 0; j < kCB; ++j) s_h[m][r][q0 + j] = o[m][j];
        }
        __syncthreads();
        for (int it = threadIdx.x; it < kTX * (kTY / kCB); it += kThreads) {
            const int q = it % kTX, r0 = (it / kTX) * kCB;
            float o[3][kCB];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int j = 0; j < kCB; ++j) o[m][j] = 0.f;
#pragma unroll
            for (int i = 0; i < kCB + 2 * kR; ++i) {
                float h[3];
#pragma unroll
                for (int m = 0; m < 3; ++m) h[m] = s_h[m][r0 + i][q];
#pragma unroll
                for (int j = 0; j < kCB; ++j) {
                    const int k = i - j;
                    if (k < 0 || k >= kWin) continue;
                    const float gk = a.g[k];
#pragma unroll
                    for (int m = 0; m < 3; ++m) o[m][j] = fmaf(gk, h[m], o[m][j]);
                }
            }
            const int gx = x0 + q;
#pragma unroll
            for (int j = 0; j < kCB; ++j) {
                const int gy = y0 + r0 + j;
                if (gy >= a.H || gx >= a.W) continue;
                const size_t pix = c * HW + (size_t)gy * a.W + gx;
                const float xv = a.x[pix], yv = a.y[pix];
                const float d = xv - yv;
                const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                const float w = row_weight(a, gy) * a.inv_wsum;
                a.grad[pix] = (1.f - a.lam) * w * sgn - a.lam * (o[0][j] + 2.f * xv * o[1][j] + yv * o[2][j]);
            }
        }
        __syncthreads();
    }
}

// lambda = 0: the weighted L1 term alone, one pass over the pixels (no window): the loss partial
// of each CTA and the gradient w sign(x - y) / (weight sum).
__global__ void __launch_bounds__(kThreads) k_l1(LossArgs a) {
    __shared__ float s_red[kThreads / 32];
    float part = 0.f;
    // 16-byte loads and stores when every row starts on a 16-byte boundary
    const bool vec = (a.W & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.y) |
                                         reinterpret_cast<uintptr_t>(a.grad)) & 15u) == 0;
    for (int rc = blockIdx.x; rc < 3 * a.H; rc += gridDim.x) {  // (channel, row) pairs
        const int row = rc % a.H;
        const float w = row_weight(a, row) * a.inv_wsum;
        const size_t base = (size_t)rc * a.W;
        if (vec) {
            const float4* x4 = reinterpret_cast<const float4*>(a.x + base);
            const float4* y4 = reinterpret_cast<const float4*>(a.y + base);
            for (int c4 = threadIdx.x; c4 < (a.W >> 2); c4 += kThreads) {
                const float4 xv = x4[c4], yv = y4[c4];
                const float d[4] = {xv.x - yv.x, xv.y - yv.y, xv.z - yv.z, xv.w - yv.w};
                float gq[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    part = fmaf(w, fabsf(d[k]), part);
                    gq[k] = d[k] > 0.f ? w : (d[k] < 0.f ? -w : 0.f);
                }
                if (a.grad) reinterpret_cast<float4*>(a.grad + base)[c4] = make_float4(gq[0], gq[1], gq[2], gq[3]);
            }
            continue;
        }
        for (int col = threadIdx.x; col < a.W; col += kThreads) {
            const float d = a.x[base + col] - a.y[base + col];
            part = fmaf(w, fabsf(d), part);
            if (a.grad) a.grad[base + col] = d > 0.f ? w : (d < 0.f ? -w : 0.f);
        }
    }
    const float t = block_sum(part, s_red);
    if (threadIdx.x == 0) a.partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads) k_loss_reduce(const float* __restrict__ partial, int n, float* loss,
                                                          int accumulate) {
    __shared__ float s_red[kThreads / 32];
    float v = 0.f;
    for (int i = threadIdx.x; i < n; i += kThreads) v += partial[i];
    const float t = block_sum(v, s_red);
    if (threadIdx.x == 0) *loss = accumulate ? *loss + t : t;
}

int blocks_for(int W, int H) { return ((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY); }

size_t scratch_for(int W, int H) {
    const size_t maps = 9 * (size_t)W * H * sizeof(float);
    return ((maps + 15) & ~(size_t)15) + (size_t)blocks_for(W, H) * sizeof(float);
}

}  // namespace

extern "C" odgs_status odgs_loss_scratch_size(int width, int height, size_t* bytes) {
    if (!bytes || width < 1 || height < 1) return ODGS_ERR_INVALID_ARG;
    *bytes = scratch_for(width, height);
    return ODGS_OK;
}

extern "C" odgs_status odgs_loss_l1_dssim(const float* image, const float* target, int width, int height,
                                          const odgs_loss_params* p, float* grad, float* loss, void* scratch,
                                          size_t scratch_bytes, void* stream) {
    if (!image || !target || !p || !loss || width < 1 || height < 1) return ODGS_ERR_INVALID_ARG;
    if (!(p->lambda >= 0.f && p->lambda <= 1.f)) return ODGS_ERR_INVALID_ARG;
    if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 15u) || scratch_bytes < scratch_for(width, height))
        return ODGS_ERR_WORKSPACE;
    LossArgs a{};
    a.x = image; a.y = target; a.grad = grad;
    a.maps = static_cast<float*>(scratch);
    a.partial = reinterpret_cast<float*>(static_cast<char*>(scratch) + (scratch_for(width, height) -
                                                                        (size_t)blocks_for(width, height) * sizeof(float)));
    a.W = width; a.H = height; a.wrap = p->wrap_u ? 1 : 0; a.area = p->area_weight ? 1 : 0;
    a.lam = p->lambda;
    double wsum = 0.0, gsum = 0.0;
    for (int j = 0; j < height; ++j) wsum += a.area ? std::sin(M_PI * (j + 0.5) / height) : 1.0;
    a.inv_wsum = (float)(1.0 / (3.0 * width * wsum));
    double g[kWin];
    for (int k = 0; k < kWin; ++k) {
        const double d = k - kR;
        g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        gsum += g[k];
    }
    for (int k = 0; k < kWin; ++k) a.g[k] = (float)(g[k] / gsum);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->lambda == 0.f) {  // L1 alone: no SSIM window
        const int blocks = min(blocks_for(width, height), 3 * height);
        k_l1<<<blocks, kThreads, 0, st>>>(a);
        k_loss_reduce<<<1, kThreads, 0, st>>>(a.partial, blocks, loss, p->accumulate ? 1 : 0);
        return cudaGetLastError() == cudaSuccess ? ODGS_OK : ODGS_ERR_CUDA;
    }
    const dim3 grid((width + kTX - 1) / kTX, (height + kTY - 1) / kTY);
    constexpr size_t kFwdSmem = sizeof(float) * (4 * kInH * kLd + 5 * kInH * kHd);
    constexpr size_t kBwdSmem = sizeof(float) * (6 * kInH * kLd + 3 * kInH * kHd);
    static bool smem_set = false;
    if (!smem_set) {
        if (cudaFuncSetAttribute(k_ssim_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_ssim_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem) != cudaSuccess)
            return ODGS_ERR_CUDA;
        smem_set = true;
    }
    k_ssim_fwd<<<grid, kThreads, kFwdSmem, st>>>(a);
    k_loss_reduce<<<1, kThreads, 0, st>>>(a.partial, blocks_for(width, height), loss, p->accumulate ? 1 : 0);
    if (grad) k_ssim_bwd<<<grid, kThreads, kBwdSmem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? ODGS_OK : ODGS_ERR_CUDA;
}
