// L1 + D-SSIM loss of 3DGS training on ERP images, forward and gradient (sm_103a).
//
// SSIM_mean = sum_q c_q s_q with c_q the pixel's weight (cos(theta) of its row, or 1) over the
// weight of all 3 W H values, and s_q = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sxx + syy + C2))
// from window moments mx = g * x, sxx = g * x^2 - mx^2, sxy = g * xy - mx my (g: the separable
// 11-tap Gaussian). Because every moment is a correlation with g, which is symmetric,
//   dSSIM_mean / dx_p = (g * A)_p + 2 x_p (g * B)_p + y_p (g * C)_p,
//   A = c (ds/dmx - 2 mx ds/dsxx - my ds/dsxy),  B = c ds/dsxx,  C = c ds/dsxy.
//   k_ssim_fwd    per 32 x 16 tile and channel: the image and target with a 5-pixel halo in shared
//                 memory, a horizontal then a vertical 11-tap pass for the five moments, then s,
//                 the loss partial and the maps A, B, C (scratch)
//   k_ssim_bwd    the same tiling over A, B, C: two passes, then the gradient with the L1 term
//   k_loss_reduce one CTA: the CTAs' partials in a fixed order (deterministic)
// Rows outside the image are zero (zero padding); columns wrap around the seam or are zero.
#include <cuda_runtime.h>

#include <cmath>

#include "odgs_train.h"

namespace {

constexpr int kR = 5;
constexpr int kWin = 2 * kR + 1;
constexpr int kTX = 32, kTY = 16;
constexpr int kInW = kTX + 2 * kR, kInH = kTY + 2 * kR;
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

// Loads rows [y0 - kR, y0 + kTY + kR) x columns [x0 - kR, x0 + kTX + kR) of src into dst.
__device__ __forceinline__ void load_halo(const LossArgs& a, const float* __restrict__ src, float (*dst)[kInW], int x0,
                                          int y0) {
    for (int i = threadIdx.x; i < kInH * kInW; i += kThreads) {
        const int r = i / kInW, q = i - r * kInW;
        const int gy = y0 + r - kR;
        int gx = x0 + q - kR;
        float v = 0.f;
        if (gy >= 0 && gy < a.H) {
            if (a.wrap) {
                gx %= a.W;
                if (gx < 0) gx += a.W;
                v = src[(size_t)gy * a.W + gx];
            } else if (gx >= 0 && gx < a.W) {
                v = src[(size_t)gy * a.W + gx];
            }
        }
        dst[r][q] = v;
    }
}

__device__ __forceinline__ float block_sum(float v, float* s_red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
    return t;
}

__global__ void __launch_bounds__(kThreads) k_ssim_fwd(LossArgs a) {
    __shared__ float s_x[kInH][kInW], s_y[kInH][kInW];
    __shared__ float s_h[5][kInH][kTX];
    __shared__ float s_red[kThreads / 32];
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const size_t HW = (size_t)a.W * a.H;
    float part = 0.f;
    for (int c = 0; c < 3; ++c) {
        load_halo(a, a.x + c * HW, s_x, x0, y0);
        load_halo(a, a.y + c * HW, s_y, x0, y0);
        __syncthreads();
        for (int i = threadIdx.x; i < kInH * kTX; i += kThreads) {
            const int r = i / kTX, q = i - r * kTX;
            float hx = 0.f, hy = 0.f, hxx = 0.f, hyy = 0.f, hxy = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float xv = s_x[r][q + k], yv = s_y[r][q + k], gk = a.g[k];
                hx = fmaf(gk, xv, hx);
                hy = fmaf(gk, yv, hy);
                hxx = fmaf(gk, xv * xv, hxx);
                hyy = fmaf(gk, yv * yv, hyy);
                hxy = fmaf(gk, xv * yv, hxy);
            }
            s_h[0][r][q] = hx; s_h[1][r][q] = hy; s_h[2][r][q] = hxx; s_h[3][r][q] = hyy; s_h[4][r][q] = hxy;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTY * kTX; i += kThreads) {
            const int r = i / kTX, q = i - r * kTX;
            const int gy = y0 + r, gx = x0 + q;
            float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float gk = a.g[k];
                mx = fmaf(gk, s_h[0][r + k][q], mx);
                my = fmaf(gk, s_h[1][r + k][q], my);
                exx = fmaf(gk, s_h[2][r + k][q], exx);
                eyy = fmaf(gk, s_h[3][r + k][q], eyy);
                exy = fmaf(gk, s_h[4][r + k][q], exy);
            }
            if (gy >= a.H || gx >= a.W) continue;
            const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
            const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
            const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
            const float iB1 = 1.f / B1, iB2 = 1.f / B2;
            const float s = A1 * A2 * iB1 * iB2;
            const float ds_dmx = 2.f * A2 * (my * B1 - mx * A1) * iB1 * iB1 * iB2;
            const float ds_dsxx = -s * iB2;
            const float ds_dsxy = 2.f * A1 * iB1 * iB2;
            const float xv = s_x[r + kR][q + kR], yv = s_y[r + kR][q + kR];
            const float w = row_weight(a, gy) * a.inv_wsum;
            part = fmaf(w, (1.f - a.lam) * fabsf(xv - yv) + a.lam * (1.f - s), part);
            float* m = a.maps + (size_t)(3 * c) * HW + (size_t)gy * a.W + gx;
            m[0] = w * (ds_dmx - 2.f * mx * ds_dsxx - my * ds_dsxy);
            m[HW] = w * ds_dsxx;
            m[2 * HW] = w * ds_dsxy;
        }
        __syncthreads();  // the next channel overwrites the tiles
    }
    const float t = block_sum(part, s_red);
    if (threadIdx.x == 0) a.partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads) k_ssim_bwd(LossArgs a) {
    __shared__ float s_m[3][kInH][kInW];
    __shared__ float s_h[3][kInH][kTX];
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const size_t HW = (size_t)a.W * a.H;
    for (int c = 0; c < 3; ++c) {
        for (int k = 0; k < 3; ++k) load_halo(a, a.maps + (size_t)(3 * c + k) * HW, s_m[k], x0, y0);
        __syncthreads();
        for (int i = threadIdx.x; i < kInH * kTX; i += kThreads) {
            const int r = i / kTX, q = i - r * kTX;
            float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float gk = a.g[k];
                h0 = fmaf(gk, s_m[0][r][q + k], h0);
                h1 = fmaf(gk, s_m[1][r][q + k], h1);
                h2 = fmaf(gk, s_m[2][r][q + k], h2);
            }
            s_h[0][r][q] = h0; s_h[1][r][q] = h1; s_h[2][r][q] = h2;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTY * kTX; i += kThreads) {
            const int r = i / kTX, q = i - r * kTX;
            const int gy = y0 + r, gx = x0 + q;
            if (gy >= a.H || gx >= a.W) continue;
            float ga = 0.f, gb = 0.f, gc = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const float gk = a.g[k];
                ga = fmaf(gk, s_h[0][r + k][q], ga);
                gb = fmaf(gk, s_h[1][r + k][q], gb);
                gc = fmaf(gk, s_h[2][r + k][q], gc);
            }
            const size_t pix = c * HW + (size_t)gy * a.W + gx;
            const float xv = a.x[pix], yv = a.y[pix];
            const float d = xv - yv;
            const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            const float w = row_weight(a, gy) * a.inv_wsum;
            a.grad[pix] = (1.f - a.lam) * w * sgn - a.lam * (ga + 2.f * xv * gb + yv * gc);
        }
        __syncthreads();
    }
}

// lambda = 0: the weighted L1 term alone, one pass over the pixels (no window): the loss partial
// of each CTA and the gradient w sign(x - y) / (weight sum).
__global__ void __launch_bounds__(kThreads) k_l1(LossArgs a) {
    __shared__ float s_red[kThreads / 32];
    float part = 0.f;
    for (int rc = blockIdx.x; rc < 3 * a.H; rc += gridDim.x) {  // (channel, row) pairs
        const int row = rc % a.H;
        const float w = row_weight(a, row) * a.inv_wsum;
        const size_t base = (size_t)rc * a.W;
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
    k_ssim_fwd<<<grid, kThreads, 0, st>>>(a);
    k_loss_reduce<<<1, kThreads, 0, st>>>(a.partial, blocks_for(width, height), loss, p->accumulate ? 1 : 0);
    if (grad) k_ssim_bwd<<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? ODGS_OK : ODGS_ERR_CUDA;
}
