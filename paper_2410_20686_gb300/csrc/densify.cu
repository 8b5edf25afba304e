// Densification of ODGS (Sec. 3.3, App. A.1) on the GPU (sm_103a).
//
//   k_densify_select     one thread per Gaussian: the elevation-dependent threshold applied to
//                        the statistics that the backward preprocess accumulated
//   k_apply_count        per tile of 1024 Gaussians: how many are kept, cloned, split
//   k_apply_scan         one CTA: exclusive offsets of the tiles and the totals
//   k_apply_scatter      per tile again: each Gaussian's output slots (block scan + tile
//                        offset), then its copies / children (all but the SH rows) and the
//                        source index of every slot
//   k_apply_sh           the SH rows, slot by slot in 16-byte chunks (coalesced)
// Each step streams its arrays once; densification runs every few hundred iterations, so the
// point is to keep the parameters on the device, not to reach the copy bandwidth.
#include <cuda_runtime.h>

#include <cmath>

#include "odgs_common.cuh"
#include "odgs_train.h"

namespace odgs {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;
constexpr int kTile = kThreads * kPerThread;
constexpr float kLog1p6 = 0.470003629245735553650937f;  // ln 1.6: log-scale of a split child

__global__ void __launch_bounds__(kThreads) k_densify_select(const float* __restrict__ grad,
                                                             const float* __restrict__ elev,
                                                             const uint32_t* __restrict__ count,
                                                             const float* __restrict__ scales,
                                                             const float* __restrict__ opacity, int n,
                                                             odgs_densify_params p, float big_thr, float op_thr,
                                                             float max_thr, uint8_t* __restrict__ action) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = count[i];
    float gmean = 0.f, emean = 0.f;
    if (c > 0u) {
        const float fc = __uint2float_rn(c);
        gmean = __fdiv_rn(grad[i], fc);
        emean = __fdiv_rn(elev[i], fc);
    }
    // Sec. 3.3: tau = tau_min + (1 - cos theta)(tau_max - tau_min), with the views' mean of 1 - cos theta
    const float tau = __fadd_rn(p.tau_min, __fmul_rn(emean, __fsub_rn(p.tau_max, p.tau_min)));
    const bool hot = c > 0u && gmean >= tau;
    const float smax = fmaxf(fmaxf(scales[3 * i], scales[3 * i + 1]), scales[3 * i + 2]);
    // thresholds in the space of the inputs (activated, or log-scale / logit), set by the host
    const bool big = smax > big_thr;
    const bool prune = opacity[i] < op_thr || smax > max_thr;
    action[i] = (uint8_t)(prune ? ODGS_PRUNE : hot ? (big ? ODGS_SPLIT : ODGS_CLONE) : ODGS_KEEP);
}

// (kept, cloned, split) indicator of one action
__device__ __forceinline__ uint3 classes(uint8_t a) {
    return make_uint3(a == ODGS_KEEP || a == ODGS_CLONE, a == ODGS_CLONE, a == ODGS_SPLIT);
}

__device__ __forceinline__ uint3 add3(uint3 a, uint3 b) { return make_uint3(a.x + b.x, a.y + b.y, a.z + b.z); }

// Exclusive block scan of one uint3 per thread (kThreads threads); also returns the block total.
__device__ __forceinline__ uint3 block_scan3(uint3 v, uint3* s_warp, uint3& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint3 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint3 y = make_uint3(__shfl_up_sync(0xffffffffu, x.x, o), __shfl_up_sync(0xffffffffu, x.y, o),
                                   __shfl_up_sync(0xffffffffu, x.z, o));
        if (lane >= o) x = add3(x, y);
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    uint3 pre = make_uint3(0u, 0u, 0u), tot = make_uint3(0u, 0u, 0u);
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) {
        if (k < w) pre = add3(pre, s_warp[k]);
        tot = add3(tot, s_warp[k]);
    }
    __syncthreads();
    total = tot;
    return make_uint3(pre.x + x.x - v.x, pre.y + x.y - v.y, pre.z + x.z - v.z);
}

__global__ void __launch_bounds__(kThreads) k_apply_count(const uint8_t* __restrict__ action, int n,
                                                          uint4* __restrict__ tile_counts) {
    __shared__ uint3 s_warp[kThreads / 32];
    const int base = blockIdx.x * kTile + threadIdx.x * kPerThread;
    uint3 c = make_uint3(0u, 0u, 0u);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k)
        if (base + k < n) c = add3(c, classes(action[base + k]));
    uint3 tot;
    block_scan3(c, s_warp, tot);
    if (threadIdx.x == 0) tile_counts[blockIdx.x] = make_uint4(tot.x, tot.y, tot.z, 0u);
}

// One CTA of 1024 threads: exclusive scan of the tile counts; totals = (K, C, S, K + C + 2S).
__global__ void __launch_bounds__(1024) k_apply_scan(const uint4* __restrict__ tile_counts, int tiles,
                                                     uint4* __restrict__ tile_offsets, uint4* __restrict__ totals,
                                                     uint32_t* __restrict__ n_out) {
    __shared__ uint3 s_warp[32];
    __shared__ uint3 s_carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = make_uint3(0u, 0u, 0u);
    __syncthreads();
    for (int b = 0; b < tiles; b += 1024) {
        const int t = b + threadIdx.x;
        const uint4 c4 = t < tiles ? tile_counts[t] : make_uint4(0u, 0u, 0u, 0u);
        const uint3 v = make_uint3(c4.x, c4.y, c4.z);
        uint3 x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint3 y = make_uint3(__shfl_up_sync(0xffffffffu, x.x, o), __shfl_up_sync(0xffffffffu, x.y, o),
                                       __shfl_up_sync(0xffffffffu, x.z, o));
            if (lane >= o) x = add3(x, y);
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        uint3 pre = s_carry, tot = s_carry;
        for (int k = 0; k < 32; ++k) {
            if (k < w) pre = add3(pre, s_warp[k]);
            tot = add3(tot, s_warp[k]);
        }
        if (t < tiles) tile_offsets[t] = make_uint4(pre.x + x.x - v.x, pre.y + x.y - v.y, pre.z + x.z - v.z, 0u);
        __syncthreads();
        if (threadIdx.x == 0) s_carry = tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint3 t = s_carry;
        *totals = make_uint4(t.x, t.y, t.z, t.x + t.y + 2u * t.z);
        *n_out = t.x + t.y + 2u * t.z;
    }
}

struct ApplyArgs {
    const float *means, *scales, *quats, *opacity, *sh;
    int n, sh_coeffs;
    const uint8_t* action;
    const float* noise;
    float *o_means, *o_scales, *o_quats, *o_opacity, *o_sh;
    uint32_t cap;
    const uint4* tile_offsets;
    const uint4* totals;
    uint32_t* src;  // [cap] source Gaussian of every output slot
    int raw;        // scales are log-scales
};

// Copies Gaussian i into slot d (d < cap); child >= 0 places it as that split child.
__device__ __forceinline__ void write_gaussian(const ApplyArgs& a, int i, uint32_t d, int child) {
    if (d >= a.cap) return;
    const float4 q = *reinterpret_cast<const float4*>(a.quats + 4 * (size_t)i);
    float m[3] = {a.means[3 * i], a.means[3 * i + 1], a.means[3 * i + 2]};
    float s[3] = {a.scales[3 * i], a.scales[3 * i + 1], a.scales[3 * i + 2]};
    if (child >= 0) {
        if (a.raw) {  // the child's offset uses the activated scales
#pragma unroll
            for (int r = 0; r < 3; ++r) s[r] = expf(s[r]);
        }
        const float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        float R[9];
        quat_rot(q.x / qn, q.y / qn, q.z / qn, q.w / qn, R);
        const float* z = a.noise + 6 * (size_t)i + 3 * child;
        const float sz[3] = {s[0] * z[0], s[1] * z[1], s[2] * z[2]};
#pragma unroll
        for (int r = 0; r < 3; ++r) m[r] += R[3 * r] * sz[0] + R[3 * r + 1] * sz[1] + R[3 * r + 2] * sz[2];
        if (a.raw) {
#pragma unroll
            for (int r = 0; r < 3; ++r) s[r] = __fsub_rn(a.scales[3 * i + r], kLog1p6);
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r) s[r] = __fdiv_rn(s[r], 1.6f);
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        a.o_means[3 * (size_t)d + r] = m[r];
        a.o_scales[3 * (size_t)d + r] = s[r];
    }
    *reinterpret_cast<float4*>(a.o_quats + 4 * (size_t)d) = q;
    a.o_opacity[d] = a.opacity[i];
    a.src[d] = (uint32_t)i;
}

// SH rows of all output slots: thread t copies 16-byte chunk t % chunks of slot t / chunks (or
// single floats when the rows are not 16-byte multiples).
__global__ void __launch_bounds__(kThreads) k_apply_sh(const float* __restrict__ sh, float* __restrict__ o_sh,
                                                       const uint32_t* __restrict__ src, const uint4* __restrict__ totals,
                                                       uint32_t cap, int sh_coeffs) {
    const uint32_t slots = min(totals->w, cap);
    const int ns = 3 * sh_coeffs;
    const bool vec = (ns % 4) == 0 && (reinterpret_cast<uintptr_t>(sh) % 16) == 0 &&
                     (reinterpret_cast<uintptr_t>(o_sh) % 16) == 0;
    const int chunks = vec ? ns / 4 : ns;
    const size_t total = (size_t)slots * chunks;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t d = t / chunks;
        const int c = (int)(t - d * chunks);
        const size_t i = src[d];
        if (vec)
            reinterpret_cast<float4*>(o_sh + d * ns)[c] = reinterpret_cast<const float4*>(sh + i * ns)[c];
        else
            o_sh[d * ns + c] = sh[i * ns + c];
    }
}

__global__ void __launch_bounds__(kThreads) k_apply_scatter(ApplyArgs a) {
    __shared__ uint3 s_warp[kThreads / 32];
    const int base = blockIdx.x * kTile + threadIdx.x * kPerThread;
    uint8_t act[kPerThread];
    uint3 c = make_uint3(0u, 0u, 0u);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        act[k] = base + k < a.n ? a.action[base + k] : (uint8_t)ODGS_PRUNE;
        c = add3(c, classes(act[k]));
    }
    uint3 tot;
    uint3 off = block_scan3(c, s_warp, tot);
    const uint4 to = a.tile_offsets[blockIdx.x];
    const uint4 T = *a.totals;
    off = add3(off, make_uint3(to.x, to.y, to.z));
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int i = base + k;
        if (i >= a.n) break;
        const uint3 cl = classes(act[k]);
        if (cl.x) write_gaussian(a, i, off.x, -1);
        if (cl.y) write_gaussian(a, i, T.x + off.y, -1);
        if (cl.z) {
            write_gaussian(a, i, T.x + T.y + off.z, 0);
            write_gaussian(a, i, T.x + T.y + T.z + off.z, 1);
        }
        off = add3(off, cl);
    }
}

size_t tiles_for(int n) { return (size_t)((n + kTile - 1) / kTile); }
// tile counts and offsets, the totals, and the source index of up to 2n output slots
size_t scratch_bytes_for(int n) { return (2 * tiles_for(n) + 1) * sizeof(uint4) + 2 * (size_t)n * sizeof(uint32_t); }

}  // namespace
}  // namespace odgs

using namespace odgs;

extern "C" odgs_status odgs_densify_select(const float* grad, const float* elev, const uint32_t* count,
                                           const float* scales, const float* opacity, int n,
                                           const odgs_densify_params* p, uint8_t* action, void* stream) {
    if (n < 0 || !p) return ODGS_ERR_INVALID_ARG;
    if (n == 0) return ODGS_OK;
    if (!grad || !elev || !count || !scales || !opacity || !action) return ODGS_ERR_INVALID_ARG;
    if (!(p->scene_extent > 0.f) || !(p->tau_max >= p->tau_min) || p->max_scale < 0.f) return ODGS_ERR_INVALID_ARG;
    if (p->raw_params != 0 && p->raw_params != 1) return ODGS_ERR_INVALID_ARG;
    if (!(p->min_opacity >= 0.f && p->min_opacity < 1.f)) return ODGS_ERR_INVALID_ARG;
    const float inf = INFINITY;
    float big_thr, op_thr, max_thr;
    if (p->raw_params) {
        big_thr = (float)std::log((double)p->percent_dense * (double)p->scene_extent);
        op_thr = p->min_opacity > 0.f ? (float)std::log((double)p->min_opacity / (1.0 - (double)p->min_opacity)) : -inf;
        max_thr = p->max_scale > 0.f ? (float)std::log((double)p->max_scale) : inf;
    } else {
        big_thr = p->percent_dense * p->scene_extent;  // one float product, as the oracle takes it
        op_thr = p->min_opacity;
        max_thr = p->max_scale > 0.f ? p->max_scale : inf;
    }
    k_densify_select<<<(n + kThreads - 1) / kThreads, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        grad, elev, count, scales, opacity, n, *p, big_thr, op_thr, max_thr, action);
    return cudaGetLastError() == cudaSuccess ? ODGS_OK : ODGS_ERR_CUDA;
}

extern "C" odgs_status odgs_densify_scratch_size(int n, size_t* bytes) {
    if (n < 0 || !bytes) return ODGS_ERR_INVALID_ARG;
    *bytes = scratch_bytes_for(n);
    return ODGS_OK;
}

extern "C" odgs_status odgs_densify_apply(const odgs_gaussians* in, int sh_coeffs, int raw_params,
                                          const uint8_t* action, const float* noise, const odgs_params_out* out,
                                          int out_capacity, uint32_t* n_out, void* scratch, size_t scratch_bytes,
                                          void* stream) {
    if (!in || !out || !n_out || in->n < 0 || sh_coeffs < 1 || out_capacity < 0) return ODGS_ERR_INVALID_ARG;
    if (raw_params != 0 && raw_params != 1) return ODGS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = in->n;
    if (n == 0) return cudaMemsetAsync(n_out, 0, sizeof(uint32_t), st) == cudaSuccess ? ODGS_OK : ODGS_ERR_CUDA;
    if (!in->means || !in->scales || !in->quats || !in->opacity || !in->sh || !action || !noise) return ODGS_ERR_INVALID_ARG;
    if (!out->means || !out->scales || !out->quats || !out->opacity || !out->sh) return ODGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(in->quats) % 16 || reinterpret_cast<uintptr_t>(out->quats) % 16)
        return ODGS_ERR_INVALID_ARG;
    if (!scratch || reinterpret_cast<uintptr_t>(scratch) % 16 || scratch_bytes < scratch_bytes_for(n))
        return ODGS_ERR_WORKSPACE;
    const int tiles = (int)tiles_for(n);
    uint4* tile_counts = static_cast<uint4*>(scratch);
    uint4* tile_offsets = tile_counts + tiles;
    uint4* totals = tile_offsets + tiles;
    uint32_t* src = reinterpret_cast<uint32_t*>(totals + 1);
    const uint32_t cap = (uint32_t)min((long long)out_capacity, 2ll * n);  // at most 2 outputs each
    k_apply_count<<<tiles, kThreads, 0, st>>>(action, n, tile_counts);
    k_apply_scan<<<1, 1024, 0, st>>>(tile_counts, tiles, tile_offsets, totals, n_out);
    ApplyArgs a{};
    a.means = in->means; a.scales = in->scales; a.quats = in->quats; a.opacity = in->opacity; a.sh = in->sh;
    a.n = n; a.sh_coeffs = sh_coeffs; a.action = action; a.noise = noise;
    a.o_means = out->means; a.o_scales = out->scales; a.o_quats = out->quats; a.o_opacity = out->opacity;
    a.o_sh = out->sh; a.cap = cap; a.tile_offsets = tile_offsets; a.totals = totals; a.src = src;
    a.raw = raw_params;
    k_apply_scatter<<<tiles, kThreads, 0, st>>>(a);
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ODGS_ERR_CUDA;
    k_apply_sh<<<sms * 8, kThreads, 0, st>>>(in->sh, out->sh, src, totals, cap, sh_coeffs);
    return cudaGetLastError() == cudaSuccess ? ODGS_OK : ODGS_ERR_CUDA;
}
