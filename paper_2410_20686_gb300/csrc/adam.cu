// Fused Adam step over the Gaussian parameter groups (sm_103a). Streams p, g, m, v once and
// writes p, m, v: 28 bytes per parameter, so the kernel is bound by HBM; 16-byte accesses where
// the arrays allow them, one launch for all groups (blockIdx.y picks the group).
#include <cuda_runtime.h>

#include <cmath>

#include "odgs_train.h"

namespace {

constexpr int kThreads = 256;

struct AdamTable {
    float* p[ODGS_ADAM_MAX_GROUPS];
    const float* g[ODGS_ADAM_MAX_GROUPS];
    float* m[ODGS_ADAM_MAX_GROUPS];
    float* v[ODGS_ADAM_MAX_GROUPS];
    unsigned long long count[ODGS_ADAM_MAX_GROUPS];
    float step_head[ODGS_ADAM_MAX_GROUPS], step_tail[ODGS_ADAM_MAX_GROUPS];  // lr / (1 - b1^t)
    int row[ODGS_ADAM_MAX_GROUPS], head[ODGS_ADAM_MAX_GROUPS];
    int vec[ODGS_ADAM_MAX_GROUPS];  // 16-byte accesses possible
    float b1, b2, omb1, omb2, eps, inv_sqrt_bc2;
};

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float step, const AdamTable& t) {
    m = fmaf(t.b1, m, t.omb1 * g);
    v = fmaf(t.b2, v, t.omb2 * g * g);
    p -= step * m / fmaf(sqrtf(v), t.inv_sqrt_bc2, t.eps);
}

__global__ void __launch_bounds__(kThreads) k_adam(AdamTable t) {
    const int grp = blockIdx.y;
    const unsigned long long n = t.count[grp];
    const int row = t.row[grp], head = t.head[grp];
    const float sh = t.step_head[grp], st = t.step_tail[grp];
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    float* __restrict__ P = t.p[grp];
    const float* __restrict__ G = t.g[grp];
    float* __restrict__ M = t.m[grp];
    float* __restrict__ V = t.v[grp];
    if (t.vec[grp]) {
        const unsigned long long n4 = n / 4;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 p = reinterpret_cast<float4*>(P)[i];
            const float4 g = reinterpret_cast<const float4*>(G)[i];
            float4 m = reinterpret_cast<float4*>(M)[i];
            float4 v = reinterpret_cast<float4*>(V)[i];
            const unsigned long long j = 4 * i;
            const int r0 = (int)(j % (unsigned long long)row);
            float s[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int r = r0 + k;  // position of element j + k in its row (rows may be shorter than 4)
                while (r >= row) r -= row;
                s[k] = r < head ? sh : st;
            }
            adam_one(p.x, g.x, m.x, v.x, s[0], t);
            adam_one(p.y, g.y, m.y, v.y, s[1], t);
            adam_one(p.z, g.z, m.z, v.z, s[2], t);
            adam_one(p.w, g.w, m.w, v.w, s[3], t);
            reinterpret_cast<float4*>(P)[i] = p;
            reinterpret_cast<float4*>(M)[i] = m;
            reinterpret_cast<float4*>(V)[i] = v;
        }
    } else {
        for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
            float p = P[j], m = M[j], v = V[j];
            adam_one(p, G[j], m, v, (int)(j % (unsigned long long)row) < head ? sh : st, t);
            P[j] = p;
            M[j] = m;
            V[j] = v;
        }
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" odgs_status odgs_adam_step(const odgs_adam_group* groups, int n_groups, const odgs_adam_params* prm,
                                      void* stream) {
    if (!groups || !prm || n_groups < 1 || n_groups > ODGS_ADAM_MAX_GROUPS || prm->step < 1) return ODGS_ERR_INVALID_ARG;
    if (!(prm->beta1 >= 0.0 && prm->beta1 < 1.0) || !(prm->beta2 >= 0.0 && prm->beta2 < 1.0) || !(prm->eps >= 0.0))
        return ODGS_ERR_INVALID_ARG;
    AdamTable t{};
    const double bc1 = 1.0 - std::pow(prm->beta1, (double)prm->step);
    const double bc2 = 1.0 - std::pow(prm->beta2, (double)prm->step);
    if (!(bc1 > 0.0) || !(bc2 > 0.0)) return ODGS_ERR_INVALID_ARG;
    size_t most = 0;
    for (int k = 0; k < n_groups; ++k) {
        const odgs_adam_group& g = groups[k];
        if (g.row < 1 || g.head < 0 || g.head > g.row) return ODGS_ERR_INVALID_ARG;
        if (g.count > 0 && (!g.param || !g.grad || !g.m || !g.v)) return ODGS_ERR_INVALID_ARG;
        t.p[k] = g.param; t.g[k] = g.grad; t.m[k] = g.m; t.v[k] = g.v;
        t.count[k] = g.count;
        t.step_head[k] = (float)((double)g.lr / bc1);
        t.step_tail[k] = (float)((double)g.lr_tail / bc1);
        t.row[k] = g.row;
        t.head[k] = g.head;
        t.vec[k] = g.count % 4 == 0 && aligned16(g.param) && aligned16(g.grad) && aligned16(g.m) && aligned16(g.v);
        most = g.count > most ? g.count : most;
    }
    if (most == 0) return ODGS_OK;
    t.b1 = (float)prm->beta1;
    t.b2 = (float)prm->beta2;
    t.omb1 = (float)(1.0 - prm->beta1);
    t.omb2 = (float)(1.0 - prm->beta2);
    t.eps = (float)prm->eps;
    t.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ODGS_ERR_CUDA;
    const unsigned long long want = (most / 4 + kThreads - 1) / kThreads;
    const unsigned int gx = (unsigned int)std::min<unsigned long long>(std::max<unsigned long long>(want, 1ull),
                                                                       (unsigned long long)sms * 8ull);
    k_adam<<<dim3(gx, (unsigned)n_groups), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(t);
    return cudaGetLastError() == cudaSuccess ? ODGS_OK : ODGS_ERR_CUDA;
}
