// Per-Gaussian kernels of the ODGS ERP rasterizer (sm_103a):
//   k_setup                per-view tables (pixel-centre cos/sin in float-float), header reset
//   k_preprocess_geom      forward projection per (Gaussian, view): Sec. 3.1-3.2, Eq. 4-8
//   k_preprocess_color     SH colour per visible (Gaussian, view); digit histograms of the depth keys
//   k_preprocess_bwd       chain rule from screen-space gradients to the parameters: App. A.3
// The forward's geometry and colour halves are separate kernels so that the geometry does not
// carry the 48 SH coefficients in registers. The backward stays one kernel: split, it would read
// the screen-space accumulators and the means twice, which measured slower.
// The per-Gaussian kernels read each Gaussian's parameters once and loop over the views in
// registers, so a batch of V views costs one parameter read (HBM-bound for SH degree 3).
#include "odgs_common.cuh"
#include "odgs_internal.h"

namespace odgs {

// ------------------------------------------------------------------ setup

__global__ void k_setup(ViewTable tab, ViewDev* views, float4* trig, Header* hdr, int total_trig, uint32_t* dhist) {
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < tab.n_views) views[gid] = tab.v[gid];
    // the depth sort's digit histograms, counted by k_preprocess_geom
    for (int i = gid; i < 4 * 256; i += gridDim.x * blockDim.x) dhist[i] = 0u;
    if (gid == 0) {
        hdr->pairs = 0ull;
        hdr->pairs_emitted = 0ull;
        hdr->evals_fwd = 0ull;
        hdr->evals_bwd = 0ull;
        hdr->blended = 0ull;
        hdr->entries_tile = 0ull;
        hdr->visible = 0ull;
        hdr->status = 0u;
        hdr->n_items = tab.n_items;
        hdr->n_pairs_sort = 0u;
        hdr->work_fwd = 0u;
        hdr->work_bwd = 0u;
        hdr->n_big = 0u;
        hdr->n_count_big = 0u;  // the binning's queue counters (each binning leaves them at 0)
    }
    for (int e = gid; e < total_trig; e += gridDim.x * blockDim.x) {
        // locate the view and whether e is a column or a row entry
        int v = 0;
        while (v + 1 < tab.n_views && tab.v[v + 1].trig_u <= e) ++v;
        const ViewDev& V = tab.v[v];
        double c, s;
        if (e < V.trig_v) {
            // column centre azimuth phi0 = 2 pi (c0 + 0.5) / W - pi   (inverse of Eq. 4)
            int col = e - V.trig_u;
            sincospi(2.0 * (col + 0.5) / V.W - 1.0, &s, &c);
        } else {
            // row centre elevation theta0 = pi / 2 - pi (r0 + 0.5) / H  (inverse of Eq. 4)
            int row = e - V.trig_v;
            sincospi(0.5 - (row + 0.5) / V.H, &s, &c);
        }
        float ch = (float)c, sh = (float)s;
        trig[e] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
    }
}

// ------------------------------------------------------------------ shared math


// Real SH basis (orthonormal, no Condon-Shortley phase) as Cartesian polynomials of the unit
// direction (x, y, z); index l^2 + l + m.
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    Y[0] = 0.28209479177387814f;
    if (DEG >= 1) {
        const float c1 = 0.4886025119029199f;
        Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
    }
    if (DEG >= 2) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
        Y[4] = a * x * y; Y[5] = a * y * z; Y[6] = b * (3.f * z * z - 1.f); Y[7] = a * x * z;
        Y[8] = c * (x * x - y * y);
    }
    if (DEG >= 3) {
        const float a = 0.5900435899266435f, b = 2.890611442640554f, c = 0.4570457994644658f,
                    d = 0.3731763325901154f, e = 1.445305721320277f;
        Y[9] = a * y * (3.f * x * x - y * y);
        Y[10] = b * x * y * z;
        Y[11] = c * y * (5.f * z * z - 1.f);
        Y[12] = d * z * (5.f * z * z - 3.f);
        Y[13] = c * x * (5.f * z * z - 1.f);
        Y[14] = e * z * (x * x - y * y);
        Y[15] = a * x * (x * x - 3.f * y * y);
    }
}

// Gradient of the polynomials above w.r.t. (x, y, z), accumulated as sum_k w_k grad Y_k.
template <int DEG>
__device__ __forceinline__ void sh_grad_acc(float x, float y, float z, const float w[16], float& gx, float& gy,
                                            float& gz) {
    gx = gy = gz = 0.f;
    if (DEG >= 1) {
        const float c1 = 0.4886025119029199f;
        gy += c1 * w[1]; gz += c1 * w[2]; gx += c1 * w[3];
    }
    if (DEG >= 2) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
        gx += a * y * w[4]; gy += a * x * w[4];
        gy += a * z * w[5]; gz += a * y * w[5];
        gz += 6.f * b * z * w[6];
        gx += a * z * w[7]; gz += a * x * w[7];
        gx += 2.f * c * x * w[8]; gy -= 2.f * c * y * w[8];
    }
    if (DEG >= 3) {
        const float a = 0.5900435899266435f, b = 2.890611442640554f, c = 0.4570457994644658f,
                    d = 0.3731763325901154f, e = 1.445305721320277f;
        gx += 6.f * a * x * y * w[9]; gy += 3.f * a * (x * x - y * y) * w[9];
        gx += b * y * z * w[10]; gy += b * x * z * w[10]; gz += b * x * y * w[10];
        gy += c * (5.f * z * z - 1.f) * w[11]; gz += 10.f * c * y * z * w[11];
        gz += d * (15.f * z * z - 3.f) * w[12];
        gx += c * (5.f * z * z - 1.f) * w[13]; gz += 10.f * c * x * z * w[13];
        gx += 2.f * e * x * z * w[14]; gy -= 2.f * e * y * z * w[14]; gz += e * (x * x - y * y) * w[14];
        gx += 3.f * a * (x * x - y * y) * w[15]; gy -= 6.f * a * x * y * w[15];
    }
}

// Depth in IEEE single precision with the fixed operation order of the depth key:
// t_i = ((R_i0 m0 + R_i1 m1) + R_i2 m2) + t_i; ERP: r = sqrt((tx tx + ty ty) + tz tz), the radial
// distance; pinhole: tz, the z depth perspective 3DGS sorts by.
__device__ __forceinline__ float depth_key(const ViewDev& V, float m0, float m1, float m2) {
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float s = __fadd_rn(__fmul_rn(V.R[3 * i], m0), __fmul_rn(V.R[3 * i + 1], m1));
        s = __fadd_rn(s, __fmul_rn(V.R[3 * i + 2], m2));
        t[i] = __fadd_rn(s, V.t[i]);
    }
    if (V.model == 1) return t[2];
    float q = __fadd_rn(__fmul_rn(t[0], t[0]), __fmul_rn(t[1], t[1]));
    q = __fadd_rn(q, __fmul_rn(t[2], t[2]));
    return __fsqrt_rn(q);
}

// J_omni (Eq. 8) from the camera-space mean, written with sec(theta) = r / rho,
// cos(phi) = tz / rho, sin(phi) = tx / rho, sin(theta) = -ty / r, cos(theta) = rho / r:
//   row 1 = fx [tz, 0, -tx] / rho^2,  row 2 = fy [-tx ty / rho, rho, -ty tz / rho] / r^2.
struct JGeom {
    float J[6];
    float rho, rho2, r2;
};
__device__ __forceinline__ JGeom omni_jacobian(float tx, float ty, float tz, float fx, float fy) {
    JGeom g;
    g.rho2 = tx * tx + tz * tz;
    g.rho = sqrtf(g.rho2);
    g.r2 = g.rho2 + ty * ty;
    float a = fx / g.rho2;
    float b = fy / (g.r2 * g.rho);
    g.J[0] = a * tz; g.J[1] = 0.f; g.J[2] = -a * tx;
    g.J[3] = -b * tx * ty; g.J[4] = fy * g.rho / g.r2; g.J[5] = -b * ty * tz;
    return g;
}

// Perspective Jacobian of u = fx tx/tz + cx, v = fy ty/tz + cy (Eq. 1).
__device__ __forceinline__ void pinhole_jacobian(float tx, float ty, float tz, float fx, float fy, float J[6]) {
    const float iz = 1.f / tz;
    J[0] = fx * iz; J[1] = 0.f; J[2] = -fx * tx * iz * iz;
    J[3] = 0.f; J[4] = fy * iz; J[5] = -fy * ty * iz * iz;
}

// TM = (J W) M, the 2x3 factor of Sigma_2D = TM TM^T (+ dilation).
__device__ __forceinline__ void tm_factor(const float J[6], const float W[9], const float M[9], float T[6],
                                          float TM[6]) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            T[3 * i + k] = J[3 * i] * W[k] + J[3 * i + 1] * W[3 + k] + J[3 * i + 2] * W[6 + k];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            TM[3 * i + k] = T[3 * i] * M[k] + T[3 * i + 1] * M[3 + k] + T[3 * i + 2] * M[6 + k];
}

// Sigma_2D = TM TM^T + delta I and its determinant without cancellation:
// det(TM TM^T) = |TM_1 x TM_2|^2 (Lagrange's identity).
struct Cov2 {
    float A, B, C, det, A0, C0;
};
__device__ __forceinline__ Cov2 cov2d(const float TM[6], float delta) {
    Cov2 c;
    c.A0 = TM[0] * TM[0] + TM[1] * TM[1] + TM[2] * TM[2];
    c.C0 = TM[3] * TM[3] + TM[4] * TM[4] + TM[5] * TM[5];
    c.B = TM[0] * TM[3] + TM[1] * TM[4] + TM[2] * TM[5];
    float cx = TM[1] * TM[5] - TM[2] * TM[4];
    float cy = TM[2] * TM[3] - TM[0] * TM[5];
    float cz = TM[0] * TM[4] - TM[1] * TM[3];
    float det0 = cx * cx + cy * cy + cz * cz;
    c.A = c.A0 + delta;
    c.C = c.C0 + delta;
    c.det = det0 + delta * (c.A0 + c.C0) + delta * delta;
    return c;
}

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int DEG>
__device__ __forceinline__ void load_sh(const float* __restrict__ sh, int stride, int g, float c[16][3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float* p = sh + (size_t)g * stride * 3;
    if ((stride * 3) % 4 == 0) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
        float tmp[((K * 3 + 3) / 4) * 4];
#pragma unroll
        for (int i = 0; i < (K * 3 + 3) / 4; ++i) {
            float4 q = __ldg(p4 + i);
            tmp[4 * i] = q.x; tmp[4 * i + 1] = q.y; tmp[4 * i + 2] = q.z; tmp[4 * i + 3] = q.w;
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) c[k][ch] = tmp[3 * k + ch];
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) c[k][ch] = __ldg(p + 3 * k + ch);
    }
}

// ------------------------------------------------------------------ forward projection

// Footprints with at most this many row bands are counted by their own thread; larger ones (the
// pole-stretched Gaussians) by the whole warp, one band per lane.
constexpr int kThreadBands = 4;
static_assert(kThreadBands <= 6, "the per-thread loop stores the spans of six bands (rect, rect2)");

__global__ void __launch_bounds__(256, 3) k_preprocess_geom(PreArgs a) {
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    unsigned long long local_pairs = 0ull;
    uint32_t local_visible = 0u;
    // every lane of a warp runs the view loop (lanes past the end as culled items), so that the
    // warp can count the tiles of many-band footprints together
    const bool act = g0 < a.n;
    const int g = act ? g0 : 0;
    {
        const float m0 = __ldg(a.means + 3 * g), m1 = __ldg(a.means + 3 * g + 1), m2 = __ldg(a.means + 3 * g + 2);
        float s0 = __ldg(a.scales + 3 * g), s1 = __ldg(a.scales + 3 * g + 1), s2 = __ldg(a.scales + 3 * g + 2);
        const float4 q = __ldg(reinterpret_cast<const float4*>(a.quats) + g);
        float o = __ldg(a.opacity + g);
        if (a.st.raw) {
            s0 = expf(s0); s1 = expf(s1); s2 = expf(s2);
            o = sigmoid_act(o);
        }
        bool finite_in = true;  // checked mode: a Gaussian with a non-finite parameter is culled
        if (a.st.checked) {
            finite_in = isfinite(m0) && isfinite(m1) && isfinite(m2) && isfinite(s0) && isfinite(s1) &&
                        isfinite(s2) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w) && isfinite(o);
            const float* shg = a.sh + (size_t)g * 3 * a.sh_coeffs;
            for (int k = 0; k < 3 * a.sh_coeffs; ++k) finite_in = finite_in && isfinite(__ldg(shg + k));
            if (act && !finite_in) atomicOr(&a.hdr->status, kStNonfinite);
        }

        // Sigma = M M^T with M = R(q) S (Sec. 3.1)
        float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        float Rq[9], M[9];
        quat_rot(q.x / qn, q.y / qn, q.z / qn, q.w / qn, Rq);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            M[3 * i] = Rq[3 * i] * s0; M[3 * i + 1] = Rq[3 * i + 1] * s1; M[3 * i + 2] = Rq[3 * i + 2] * s2;
        }
        const float Qalpha = (255.f * o > 1.f) ? 2.f * logf(255.f * o) : -1.f;  // Mahalanobis^2 at alpha = 1/255
        const float Qb = Qalpha * (1.f + 1e-4f) + 1e-4f;

        for (int v = 0; v < a.n_views; ++v) {
            const ViewDev& V = a.views[v];
            const size_t item = (size_t)v * a.n + g;
            uint4 rect = make_uint4(0u, 0u, 0u, 0u);
            uint32_t key = 0xFFFFFFFFu;
            const float r = depth_key(V, m0, m1, m2);
            bool ok = act && finite_in && (r > a.st.r_near) && (r < a.st.r_far) && (Qalpha > 0.f);
            // camera-space mean in float-float: t = W mu + t_wc
            ff t[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ff acc = ff_add(two_prod(V.R[3 * i], m0), two_prod(V.R[3 * i + 1], m1));
                acc = ff_add(acc, two_prod(V.R[3 * i + 2], m2));
                t[i] = ff_add(acc, ff{V.t[i], 0.f});
            }
            const float tx = t[0].hi, ty = t[1].hi, tz = t[2].hi;
            float J[6];
            float du = 0.f, dv = 0.f;
            int c0 = 0, r0 = 0;
            if (V.model == 1) {
                // pinhole: u = fx tx/tz + cx (float-float), anchored at the pixel holding it;
                // centres outside the image widened by 30 % on each side are culled
                const ff uq = ff_add(ff{V.cx, 0.f}, ff_mulf(ff_div(t[0], t[2]), V.fx));
                const ff vq = ff_add(ff{V.cy, 0.f}, ff_mulf(ff_div(t[1], t[2]), V.fy));
                ok = ok && uq.hi >= -0.3f * V.W && uq.hi <= 1.3f * V.W && vq.hi >= -0.3f * V.H &&
                     vq.hi <= 1.3f * V.H;
                if (ok) {
                    c0 = (int)floorf(uq.hi);
                    r0 = (int)floorf(vq.hi);
                    du = __fadd_rn(__fsub_rn(__fsub_rn(uq.hi, (float)c0), 0.5f), uq.lo);
                    dv = __fadd_rn(__fsub_rn(__fsub_rn(vq.hi, (float)r0), 0.5f), vq.lo);
                    pinhole_jacobian(tx, ty, tz, V.fx, V.fy, J);
                }
            } else {
                JGeom jg = omni_jacobian(tx, ty, tz, V.fx, V.fy);
                ok = ok && (jg.rho > 1e-4f * r);  // too close to a pole: sec(theta) > 1e4
#pragma unroll
                for (int i = 0; i < 6; ++i) J[i] = jg.J[i];
            }
            if (ok && V.model == 0) {
                // ERP mean (Eq. 4) as pixel anchor + offset: rotate (t_x, t_z) by minus the
                // azimuth of the anchor column's centre, then the elevation likewise.
                float ua = atan2f(tx, tz) * V.fx + 0.5f * V.W;
                c0 = min(max((int)floorf(ua), 0), V.W - 1);
                float4 tu = a.trig[V.trig_u + c0];
                ff cph{tu.x, tu.y}, sph{tu.z, tu.w};
                ff ar = ff_add(ff_mul(t[0], cph), ff_neg(ff_mul(t[2], sph)));  // rho sin(phi - phi0)
                ff br = ff_add(ff_mul(t[0], sph), ff_mul(t[2], cph));          // rho cos(phi - phi0)
                du = atan2f(ar.hi, br.hi) * V.fx;
                ff rho = ff_sqrt(ff_add(ff_mul(ar, ar), ff_mul(br, br)));
                ff ny = ff_neg(t[1]);
                float va = -atan2f(ny.hi, rho.hi) * V.fy + 0.5f * V.H;
                r0 = min(max((int)floorf(va), 0), V.H - 1);
                float4 tv = a.trig[V.trig_v + r0];
                ff cth{tv.x, tv.y}, sth{tv.z, tv.w};
                ff ae = ff_add(ff_mul(ny, cth), ff_neg(ff_mul(rho, sth)));  // r sin(theta - theta0)
                ff be = ff_add(ff_mul(rho, cth), ff_mul(ny, sth));          // r cos(theta - theta0)
                dv = -atan2f(ae.hi, be.hi) * V.fy;
            }
            float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
            Footprint fp{};
            int jlo = 0, jhi = -1;
            if (ok) {
                // Sigma_2D = (J W M)(J W M)^T + delta I  (Eq. 8 and Sec. 3.1)
                float T[6], TM[6];
                tm_factor(J, V.R, M, T, TM);
                Cov2 c2 = cov2d(TM, a.st.dilation);
                if (c2.det > 0.f) {
                    float inv = 1.f / c2.det;
                    ra = make_float4(du, dv, pack_anchor(c0, r0), o);
                    // the conic in slice form (a, beta, gamma) = (C / det, B / C, 1 / C)
                    rb = make_float4(c2.C * inv, c2.B / c2.C, 1.f / c2.C, Qb);
                    fp = make_footprint(ra, rb);
                    footprint_rows(fp, V.H, jlo, jhi);
                }
            }
            // tiles met by the footprint, row band by row band (seam-wrapped columns)
            const bool cand = jlo <= jhi;
            const int th = a.st.tile_h;
            const int ty0 = cand ? jlo / th : 0, nb = cand ? jhi / th - ty0 + 1 : 0;
            uint32_t count = 0u, sp0 = 0u, sp1 = 0u, sp2 = 0u, sp3 = 0u, sp4 = 0u, sp5 = 0u;
            if (nb <= kThreadBands) {
                for (int b = 0; b < nb; ++b) {
                    const int ty = ty0 + b;
                    int st0, cnt;
                    band_columns(fp, max(jlo, ty * th), min(jhi, ty * th + th - 1), V.W, a.st.tile_w, V.tiles_x,
                                 V.model == 0, st0, cnt);
                    count += (uint32_t)cnt;
                    // spans of the first bands (scalars, so that they stay in registers)
                    const uint32_t sp = (uint32_t)st0 | ((uint32_t)cnt << 16);
                    sp0 = b == 0 ? sp : sp0; sp1 = b == 1 ? sp : sp1; sp2 = b == 2 ? sp : sp2;
                    sp3 = b == 3 ? sp : sp3; sp4 = b == 4 ? sp : sp4; sp5 = b == 5 ? sp : sp5;
                }
            }
            // footprints of many row bands (pole-stretched Gaussians cover up to all rows): the
            // warp counts each one's bands together, one band per lane, with the same band_columns
            // on the same floats, so that counts and spans are the per-thread loop's, bit for bit
            unsigned many = __ballot_sync(0xffffffffu, nb > kThreadBands);
            while (many) {
                const int src = __ffs(many) - 1;
                many &= many - 1u;
                Footprint f;
                f.c0 = __shfl_sync(0xffffffffu, fp.c0, src);
                f.r0 = __shfl_sync(0xffffffffu, fp.r0, src);
                f.du = __shfl_sync(0xffffffffu, fp.du, src);
                f.dv = __shfl_sync(0xffffffffu, fp.dv, src);
                f.BC = __shfl_sync(0xffffffffu, fp.BC, src);
                f.k = __shfl_sync(0xffffffffu, fp.k, src);
                f.iC = __shfl_sync(0xffffffffu, fp.iC, src);
                f.Qb = __shfl_sync(0xffffffffu, fp.Qb, src);
                f.ev = __shfl_sync(0xffffffffu, fp.ev, src);
                f.ystar = __shfl_sync(0xffffffffu, fp.ystar, src);
                const int wjlo = __shfl_sync(0xffffffffu, jlo, src), wjhi = __shfl_sync(0xffffffffu, jhi, src);
                const int wty0 = __shfl_sync(0xffffffffu, ty0, src), wnb = __shfl_sync(0xffffffffu, nb, src);
                uint32_t tot = 0u, w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u, w4 = 0u, w5 = 0u;
                for (int b0 = 0; b0 < wnb; b0 += 32) {
                    const int b = b0 + lane;
                    int st0 = 0, cnt = 0;
                    if (b < wnb) {
                        const int ty = wty0 + b;
                        band_columns(f, max(wjlo, ty * th), min(wjhi, ty * th + th - 1), V.W, a.st.tile_w,
                                     V.tiles_x, V.model == 0, st0, cnt);
                    }
                    uint32_t c = (uint32_t)cnt;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
                    tot += c;
                    if (b0 == 0) {
                        const uint32_t sp = (uint32_t)st0 | ((uint32_t)cnt << 16);
                        w0 = __shfl_sync(0xffffffffu, sp, 0); w1 = __shfl_sync(0xffffffffu, sp, 1);
                        w2 = __shfl_sync(0xffffffffu, sp, 2); w3 = __shfl_sync(0xffffffffu, sp, 3);
                        w4 = __shfl_sync(0xffffffffu, sp, 4); w5 = __shfl_sync(0xffffffffu, sp, 5);
                    }
                }
                if (lane == src) {
                    count = tot;
                    sp0 = w0; sp1 = w1; sp2 = w2; sp3 = w3; sp4 = w4; sp5 = w5;
                }
            }
            if (count > 0u) {
                rect = make_uint4((uint32_t)ty0 | ((uint32_t)nb << 16), count, sp0, sp1);
                if (nb > 2) a.rect2[item] = make_uint4(sp2, sp3, sp4, sp5);
                local_pairs += count;
                ++local_visible;
                key = __float_as_uint(r);
                a.rec_a[item] = ra;
                a.rec_b[item] = rb;
            }
            if (act) {
                if (key == 0xFFFFFFFFu) {
                    // culled: finite records that never pass the alpha test (opacity 0), so that an
                    // index that reaches the blend only through a sort that gave up reads no stale
                    // memory (the colour kernel writes rec_c of the visible items only)
                    a.rec_a[item] = make_float4(0.f, 0.f, 0.f, 0.f);
                    a.rec_b[item] = make_float4(1.f, 0.f, 1.f, 0.f);
                    a.rec_c[item] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                a.rect[item] = rect;
                a.dkey[item] = key;
                if (a.dbucket) a.dbucket[item] = (uint8_t)depth_bucket(key, a.cut_base);
                a.dval[item] = (uint32_t)item;
            }
        }
    }
    // frame pair and visible-item counts
    for (int off = 16; off > 0; off >>= 1) {
        local_pairs += __shfl_xor_sync(0xffffffffu, local_pairs, off);
        local_visible += __shfl_xor_sync(0xffffffffu, local_visible, off);
    }
    __shared__ unsigned long long s_sum[8];
    __shared__ uint32_t s_vis[8];
    if ((threadIdx.x & 31) == 0) {
        s_sum[threadIdx.x >> 5] = local_pairs;
        s_vis[threadIdx.x >> 5] = local_visible;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0ull, vis = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tot += s_sum[w];
            vis += s_vis[w];
        }
        if (tot) atomicAdd(&a.hdr->pairs, tot);
        if (vis) atomicAdd(&a.hdr->visible, vis);
    }
}

// View-dependent colour of every visible item: max(0, sum_k sh_k Y_k(d) + 0.5) with d the unit
// vector from the camera centre to the mean in world space. A separate streaming kernel, so the
// 48 SH coefficients do not weigh on the geometry kernel's registers.
template <int DEG>
__global__ void __launch_bounds__(256) k_preprocess_color(PreArgs a) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    // digit histograms of the depth keys for the depth sort (all items, culled ones included),
    // counted here, where every key is read anyway and the kernel waits on memory
    __shared__ uint32_t s_dh[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) s_dh[i >> 8][i & 255] = 0u;
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    for (int v = 0; v < a.n_views && g < a.n; ++v) {
        const uint32_t key = a.dkey[(size_t)v * a.n + g];
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_dh[p][(key >> (8 * p)) & 0xFFu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
        const uint32_t c = s_dh[i >> 8][i & 255];
        if (c) atomicAdd(a.dhist + i, c);
    }
    if (g >= a.n) return;
    const float m0 = __ldg(a.means + 3 * g), m1 = __ldg(a.means + 3 * g + 1), m2 = __ldg(a.means + 3 * g + 2);
    bool loaded = false;
    float shc[16][3];
    for (int v = 0; v < a.n_views; ++v) {
        const size_t item = (size_t)v * a.n + g;
        if (a.dkey[item] == 0xFFFFFFFFu) continue;  // culled in this view
        if (!loaded) { load_sh<DEG>(a.sh, a.sh_coeffs, g, shc); loaded = true; }
        const ViewDev& V = a.views[v];
        const float dx = m0 - V.cam[0], dy = m1 - V.cam[1], dz = m2 - V.cam[2];
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        float Y[16];
        sh_basis<DEG>(dx * il, dy * il, dz * il, Y);
        float rgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fmaf(shc[k][ch], Y[k], acc);
            rgb[ch] = fmaxf(acc, 0.f);
        }
        a.rec_c[item] = make_float4(rgb[0], rgb[1], rgb[2], 0.f);
    }
}

// ------------------------------------------------------------------ backward chain rule

// ONE: a frame of one view. Its colour phase reads the SH coefficient row twice (colours, then
// the direction's gradient) and forms dL/dsh = m_c dL/drgb_c Y_k when it writes them (m_c = 0 for
// a clamped channel), so neither the 48 coefficients nor 48 accumulators stay in registers.
// Frames of several views accumulate dL/dsh over the views in registers.
template <int DEG, bool ONE>
__global__ void __launch_bounds__(128) k_preprocess_bwd(PreBwdArgs a) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    const float m0 = __ldg(a.means + 3 * g), m1 = __ldg(a.means + 3 * g + 1), m2 = __ldg(a.means + 3 * g + 2);
    float s[3] = {__ldg(a.scales + 3 * g), __ldg(a.scales + 3 * g + 1), __ldg(a.scales + 3 * g + 2)};
    if (a.raw) {
#pragma unroll
        for (int i = 0; i < 3; ++i) s[i] = expf(s[i]);
    }
    const float4 q = __ldg(reinterpret_cast<const float4*>(a.quats) + g);

    float gm[3] = {0.f, 0.f, 0.f}, gop = 0.f;
    float dM[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) dM[i] = 0.f;

    float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float qw = q.x / qn, qx = q.y / qn, qy = q.z / qn, qz = q.w / qn;
    float Rq[9], M[9];
    quat_rot(qw, qx, qy, qz, Rq);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * s[j];

    bool any = false;
    // densification statistics of this Gaussian (Sec. 3.3): the running sums are loaded here, so
    // their latency overlaps the loop instead of ending every thread
    float st_grad = 0.f, st_elev = 0.f;
    uint32_t st_count = 0u;
    if (a.d_count) {
        st_grad = a.d_grad[g];
        st_elev = a.d_elev[g];
        st_count = a.d_count[g];
    }
    const uint32_t st_count0 = st_count;
    for (int v = 0; v < a.n_views; ++v) {
        const size_t item = (size_t)v * a.n + g;
        const float4 g0 = a.acc[3 * item], g1 = a.acc[3 * item + 1], g2 = a.acc[3 * item + 2];
        if (a.d_count && a.rect[item].y > 0u) {
            // visible in view v: ERP-mean gradient in [-1, 1] image units, and 1 - cos(theta)
            // as t_y^2 / (r (r + rho)), free of the cancellation of 1 - rho / r
            const ViewDev& V = a.views[v];
            float t[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) t[i] = V.R[3 * i] * m0 + V.R[3 * i + 1] * m1 + V.R[3 * i + 2] * m2 + V.t[i];
            const float rho = sqrtf(t[0] * t[0] + t[2] * t[2]);
            const float r = sqrtf(rho * rho + t[1] * t[1]);
            const float gu = g0.x * (0.5f * (float)V.W), gv = g0.y * (0.5f * (float)V.H);
            st_grad += sqrtf(gu * gu + gv * gv);
            st_elev += t[1] * t[1] / (r * (r + rho));
            ++st_count;
        }
        // accumulator layout: (du, dv, da, db), (dc, dopacity, dr, dg), (db, 0, 0, 0)
        if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
            g1.z == 0.f && g1.w == 0.f && g2.x == 0.f)
            continue;
        any = true;
        const ViewDev& V = a.views[v];
        const float* W = V.R;
        float t[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) t[i] = W[3 * i] * m0 + W[3 * i + 1] * m1 + W[3 * i + 2] * m2 + V.t[i];
        const float tx = t[0], ty = t[1], tz = t[2];
        const bool pin = V.model == 1;
        JGeom jg{};
        float Jm[6];
        if (pin) {
            pinhole_jacobian(tx, ty, tz, V.fx, V.fy, Jm);
        } else {
            jg = omni_jacobian(tx, ty, tz, V.fx, V.fy);
#pragma unroll
            for (int i = 0; i < 6; ++i) Jm[i] = jg.J[i];
        }
        float T[6], TM[6];
        tm_factor(Jm, W, M, T, TM);
        Cov2 c2 = cov2d(TM, a.dilation);
        // The blend's conic gradients are w.r.t. the slice form a = C / det, beta = B / C,
        // gamma = 1 / C of Sigma_2D = TM TM^T + delta I (A = |TM_1|^2 + delta, B = TM_1 . TM_2,
        // C = |TM_2|^2 + delta). With r = TM_1 - beta TM_2 and 1 / a = A - beta B:
        //   d(1/a)/dTM_1 = 2 r, d(1/a)/dTM_2 = -2 beta r, dbeta/dTM_1 = TM_2 / C,
        //   dbeta/dTM_2 = (TM_1 - 2 beta TM_2) / C, dgamma/dTM_2 = -2 gamma^2 TM_2, so
        //   dL/dTM_1 = ka r + kb TM_2,  dL/dTM_2 = -beta ka r + kb (r - beta TM_2) + kg TM_2
        // with ka = -2 a^2 dL/da, kb = gamma dL/dbeta, kg = -2 gamma^2 dL/dgamma. For a needle-like
        // Gaussian r (its thin row) is small: every term is a product with r or tau = T_1 - beta T_2,
        // never a difference of the long direction's terms, whose rounding would be about
        // cond(Sigma_2D) times the thin direction's gradient.
        const float ga = g0.z, gbeta = g0.w, ggam = g1.x;
        const float sa = c2.C * (1.f / c2.det), beta = c2.B / c2.C, gam = 1.f / c2.C;
        const float ka = -2.f * sa * sa * ga, kb = gam * gbeta, kg = -2.f * gam * gam * ggam;
        float r[3], tau[3], dTM1[3], dTM2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            r[k] = fmaf(-beta, TM[3 + k], TM[k]);
            tau[k] = fmaf(-beta, T[3 + k], T[k]);
            dTM1[k] = fmaf(ka, r[k], kb * TM[3 + k]);
            dTM2[k] = fmaf(-beta * ka, r[k], fmaf(kb, fmaf(-beta, TM[3 + k], r[k]), kg * TM[3 + k]));
        }
        // TM = T M: dM += T_1 (x) dTM_1 + T_2 (x) dTM_2, written with tau so that the r terms do not
        // cancel: dM = ka tau (x) r + kb (tau (x) TM_2 + T_2 (x) r) + kg T_2 (x) TM_2
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                dM[3 * j + k] += fmaf(ka * tau[j], r[k], fmaf(kb, fmaf(tau[j], TM[3 + k], T[3 + j] * r[k]),
                                                            kg * T[3 + j] * TM[3 + k]));
        // dT = dTM M^T, T = J W: dJ = dT W^T
        float dT1[3], dT2[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dT1[j] = dTM1[0] * M[3 * j] + dTM1[1] * M[3 * j + 1] + dTM1[2] * M[3 * j + 2];
            dT2[j] = dTM2[0] * M[3 * j] + dTM2[1] * M[3 * j + 1] + dTM2[2] * M[3 * j + 2];
        }
        float dJ[6];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dJ[j] = dT1[0] * W[3 * j] + dT1[1] * W[3 * j + 1] + dT1[2] * W[3 * j + 2];
            dJ[3 + j] = dT2[0] * W[3 * j] + dT2[1] * W[3 * j + 1] + dT2[2] * W[3 * j + 2];
        }
        // dL/dt: mean path d(u, v)/dt = J (Eq. 10 for ERP) plus J's dependence on t
        const float fx = V.fx, fy = V.fy;
        float dtx, dty, dtz;
        if (pin) {
            // J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]] (Eq. 1)
            const float iz = 1.f / tz, iz2 = iz * iz, iz3 = iz2 * iz;
            dtx = Jm[0] * g0.x - dJ[2] * fx * iz2;
            dty = Jm[4] * g0.y - dJ[5] * fy * iz2;
            dtz = Jm[2] * g0.x + Jm[5] * g0.y - dJ[0] * fx * iz2 + 2.f * dJ[2] * fx * tx * iz3 - dJ[4] * fy * iz2 +
                  2.f * dJ[5] * fy * ty * iz3;
        } else {
            const float rho = jg.rho, rho2 = jg.rho2, r2 = jg.r2;
            const float irho4 = 1.f / (rho2 * rho2);
            const float ir4 = 1.f / (r2 * r2);
            const float irho = 1.f / rho, irho3 = irho / rho2;
            dtx = jg.J[0] * g0.x + jg.J[3] * g0.y;
            dty = jg.J[4] * g0.y;
            dtz = jg.J[2] * g0.x + jg.J[5] * g0.y;
            // row 1: J11 = fx tz / rho^2, J13 = -fx tx / rho^2
            dtx += fx * irho4 * (-2.f * tx * tz * dJ[0] + (tx * tx - tz * tz) * dJ[2]);
            dtz += fx * irho4 * ((tx * tx - tz * tz) * dJ[0] + 2.f * tx * tz * dJ[2]);
            // row 2: J21 = -fy tx ty / (r^2 rho), J22 = fy rho / r^2, J23 = -fy ty tz / (r^2 rho)
            const float k3 = fy * ir4 * irho3, k1 = fy * ir4 * irho;
            const float rr = 2.f * rho2 + r2;
            dtx += -k3 * ty * (tz * tz * r2 - 2.f * tx * tx * rho2) * dJ[3];
            dty += -k1 * tx * (r2 - 2.f * ty * ty) * dJ[3];
            dtz += k3 * tx * ty * tz * rr * dJ[3];
            dtx += k1 * tx * (r2 - 2.f * rho2) * dJ[4];
            dty += -2.f * fy * ir4 * rho * ty * dJ[4];
            dtz += k1 * tz * (r2 - 2.f * rho2) * dJ[4];
            dtx += k3 * tx * ty * tz * rr * dJ[5];
            dty += -k1 * tz * (r2 - 2.f * ty * ty) * dJ[5];
            dtz += -k3 * ty * (tx * tx * r2 - 2.f * tz * tz * rho2) * dJ[5];
        }
        // t = W mu + t_wc
        gm[0] += W[0] * dtx + W[3] * dty + W[6] * dtz;
        gm[1] += W[1] * dtx + W[4] * dty + W[7] * dtz;
        gm[2] += W[2] * dtx + W[5] * dty + W[8] * dtz;
        gop += g1.y;

    }

    if (a.d_count && st_count != st_count0) {  // this thread owns Gaussian g
        a.d_grad[g] = st_grad;
        a.d_elev[g] = st_elev;
        a.d_count[g] = st_count;
    }

    float gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
    if (any) {
        // M = R diag(s): ds_j = sum_i dM_ij R_ij, dR_ij = dM_ij s_j
        float dR[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                gs[j] += dM[3 * i + j] * Rq[3 * i + j];
                dR[3 * i + j] = dM[3 * i + j] * s[j];
            }
        // R(q) partials (q normalized)
        float dw = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
        float dx = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - qw * dR[5] + qz * dR[6] +
                          qw * dR[7] - 2.f * qx * dR[8]);
        float dy = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] +
                          qz * dR[7] - 2.f * qy * dR[8]);
        float dz = 2.f * (-2.f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.f * qz * dR[4] +
                          qy * dR[5] + qx * dR[6] + qy * dR[7]);
        float dot = qw * dw + qx * dx + qy * dy + qz * dz;
        gq[0] = (dw - qw * dot) / qn; gq[1] = (dx - qx * dot) / qn;
        gq[2] = (dy - qy * dot) / qn; gq[3] = (dz - qz * dot) / qn;
    }
    // colour phase (after the geometry, so that its SH registers are not live together with the
    // covariance chain): dL/dsh and the view direction's gradient, view by view
    constexpr int KG = ONE ? 1 : 16;
    float gsh[KG][3];
#pragma unroll
    for (int k = 0; k < KG; ++k) gsh[k][0] = gsh[k][1] = gsh[k][2] = 0.f;
    float ysh[ONE ? 16 : 1], msh[3] = {0.f, 0.f, 0.f};  // one view: dL/dsh[k][c] = msh[c] ysh[k]
#pragma unroll
    for (int k = 0; k < (ONE ? 16 : 1); ++k) ysh[k] = 0.f;
    if (ONE && any) {
        const float4 g1 = a.acc[1 + 3 * (size_t)g], g2 = a.acc[2 + 3 * (size_t)g];
        if (g1.z != 0.f || g1.w != 0.f || g2.x != 0.f) {
            const ViewDev& V = a.views[0];
            const float vx = m0 - V.cam[0], vy = m1 - V.cam[1], vz = m2 - V.cam[2];
            const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
            const float x = vx * il, y = vy * il, z = vz * il;
            float Y[16];
            sh_basis<DEG>(x, y, z, Y);
            const float drgb[3] = {g1.z, g1.w, g2.x};
            const float* shg = a.sh + (size_t)g * a.sh_coeffs * 3;
            // two passes over the coefficient row, 16-byte loads where the rows allow them (the
            // second pass hits L1): the colours (which channels are clamped), then the weights
            // w_k = sum over unclamped channels of dL/drgb_c sh_kc of the direction's gradient
            const bool vec = (a.sh_coeffs * 3) % 4 == 0;
            float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
            for (int i = 0; i < (K * 3 + 3) / 4; ++i) {
                float q[4];
                if (vec) {
                    const float4 t4 = __ldg(reinterpret_cast<const float4*>(shg) + i);
                    q[0] = t4.x; q[1] = t4.y; q[2] = t4.z; q[3] = t4.w;
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) q[r] = 4 * i + r < K * 3 ? __ldg(shg + 4 * i + r) : 0.f;
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int e = 4 * i + r;
                    if (e < K * 3) col[e % 3] = fmaf(q[r], Y[e / 3], col[e % 3]);
                }
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) msh[ch] = col[ch] < 0.f ? 0.f : drgb[ch];  // clamped channels
            if (DEG > 0) {
                float w[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) w[k] = 0.f;
#pragma unroll
                for (int i = 0; i < (K * 3 + 3) / 4; ++i) {
                    float q[4];
                    if (vec) {
                        const float4 t4 = __ldg(reinterpret_cast<const float4*>(shg) + i);
                        q[0] = t4.x; q[1] = t4.y; q[2] = t4.z; q[3] = t4.w;
                    } else {
#pragma unroll
                        for (int r = 0; r < 4; ++r) q[r] = 4 * i + r < K * 3 ? __ldg(shg + 4 * i + r) : 0.f;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int e = 4 * i + r;
                        if (e < K * 3) w[e / 3] = fmaf(msh[e % 3], q[r], w[e / 3]);
                    }
                }
                float gx, gy, gz;
                sh_grad_acc<DEG>(x, y, z, w, gx, gy, gz);
                const float dd = gx * x + gy * y + gz * z;  // project out the radial part
                gm[0] += (gx - dd * x) * il;
                gm[1] += (gy - dd * y) * il;
                gm[2] += (gz - dd * z) * il;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) ysh[k] = Y[k];
        }
    }
    if (!ONE && any) {
        float shc[16][3];
        load_sh<DEG>(a.sh, a.sh_coeffs, g, shc);
        for (int v = 0; v < a.n_views; ++v) {
            const size_t item = (size_t)v * a.n + g;
            const float4 g1 = a.acc[3 * item + 1], g2 = a.acc[3 * item + 2];
            if (g1.z == 0.f && g1.w == 0.f && g2.x == 0.f) continue;
            const ViewDev& V = a.views[v];
            const float vx = m0 - V.cam[0], vy = m1 - V.cam[1], vz = m2 - V.cam[2];
            const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
            const float x = vx * il, y = vy * il, z = vz * il;
            float Y[16];
            sh_basis<DEG>(x, y, z, Y);
            const float drgb[3] = {g1.z, g1.w, g2.x};
            float wsum[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) wsum[k] = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float acc = 0.5f;
#pragma unroll
                for (int k = 0; k < K; ++k) acc = fmaf(shc[k][ch], Y[k], acc);
                if (acc < 0.f) continue;  // clamped channel
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    gsh[ONE ? 0 : k][ch] += drgb[ch] * Y[k];
                    wsum[k] += drgb[ch] * shc[k][ch];
                }
            }
            if (DEG > 0) {
                float gx, gy, gz;
                sh_grad_acc<DEG>(x, y, z, wsum, gx, gy, gz);
                const float dd = gx * x + gy * y + gz * z;  // project out the radial part
                gm[0] += (gx - dd * x) * il;
                gm[1] += (gy - dd * y) * il;
                gm[2] += (gz - dd * z) * il;
            }
        }
    }

    // chain through the activations: d/dlog s = d/ds * s, d/dlogit = d/do * o (1 - o); a Gaussian
    // that contributed nowhere keeps exact zeros (also when a scale is inf)
    if (a.raw && any) {
#pragma unroll
        for (int i = 0; i < 3; ++i) gs[i] *= s[i];
        const float o = sigmoid_act(__ldg(a.opacity + g));
        gop *= o * (1.f - o);
    }
    // write (or accumulate) the parameter gradients
    float* pm = a.g_means + 3 * g;
    float* ps = a.g_scales + 3 * g;
    float* pq = a.g_quats + 4 * g;
    float* psh = a.g_sh + (size_t)g * a.sh_coeffs * 3;
    if (a.accumulate) {
        if (!any) return;
#pragma unroll
        for (int i = 0; i < 3; ++i) { pm[i] += gm[i]; ps[i] += gs[i]; }
#pragma unroll
        for (int i = 0; i < 4; ++i) pq[i] += gq[i];
        a.g_opacity[g] += gop;
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) psh[3 * k + ch] += ONE ? msh[ch] * ysh[k] : gsh[ONE ? 0 : k][ch];
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) { pm[i] = gm[i]; ps[i] = gs[i]; }
        reinterpret_cast<float4*>(pq)[0] = make_float4(gq[0], gq[1], gq[2], gq[3]);
        a.g_opacity[g] = gop;
        if ((a.sh_coeffs * 3) % 4 == 0 && (K * 3) % 4 == 0) {
            float4* p4 = reinterpret_cast<float4*>(psh);
#pragma unroll
            for (int i = 0; i < K * 3 / 4; ++i) {
                const int e = 4 * i;
                float q[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int kk = (e + r) / 3, ch = (e + r) % 3;
                    q[r] = ONE ? msh[ch] * ysh[kk] : gsh[ONE ? 0 : kk][ch];
                }
                p4[i] = make_float4(q[0], q[1], q[2], q[3]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) psh[3 * k + ch] = ONE ? msh[ch] * ysh[k] : gsh[ONE ? 0 : k][ch];
        }
        for (int k = K; k < a.sh_coeffs; ++k)
            for (int ch = 0; ch < 3; ++ch) psh[3 * k + ch] = 0.f;
    }
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_setup(const ViewTable& tab, ViewDev* views, float4* trig, Header* hdr, int total_trig,
                         uint32_t* dhist, cudaStream_t st) {
    int threads = 256;
    int blocks = (max(total_trig, tab.n_views) + threads - 1) / threads;
    blocks = max(1, min(blocks, 1024));
    k_setup<<<blocks, threads, 0, st>>>(tab, views, trig, hdr, total_trig, dhist);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(const PreArgs& a, int sh_degree, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    const int threads = 256, blocks = (a.n + threads - 1) / threads;
    k_preprocess_geom<<<blocks, threads, 0, st>>>(a);
    switch (sh_degree) {
        case 0: k_preprocess_color<0><<<blocks, threads, 0, st>>>(a); break;
        case 1: k_preprocess_color<1><<<blocks, threads, 0, st>>>(a); break;
        case 2: k_preprocess_color<2><<<blocks, threads, 0, st>>>(a); break;
        default: k_preprocess_color<3><<<blocks, threads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const PreBwdArgs& a, int sh_degree, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    int threads = 128, blocks = (a.n + threads - 1) / threads;
    const bool one = a.n_views == 1;
    switch (sh_degree) {
        case 0: one ? k_preprocess_bwd<0, true><<<blocks, threads, 0, st>>>(a)
                    : k_preprocess_bwd<0, false><<<blocks, threads, 0, st>>>(a); break;
        case 1: one ? k_preprocess_bwd<1, true><<<blocks, threads, 0, st>>>(a)
                    : k_preprocess_bwd<1, false><<<blocks, threads, 0, st>>>(a); break;
        case 2: one ? k_preprocess_bwd<2, true><<<blocks, threads, 0, st>>>(a)
                    : k_preprocess_bwd<2, false><<<blocks, threads, 0, st>>>(a); break;
        default: one ? k_preprocess_bwd<3, true><<<blocks, threads, 0, st>>>(a)
                     : k_preprocess_bwd<3, false><<<blocks, threads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace odgs
