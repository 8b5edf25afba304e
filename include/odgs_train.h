/*
 * odgs_train.h -- C ABI of the training-side steps around the ODGS rasterizer (sm_103a).
 *
 * Densification (ODGS Sec. 3.3, hyper-parameters of App. A.1). ODGS keeps the densification
 * loop of 3D Gaussian splatting and makes its gradient threshold depend on the elevation of the
 * Gaussian seen from the camera,
 *     tau_mu = tau_min + (1 - cos theta_mu) (tau_max - tau_min),   tau_min = 2e-5, tau_max = 1e-4,
 * because the ERP projection stretches Gaussians near the poles. The statistics are gathered by
 * odgs_preprocess_bwd (odgs_grads.densify_*, odgs.h); the calls below turn them into decisions
 * and build the densified parameter arrays.
 *
 * All pointers are device pointers owned by the caller unless noted; the structs are host
 * memory read during the call. Calls are asynchronous on the given stream (cudaStream_t as
 * void*, NULL = legacy default stream) and allocate nothing.
 */
#ifndef ODGS_TRAIN_H
#define ODGS_TRAIN_H

#include "odgs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Densification actions (one byte per Gaussian). */
#define ODGS_KEEP 0u
#define ODGS_CLONE 1u /* kept, plus one identical copy                                    */
#define ODGS_SPLIT 2u /* replaced by two children at mu + R(q)(s * z), scales s / 1.6       */
#define ODGS_PRUNE 4u /* removed                                                           */

typedef struct {
    float tau_min, tau_max; /* thresholds at the equator and at the poles (2e-5, 1e-4)          */
    float percent_dense;    /* clone when max scale <= percent_dense * scene_extent, else split
                               (App. A.1: 1e-3)                                                  */
    float scene_extent;     /* > 0                                                               */
    float min_opacity;      /* prune when opacity < min_opacity (3DGS: 0.005)                    */
    float max_scale;        /* prune when a scale > max_scale; 0 disables                        */
    int raw_params;         /* 1: scales are log-scales and opacity logits (odgs_settings
                               .raw_params); the comparisons below then run in that space, against
                               thresholds computed once on the host in double precision and
                               rounded to float: log(percent_dense * scene_extent), the logit of
                               min_opacity, log(max_scale); split children get log s - log 1.6 */
} odgs_densify_params;

/* Decision per Gaussian from the accumulated statistics (float32 arithmetic, fixed order):
 *   c = count[i]; if c > 0: g = grad[i] / c, e = elev[i] / c (each one IEEE division)
 *   tau = tau_min + e * (tau_max - tau_min)   (one rounded product, one rounded sum)
 *   densify = c > 0 && g >= tau;  big = max(scales[i]) > percent_dense * scene_extent (a float
 *   product); prune = opacity[i] < min_opacity || (max_scale > 0 && max(scales[i]) > max_scale)
 *   action = prune ? ODGS_PRUNE : densify ? (big ? ODGS_SPLIT : ODGS_CLONE) : ODGS_KEEP
 * grad, elev: [n] float; count: [n] uint32; scales [n][3] and opacity [n] (activated, or raw as
 * described under raw_params); action: [n] bytes written. n >= 0. */
odgs_status odgs_densify_select(const float *grad, const float *elev, const uint32_t *count,
                                const float *scales, const float *opacity, int n,
                                const odgs_densify_params *p, uint8_t *action, void *stream);

/* Output parameter arrays (device, layouts of odgs_gaussians). */
typedef struct {
    float *means, *scales, *quats, *opacity, *sh;
} odgs_params_out;

/* Bytes of scratch odgs_densify_apply needs for n Gaussians (host-only, pure). */
odgs_status odgs_densify_scratch_size(int n, size_t *bytes);

/* Builds the densified Gaussians from in (n Gaussians, sh_coeffs coefficients each; log-scales
 * when raw_params = 1) and action:
 *   [0, K)                 Gaussians with ODGS_KEEP or ODGS_CLONE, in index order
 *   [K, K + C)             the copies of the ODGS_CLONE ones, in index order
 *   [K + C, K + C + S)     the first children of the ODGS_SPLIT ones, in index order
 *   [K + C + S, K + C + 2S) their second children
 * A child c of Gaussian i sits at mu_i + R(q_i) (s_i * noise[i][c]) (noise: [n][2][3] standard
 * normal draws, read for split Gaussians only) with scales s_i / 1.6 (log-scales log s_i - ln 1.6
 * when raw_params = 1); rotation, opacity and SH are copied. *n_out (device, one uint32)
 * receives K + C + 2S; outputs at or beyond out_capacity are not written (the caller compares
 * *n_out with its capacity). The output arrays must not
 * overlap the inputs. scratch: odgs_densify_scratch_size(n) bytes, 16-byte aligned. */
odgs_status odgs_densify_apply(const odgs_gaussians *in, int sh_coeffs, int raw_params,
                               const uint8_t *action, const float *noise, const odgs_params_out *out,
                               int out_capacity, uint32_t *n_out, void *scratch, size_t scratch_bytes,
                               void *stream);

/* Adam (Kingma & Ba 2015, bias-corrected), the optimiser ODGS trains with (App. A.1: the 3DGS
 * recipe), over up to ODGS_ADAM_MAX_GROUPS groups of float32 parameters in one launch. Per
 * element of a group, at step t >= 1:
 *   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2
 *   p <- p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
 * with the bias corrections computed once on the host in double precision. Element j of a group
 * uses lr when (j mod row) < head and lr_tail otherwise: with row = 3 K and head = 3 an SH array
 * [n][K][3] gets 3DGS's separate rates for the DC and the higher-order coefficients.
 * param, m, v: device arrays updated in place; grad: device array read; count elements each (no
 * overlap between groups). m and v start at zero (step 1). */
#define ODGS_ADAM_MAX_GROUPS 8
typedef struct {
    float *param;
    const float *grad;
    float *m, *v;
    size_t count;
    float lr, lr_tail;
    int row, head; /* row >= 1, 0 <= head <= row                                         */
} odgs_adam_group;

typedef struct {
    double beta1, beta2;     /* 3DGS: 0.9, 0.999. Double, so that 1 - beta is formed before any
                                rounding to float (1 - (float)0.999 is off by 1.3e-5 relative)  */
    double eps;              /* 3DGS: 1e-15                                                   */
    int step;                /* t >= 1                                                        */
} odgs_adam_params;

odgs_status odgs_adam_step(const odgs_adam_group *groups, int n_groups, const odgs_adam_params *p,
                           void *stream);

/* Photometric loss of 3DGS training on one ERP image (App. A.1 keeps the 3DGS loss):
 *   L = (1 - lambda) L1 + lambda (1 - SSIM),
 * SSIM of Wang et al. 2004 with an 11 x 11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2,
 * per channel. Both terms are means over the 3 x W x H values, weighted per pixel row by
 * cos(theta_j) when area_weight = 1 (theta_j = pi (1/2 - (j + 1/2) / H), Eq. 4's elevation of
 * the row centre: the solid angle of the row). The window wraps around the longitude seam when
 * wrap_u = 1 (zero padding otherwise) and is zero-padded above and below the image.
 * With lambda = 0 the call computes the (weighted) L1 term alone in one pass over the pixels.
 * image, target: device [3][H][W] float32. grad: device [3][H][W], receives dL/dimage (the L1
 * term's derivative at image == target is 0); may be NULL. loss: device float, receives L (or L
 * is added to it when accumulate = 1, so that views sum into one value). scratch:
 * odgs_loss_scratch_size bytes, 16-byte aligned, reused by every call on the same stream. */
typedef struct {
    float lambda;    /* D-SSIM weight; 3DGS: 0.2                          */
    int area_weight; /* 1: cos(theta) row weights                         */
    int wrap_u;      /* 1: the window wraps around the seam               */
    int accumulate;  /* 1: *loss += L; 0: *loss = L                       */
} odgs_loss_params;

odgs_status odgs_loss_scratch_size(int width, int height, size_t *bytes);

odgs_status odgs_loss_l1_dssim(const float *image, const float *target, int width, int height,
                               const odgs_loss_params *p, float *grad, float *loss, void *scratch,
                               size_t scratch_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ODGS_TRAIN_H */
