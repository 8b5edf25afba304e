/*
 * odgs.h -- C ABI of the GB300 (sm_103a) differentiable omnidirectional Gaussian rasterizer.
 *
 * The library renders 3D Gaussians into equirectangular (ERP) images and back-propagates
 * image gradients to the Gaussian parameters, as described by ODGS (arXiv 2410.20686):
 *   - projection of each Gaussian onto the tangent plane of the unit sphere at its centre and
 *     the ERP Jacobian J_omni (Sec. 3.2, Eq. 4-8), Sigma_2D = J_omni W Sigma W^T J_omni^T;
 *   - spherical-shell culling (Sec. 3.2), view-dependent colour from spherical harmonics;
 *   - depth-ordered front-to-back alpha blending of the 2D Gaussians (Sec. 3.1, Eq. 2-3);
 *   - the backward pass of App. A.3 (Eq. 11 and the Jacobian's dependence on the mean).
 *
 * Call sequence for one frame (one or many views of the same Gaussians):
 *   odgs_preprocess -> [odgs_query_pairs] -> odgs_bin_sort -> odgs_render_fwd
 *   -> odgs_render_bwd -> odgs_preprocess_bwd
 * All compute calls are asynchronous on the given CUDA stream (a cudaStream_t passed as void*;
 * NULL = legacy default stream). Only odgs_query_pairs, odgs_get_status and odgs_frame_stats
 * synchronize. odgs_bin_sort also runs work on a stream of the context, forked from the given
 * stream and joined back to it by events within the call, so the call is ordered on the given
 * stream as a whole (and can be captured in a CUDA graph from it).
 *
 * Memory: the caller owns every buffer. Device pointers below point to device memory; the
 * structs themselves and the pointer arrays (images, final_T, dL_dimages) live in host memory
 * and are read during the call. The library allocates no device memory: its scratch is the
 * caller's "workspace" (sized by odgs_workspace_size) and "pair buffer" (sized by
 * odgs_pair_buffer_size). Both must stay allocated, and the Gaussian arrays unchanged, from
 * odgs_preprocess until the last call of the frame (dL_dimages until odgs_render_bwd has
 * been followed by odgs_preprocess_bwd). Host state lives in an odgs_ctx.
 *
 * Errors: argument errors are returned synchronously (nothing is launched). CUDA launch errors
 * return ODGS_ERR_CUDA. Errors found on the device (pair capacity exceeded, a bounded wait
 * that gave up, non-finite inputs when odgs_settings.checked is set) set bits in a device
 * status word: the kernels skip the work they cannot do without writing out of bounds, and
 * odgs_query_pairs / odgs_get_status report the bits.
 */
#ifndef ODGS_H
#define ODGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ODGS_OK = 0,
    ODGS_ERR_INVALID_ARG = -1, /* bad pointer, size, layout or setting; nothing launched      */
    ODGS_ERR_CAPACITY = -2,    /* more tile/Gaussian pairs than the pair buffer holds          */
    ODGS_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed                  */
    ODGS_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up (results are invalid)     */
    ODGS_ERR_NONFINITE = -5,   /* a non-finite parameter or image gradient (checked mode)      */
    ODGS_ERR_STATE = -6,       /* calls made out of order (e.g. render before bin_sort)        */
    ODGS_ERR_WORKSPACE = -7    /* workspace or pair buffer smaller than required               */
} odgs_status;

/* Device status word bits, reported by odgs_get_status. */
#define ODGS_DEV_CAPACITY 1u
#define ODGS_DEV_TIMEOUT 2u
#define ODGS_DEV_NONFINITE 4u  /* checked mode: a Gaussian with a non-finite parameter (culled
                                  in every view) or a non-finite dL/dimage value (taken as 0) */

#define ODGS_MAX_VIEWS 64

/* One camera. World point mu maps to camera space as t = R_wc mu + t_wc, with OpenCV axes
 * (x right, y down, z forward; Sec. 3.2). Pixel (i, j) is sampled at (i + 0.5, j + 0.5) of the
 * image plane:
 *   model 0 (ERP, the paper's camera): Eq. 4, u = W/(2 pi) phi + W/2, v = -H/pi theta + H/2;
 *     culled inside the spherical shell r <= r_near or r >= r_far; depth key r = |t|; the
 *     image wraps around the longitude seam.
 *   model 1 (pinhole, the perspective case of Eq. 1, as in 3DGS(P) cube faces):
 *     u = fx tx/tz + cx, v = fy ty/tz + cy; culled when tz <= r_near or tz >= r_far or when the
 *     projected centre lies outside [-0.3 W, 1.3 W] x [-0.3 H, 1.3 H]; depth key tz; no wrap. */
typedef struct {
    int width, height;     /* 1 <= W, H <= 16384; W a multiple of the tile width      */
    float R_wc[9];         /* row-major world -> camera rotation                       */
    float t_wc[3];
    int model;             /* 0: ERP, 1: pinhole                                       */
    float fx, fy, cx, cy;  /* pinhole focal lengths (> 0) and principal point, pixels  */
} odgs_view;

typedef struct {
    int sh_degree;      /* 0..3; colour = max(0, sum_k sh_k Y_k(d) + 0.5)               */
    int sh_coeffs;      /* coefficients stored per Gaussian in sh (>= (deg+1)^2)        */
    int tile_w, tile_h; /* pixel tile; 0 -> 16 x 16. tile_w * tile_h in [32, 1024],
                           tile_w in {8, 16, 32}                                       */
    int batch;          /* Gaussians staged per shared-memory batch by the forward blend;
                           0 -> 128 (<= 256); the backward stages min(batch, 64)         */
    float cov_dilation; /* added to both diagonals of Sigma_2D (px^2); e.g. 0.3          */
    float r_near, r_far;/* spherical-shell culling radii (Sec. 3.2); e.g. 0.2, 1e4       */
    float bg[3];        /* background colour blended with the final transmittance        */
    int recompute_lists;/* 1: odgs_render_bwd rebuilds the tile lists (odgs_bin_sort) in the
                           pair buffer last given to odgs_bin_sort, which the caller may
                           reuse for other frames between the forward and backward passes */
    int grad_accumulate;/* 1: gradients are added (+=) to the output arrays; 0: written  */
    int pixels_per_thread; /* forward blend: pixels of one row per thread, 1, 2, 4 or 8, such
                              that it divides tile_w and tile_w * tile_h / pixels_per_thread is
                              a multiple of 32 and at most 256; 0 -> 2 if that fits, else the
                              largest of 4, 2, 1 that does                                     */
    int raw_params;     /* 1: odgs_gaussians.scales hold log-scales and .opacity logits, the
                           variables 3DGS optimises; the library applies exp and the sigmoid
                           and odgs_preprocess_bwd returns the gradients w.r.t. these raw
                           variables. 0: activated values (scales > 0, opacity in (0, 1)) */
    int pixels_per_thread_bwd; /* backward blend, the same choices; 0 -> 4 if that fits, else the
                                  largest of 4, 2, 1 that does. Per-pixel results do not depend
                                  on either value                                           */
    int checked;        /* 1: check the Gaussian parameters (after activation) and dL/dimage
                           for NaN / inf: an offending Gaussian is culled in every view, an
                           offending gradient value counts as 0, and ODGS_DEV_NONFINITE is set.
                           0: no checks (non-finite inputs give unspecified results)      */
    int full_lists;     /* 0: odgs_bin_sort cuts each tile's list after the depth at which every
                           pixel of the tile has provably stopped (T < 1e-4): it sums, depth
                           bucket by depth bucket, -log2(1 - a) over the Gaussians whose alpha
                           is at least a >= 1/255 at all the tile's pixel centres (the minimum
                           of a convex exponent over the tile is at a corner pixel). Images,
                           final T and gradients are the same as with the whole lists; fewer
                           pairs are emitted and sorted. Frames of more than 2^19 tiles keep
                           the whole lists. 1: the whole lists (every Gaussian whose footprint
                           meets the tile)                                                 */
} odgs_settings;

/* Gaussian parameters, device pointers, float32, contiguous:
 *   means [n][3], scales [n][3] (activated, > 0), quats [n][4] (w, x, y, z; normalized by the
 *   library), opacity [n] (activated, in (0, 1)), sh [n][sh_coeffs][3] (16-byte aligned when
 *   3*sh_coeffs is a multiple of 4). n >= 0. */
typedef struct {
    const float *means, *scales, *quats, *opacity, *sh;
    int n;
} odgs_gaussians;

/* Parameter gradients, device pointers with the layouts of odgs_gaussians.
 * Optional densification statistics (Sec. 3.3): three device arrays of n elements, all given or
 * all NULL. odgs_preprocess_bwd always ADDS to them (they run over many frames until the caller
 * densifies and clears them): for every view in which the Gaussian survived culling,
 *   densify_grad  += || (dL/du * W/2, dL/dv * H/2) ||   (the frame's ERP-mean gradient in the
 *                                                       [-1, 1] image coordinates of 3DGS)
 *   densify_elev  += 1 - cos(theta)                      (theta: elevation of the mean, Eq. 4)
 *   densify_count += 1
 * odgs_densify_select (odgs_train.h) turns them into clone / split / prune decisions. */
typedef struct {
    float *means, *scales, *quats, *opacity, *sh;
    float *densify_grad, *densify_elev;
    uint32_t *densify_count;
} odgs_grads;

typedef struct odgs_ctx odgs_ctx;

/* Create / destroy host-side state for the current CUDA device. Creating queries the device
 * (SM count, occupancy); it allocates host memory only. */
odgs_status odgs_create(odgs_ctx **out);
void odgs_destroy(odgs_ctx *ctx);

/* Bytes of device workspace needed for n Gaussians and these views (host-only, pure). */
odgs_status odgs_workspace_size(int n, const odgs_view *views, int n_views, const odgs_settings *s,
                                size_t *bytes);

/* Bytes of pair buffer for up to pair_capacity (tile, Gaussian) pairs (< 2^30). */
odgs_status odgs_pair_buffer_size(size_t pair_capacity, size_t *bytes);

/* Per Gaussian and view (Sec. 3.1-3.2, Eq. 4-8): covariance, camera transform, shell culling,
 * ERP mean and covariance, SH colour, conservative tile rectangle with longitude-seam wrap and
 * pole stretch, depth key. Also counts the (tile, Gaussian) pairs of the frame. */
odgs_status odgs_preprocess(odgs_ctx *ctx, const odgs_gaussians *g, const odgs_view *views,
                            int n_views, const odgs_settings *s, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Synchronizes the stream; returns the number of pairs the last odgs_preprocess produced
 * and, as the return value, the first error recorded on the device (or ODGS_OK). */
odgs_status odgs_query_pairs(odgs_ctx *ctx, size_t *pairs, void *stream);

/* Depth sort, per-tile pair emission and stable tile sort (the "sorting by depth" of Sec.
 * 3.1, binned into ERP tiles), then per-tile list ranges. Pairs beyond pair_capacity are
 * dropped and set ODGS_DEV_CAPACITY. */
odgs_status odgs_bin_sort(odgs_ctx *ctx, void *pair_buffer, size_t pair_capacity, void *stream);

/* Front-to-back alpha blending of Eq. 3 for every view in one persistent launch.
 * images[v]: device [3][H][W] float32 (channel-major); final_T[v]: device [H][W] or NULL
 * (the array final_T itself may be NULL). */
odgs_status odgs_render_fwd(odgs_ctx *ctx, float *const *images, float *const *final_T, void *stream);

/* Backward pass, part 1: reverse of the blend of Eq. 3 per pixel (back to front from each
 * pixel's last blended Gaussian), accumulating per (view, Gaussian) the gradients w.r.t. its ERP
 * mean, conic, opacity and colour in the workspace. dL_dimages[v]: device [3][H][W] float32.
 * With recompute_lists = 1 it first rebuilds the tile lists (identical to the forward's) from the
 * records kept in the workspace, into the pair buffer last given to odgs_bin_sort. */
odgs_status odgs_render_bwd(odgs_ctx *ctx, const float *const *dL_dimages, void *stream);

/* Backward pass, part 2: chain rule from the accumulated screen-space gradients to the Gaussian
 * parameters (App. A.3: Eq. 11, dL/dJ = dL/dT W^T, the dependence of J_omni on the mean, the
 * mean path of Eq. 10, SH colour, quaternion and scale), summed over all views. Writes (or
 * adds, per grad_accumulate) all five gradient arrays. */
odgs_status odgs_preprocess_bwd(odgs_ctx *ctx, const odgs_grads *grads, void *stream);

/* Work counters of the current frame, read back after a stream synchronization. */
typedef struct {
    uint64_t pairs;         /* (tile, Gaussian) pairs counted by odgs_preprocess              */
    uint64_t pairs_sorted;  /* pairs emitted and sorted (min(pairs, capacity))                */
    uint64_t evals_fwd;     /* (pixel, list entry) evaluations of the last odgs_render_fwd    */
    uint64_t evals_bwd;     /* (pixel, list entry) evaluations of the last odgs_render_bwd    */
    uint64_t blended;       /* (pixel, Gaussian) pairs blended by the last odgs_render_fwd    */
    uint64_t entries_tile;  /* sum over tiles of the list entries the last odgs_render_fwd
                               processed until every pixel of the tile had stopped (each pixel
                               itself stops earlier: evals_fwd counts only its own entries)   */
    uint64_t visible;       /* (view, Gaussian) items that survived culling in odgs_preprocess */
    uint32_t status;        /* device status bits (ODGS_DEV_*)                                */
} odgs_stats;

odgs_status odgs_frame_stats(odgs_ctx *ctx, odgs_stats *out, void *stream);

/* Synchronizes the stream and returns the device status bits (ODGS_DEV_*) in *bits. */
odgs_status odgs_get_status(odgs_ctx *ctx, uint32_t *bits, void *stream);

/* Bound of the device-side waits (test and tuning hook). The sorts of odgs_bin_sort wait for the
 * per-digit counts of earlier sort tiles (decoupled look-back); a sort CTA that has read those
 * words `reads` times without reaching a complete prefix gives up, sets ODGS_DEV_TIMEOUT and
 * finishes with wrong (but in-bounds) positions: the frame's lists, images and gradients are then
 * invalid but finite, nothing is written or read out of bounds, and odgs_query_pairs returns
 * ODGS_ERR_TIMEOUT. Default 4194304 reads (seconds of waiting). 0 makes every sort of more than
 * one tile (more than 2048 keys) give up at once, which exercises the failure path without a GPU
 * fault. Takes effect from the next odgs_bin_sort of this context. */
odgs_status odgs_set_wait_limit(odgs_ctx *ctx, uint32_t reads);

/* Copies of the frame's integer binning state, for tests and inspection: the order in which
 * every tile blends its Gaussians, "sorting by depth" (Sec. 3.1, the order of Eq. 3). Valid after
 * odgs_bin_sort (or an odgs_render_bwd that rebuilt the lists). Asynchronous device-to-device
 * copies on `stream` into caller buffers (device, uint32); each pointer may be NULL:
 *   depth_keys  [n_items]  the depth keys in sorted order: IEEE bits of the FP32 depth (radial
 *                          distance |t| for ERP views, t_z for pinhole views), 0xFFFFFFFF for an
 *                          item culled or covering no pixel centre;
 *   depth_items [n_items]  the item (view * n + Gaussian) of each sorted key (ties by item);
 *   pair_tiles  [n_pairs]  the global tile id (view's first tile + row * tiles_x + column) of each
 *                          (tile, item) pair, tile-sorted; within a tile the pairs keep depth order;
 *   pair_items  [n_pairs]  the item of each pair;
 *   ranges      [2 * n_tiles]  [start, end) of every tile's run in the pair list ([0, 0) if none).
 * n_items must be views * n, n_tiles the frame's tile count (sum over views of
 * (W / tile_w) * ceil(H / tile_h)), n_pairs at most the pair capacity (odgs_frame_stats gives
 * the pairs sorted); otherwise ODGS_ERR_INVALID_ARG and nothing is copied. */
odgs_status odgs_debug_lists(odgs_ctx *ctx, uint32_t *depth_keys, uint32_t *depth_items, size_t n_items,
                             uint32_t *pair_tiles, uint32_t *pair_items, size_t n_pairs, uint32_t *ranges,
                             size_t n_tiles, void *stream);

/* Copy of the per-(view, Gaussian) screen-space gradients accumulated by the last
 * odgs_render_bwd, for tests and inspection (the reverse of Eq. 2-3 before the chain rule of
 * App. A.3). Asynchronous device-to-device copy on `stream` into out: device float32
 * [n_items][12], n_items = views * n, item = view * n + Gaussian, per item
 *   dL/du, dL/dv (ERP mean, pixels), dL/da, dL/dbeta, dL/dgamma (the conic in slice form:
 *   power = ln o - (a t^2 + gamma dy^2) / 2 with t = dx - beta dy; with Sigma_2D = [[A, B],
 *   [B, C]], a = C / det, beta = B / C, gamma = 1 / C, so that the conic's entries are a,
 *   -a beta, gamma + a beta^2), dL/do (opacity), dL/dr, dL/dg, dL/db (colour), 0, 0, 0.
 * ODGS_ERR_STATE before odgs_render_bwd; ODGS_ERR_INVALID_ARG if n_items differs. */
odgs_status odgs_debug_screen_grads(odgs_ctx *ctx, float *out, size_t n_items, void *stream);

/* Forward render of ONE view that allocates nothing and needs no workspace or pair buffer, for
 * callers that cannot call cudaMalloc (a plugin or frame callback inside a host application that
 * owns a fixed device-memory budget, or a real-time loop where cudaMalloc / cudaFree would
 * synchronize the device). The paper has no counterpart: it is a packaging of the forward path
 * (odgs_preprocess + odgs_bin_sort + odgs_render_fwd, same kernels, same image).
 * Inputs: g, view, s (host structs; device arrays as for odgs_preprocess, checked by the same
 * rules: a non-finite pose, an invalid setting or a misaligned array returns ODGS_ERR_INVALID_ARG).
 * The view may be ERP (model 0) or pinhole (model 1). Outputs: image [3][H][W] and final_T
 * [H][W] (device, final_T may be NULL), and status_out (device, one uint32_t) which receives the
 * device status bits (ODGS_DEV_CAPACITY when the frame had more pairs than fit: the pairs beyond
 * the capacity are dropped, the image stays finite) without a host synchronization.
 * Scratch: a 32 MiB file-scope device array that every GPU using this library holds until the
 * process exits. Limits: n <= 32768 Gaussians, W * H <= 524288 pixels, pairs up to what fits in
 * the rest of the array (about 1.4 million); larger sizes return ODGS_ERR_INVALID_ARG and
 * launch nothing. The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream capture. The address
 * is kept for the life of the process, so the device must not be reset (cudaDeviceReset) between
 * calls: after a reset the kept address no longer refers to the array. All calls
 * share the array and each one resets the parts that must start at zero; calls whose work
 * overlaps on the GPU (other streams, unordered host threads) race on it. */
odgs_status odgs_render_fwd_static(const odgs_gaussians *g, const odgs_view *view, const odgs_settings *s,
                                   float *image, float *final_T, uint32_t *status_out, void *stream);

/* Throughput of the arithmetic that bounds the blend kernels, measured on the current device
 * with CUDA events over every SM: independent FP32 FMA chains (an FMA counts 2 flop) and chains
 * of exp2f, the exponential the blend evaluates. They are the denominators of the blend
 * kernels' rooflines. Synchronizes the stream; allocates and frees one device buffer of
 * (SMs * 1024) floats; takes a few tens of milliseconds. */
typedef struct {
    double ffma_tflops; /* FP32 FMA throughput, TFLOP/s                               */
    double ex2_gops;    /* exp2f results per second, in units of 1e9                  */
    int sms;            /* multiprocessors of the device (all of them are used)       */
} odgs_peaks;

odgs_status odgs_measure_peaks(odgs_peaks *out, void *stream);

/* Kernel launches the last frame issued (for accounting). */
int odgs_last_launch_count(const odgs_ctx *ctx);

const char *odgs_status_string(odgs_status st);

#ifdef __cplusplus
}
#endif

#endif /* ODGS_H */
