/*
 * odgs_oracle.c -- plain FP64 CPU reference of the ODGS omnidirectional (equirectangular,
 * ERP) Gaussian rasterizer: forward image and hand-derived adjoint.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this file;
 * only the tests, the package smoke check and the bench's CPU-baseline leg use it. It shares
 * no code, header, constant table or helper with the CUDA path.
 *
 * What it computes (ODGS, Sec. 3.1-3.2 and App. A.2-A.3):
 *   per Gaussian   Sigma = R S S^T R^T (Sec. 3.1); camera-space mean t = W mu + t_wc;
 *                  phi = atan2(t_x, t_z), theta = atan2(-t_y, sqrt(t_x^2 + t_z^2)) (Sec. 3.2);
 *                  pixel mean by the ERP projection pi_o (Eq. 4); tangent-plane rotation
 *                  T_mu (Eq. 5), unit-focal Jacobian J_o (Eq. 6), stretch Q_o and pixel scale
 *                  S_o (Eq. 7), J_omni = S_o Q_o J_o T_mu (Eq. 8) computed as that product;
 *                  Sigma_2D = J_omni W Sigma W^T J_omni^T (+ dilation, see below);
 *                  spherical-shell culling (Sec. 3.2); view-dependent colour from real SH.
 *   per pixel      Gaussian footprint (Eq. 2), alpha = opacity * G, front-to-back blending
 *                  in depth order (Eq. 3).  No tiles and no bounding boxes: every surviving
 *                  Gaussian is tested at every requested pixel, in one global order.
 *   adjoint        reverse blend, then App. A.3: dL/dSigma_2D -> dL/dT with T = J W (Eq. 11)
 *                  -> dL/dJ = dL/dT W^T -> dL/dt through J_omni's dependence on the mean,
 *                  which this file derives in spherical coordinates (r, theta, phi) rather
 *                  than from Eq. 12 (whose second-row terms have the opposite sign to the
 *                  derivative of Eq. 8); plus the mean path d(u,v)/dt = J_omni (Eq. 10).
 *
 * Readings where the paper is silent (each is a fixed parameter or rule here):
 *   pixel (i, j) is sampled at (i + pix_offset, j + pix_offset), pix_offset = 0.5;
 *   Sigma_2D gets "dilation" added to both diagonal entries (3DGS-lineage low-pass);
 *   depth for sorting = radial distance |t| evaluated in IEEE single precision by the fixed
 *   operation order of depth_key_f32(); ties broken by Gaussian index;
 *   alpha = min(0.99, o G); a Gaussian with alpha < 1/255 is skipped; blending stops before
 *   the Gaussian that would take transmittance below 1e-4; background added with final T;
 *   culled: r <= r_near, r >= r_far, rho <= 1e-4 r, det(Sigma_2D) <= 0, 255 o <= 1;
 *   seam wrap: the horizontal offset x - u is wrapped to the nearest image in [-W/2, W/2);
 *   no wrap over the poles; colour = max(0, sum_k sh_k Y_k(d) + 0.5) with d the unit vector
 *   from the camera centre to the mean in world space and Y_k real orthonormal SH (no
 *   Condon-Shortley phase, order l = 0..3, m = -l..l) built from associated Legendre
 *   functions; the derivative of a clamped branch (alpha clamp, colour clamp) is zero.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared odgs_oracle.c -lm
 * (-ffp-contract=off keeps depth_key_f32() free of fused multiply-adds.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int width, height;
    double R[9]; /* world -> camera rotation W, row-major */
    double t[3]; /* world -> camera translation */
    int model;   /* 0: ERP (Eq. 4); 1: pinhole, u = fx tx/tz + cx, v = fy ty/tz + cy (Eq. 1) */
    double fx, fy, cx, cy; /* pinhole only */
} orc_view;

typedef struct {
    int sh_degree;   /* 0..3 */
    int sh_coeffs;   /* coefficients stored per Gaussian (>= (deg+1)^2) */
    double dilation; /* added to both diagonals of Sigma_2D, px^2 */
    double r_near, r_far;
    double bg[3];
    double pix_offset; /* pixel centre offset, 0.5 */
} orc_settings;

/* Per-Gaussian projection record (doubles), exported for the tests. */
enum {
    PJ_VALID = 0, PJ_KEY, PJ_DEPTH, PJ_R, PJ_PHI, PJ_THETA, PJ_U, PJ_V,
    PJ_T = 8,        /* camera-space mean, 3 */
    PJ_J = 11,       /* J_omni, 2x3 row-major, 6 */
    PJ_COV3 = 17,    /* world Sigma: xx xy xz yy yz zz, 6 */
    PJ_COV2 = 23,    /* Sigma_2D (dilated): A B C, 3 */
    PJ_CONIC = 26,   /* inverse: a b c, 3 */
    PJ_RGB = 29,     /* 3 */
    PJ_CLAMP = 32,   /* colour clamp flags, 3 */
    PJ_DIR = 35,     /* unit view direction (world), 3 */
    PJ_OPAC = 38,
    PJ_NFIELDS = 40
};

int orc_pj_nfields(void) { return PJ_NFIELDS; }

/* ---------------------------------------------------------------- small linear algebra */

static void mat3_mul(const double *A, const double *B, double *C) /* C = A B */
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void mat3_transpose(const double *A, double *At)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) At[3 * j + i] = A[3 * i + j];
}

/* Rotation matrix of a unit quaternion q = (w, x, y, z) (Hamilton convention). */
static void quat_to_rot(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR[k][e] = d R_e / d q_k for the map above (entries are quadratic in q). */
static void quat_to_rot_partials(const double *q, double dR[4][9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double d[4][9] = {
        /* d/dw */ {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0},
        /* d/dx */ {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x},
        /* d/dy */ {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y},
        /* d/dz */ {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0},
    };
    memcpy(dR, d, sizeof(d));
}

/* ---------------------------------------------------------------- spherical harmonics */

/* Associated Legendre functions P_l^m(cos vt) without the Condon-Shortley phase, l <= 3,
 * and their derivatives with respect to the polar angle vt; c = cos vt, s = sin vt.
 * Index l*(l+1)/2 + m for m = 0..l. */
static void legendre(double c, double s, double P[10], double dP[10])
{
    P[0] = 1.0;                              dP[0] = 0.0;
    P[1] = c;                                dP[1] = -s;                                 /* l1 m0 */
    P[2] = s;                                dP[2] = c;                                  /* l1 m1 */
    P[3] = 0.5 * (3 * c * c - 1);            dP[3] = -3 * c * s;                         /* l2 m0 */
    P[4] = 3 * c * s;                        dP[4] = 3 * (c * c - s * s);                /* l2 m1 */
    P[5] = 3 * s * s;                        dP[5] = 6 * s * c;                          /* l2 m2 */
    P[6] = 0.5 * (5 * c * c * c - 3 * c);    dP[6] = 0.5 * (-15 * c * c * s + 3 * s);    /* l3 m0 */
    P[7] = 1.5 * (5 * c * c - 1) * s;        dP[7] = 1.5 * (-10 * c * s * s + (5 * c * c - 1) * c);
    P[8] = 15 * c * s * s;                   dP[8] = 15 * (-s * s * s + 2 * c * c * s);  /* l3 m2 */
    P[9] = 15 * s * s * s;                   dP[9] = 45 * s * s * c;                     /* l3 m3 */
}

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* Real orthonormal SH Y_k (k = l^2 + l + m) at the direction with polar angle vt (from +z),
 * given by its cosine ct and sine st (taken from the direction itself, so that they stay exact
 * near the poles, where vt from atan2 would round to 0 or to the double nearest pi), and
 * azimuth vp (atan2(y, x)), plus dY/dvt and dY/dvp:
 *   Y_lm = sqrt(2) K_lm P_l^m cos(m vp)      (m > 0)
 *   Y_l0 = K_l0 P_l^0
 *   Y_lm = sqrt(2) K_l|m| P_l^|m| sin(|m| vp) (m < 0)
 * with K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). */
static void sh_basis(int deg, double ct, double st, double vp, double *Y, double *dYt, double *dYp)
{
    double P[10], dP[10];
    legendre(ct, st, P, dP);
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * factorial(l - am) / factorial(l + am));
            int pi = l * (l + 1) / 2 + am;
            int k = l * l + l + m;
            if (m == 0) {
                Y[k] = K * P[pi];
                dYt[k] = K * dP[pi];
                dYp[k] = 0.0;
            } else if (m > 0) {
                Y[k] = sqrt(2.0) * K * P[pi] * cos(am * vp);
                dYt[k] = sqrt(2.0) * K * dP[pi] * cos(am * vp);
                dYp[k] = -sqrt(2.0) * K * P[pi] * am * sin(am * vp);
            } else {
                Y[k] = sqrt(2.0) * K * P[pi] * sin(am * vp);
                dYt[k] = sqrt(2.0) * K * dP[pi] * sin(am * vp);
                dYp[k] = sqrt(2.0) * K * P[pi] * am * cos(am * vp);
            }
        }
    }
}

/* Exported for the SH pins: Y_k at a unit direction (world x, y, z). */
void orc_sh_eval(int deg, const double *dir, double *Y)
{
    double dYt[16], dYp[16];
    double n = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    double vp = atan2(dir[1], dir[0]);
    sh_basis(deg, dir[2] / n, sqrt(dir[0] * dir[0] + dir[1] * dir[1]) / n, vp, Y, dYt, dYp);
}

/* ---------------------------------------------------------------- depth key */

/* Radial depth |t| in IEEE single precision with a fixed operation order (no FMA):
 * t_i = ((W_i0 mu_0 + W_i1 mu_1) + W_i2 mu_2) + t_wc_i, r = sqrt((tx tx + ty ty) + tz tz).
 * Returns the float; its bit pattern is the sort key. */
static float depth_key_f32(const double *mu, const orc_view *v)
{
    float m0 = (float)mu[0], m1 = (float)mu[1], m2 = (float)mu[2];
    float t[3];
    for (int i = 0; i < 3; ++i) {
        float a = (float)v->R[3 * i + 0] * m0;
        float b = (float)v->R[3 * i + 1] * m1;
        float c = (float)v->R[3 * i + 2] * m2;
        float s = a + b;
        s = s + c;
        s = s + (float)v->t[i];
        t[i] = s;
    }
    if (v->model == 1) return t[2]; /* pinhole: the z depth, as perspective 3DGS sorts */
    float xx = t[0] * t[0];
    float yy = t[1] * t[1];
    float zz = t[2] * t[2];
    float q = xx + yy;
    q = q + zz;
    return sqrtf(q);
}

float orc_depth_f32(const double *mu, const orc_view *v) { return depth_key_f32(mu, v); }

/* ---------------------------------------------------------------- projection (forward) */

static void project_one(const double *mean, const double *scale, const double *quat, double opac,
                        const double *sh, const orc_view *v, const orc_settings *s, double *pj)
{
    memset(pj, 0, sizeof(double) * PJ_NFIELDS);
    const int W = v->width, H = v->height;

    /* Sigma = R S S^T R^T (Sec. 3.1) */
    double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    double q[4] = {quat[0] / qn, quat[1] / qn, quat[2] / qn, quat[3] / qn};
    double R[9], M[9], Mt[9], Sig[9];
    quat_to_rot(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * scale[j];
    mat3_transpose(M, Mt);
    mat3_mul(M, Mt, Sig);
    pj[PJ_COV3 + 0] = Sig[0]; pj[PJ_COV3 + 1] = Sig[1]; pj[PJ_COV3 + 2] = Sig[2];
    pj[PJ_COV3 + 3] = Sig[4]; pj[PJ_COV3 + 4] = Sig[5]; pj[PJ_COV3 + 5] = Sig[8];
    pj[PJ_OPAC] = opac;

    /* camera-space mean t = W mu + t_wc */
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = v->R[3 * i] * mean[0] + v->R[3 * i + 1] * mean[1] + v->R[3 * i + 2] * mean[2] + v->t[i];
    pj[PJ_T] = t[0]; pj[PJ_T + 1] = t[1]; pj[PJ_T + 2] = t[2];

    float rf = depth_key_f32(mean, v);
    uint32_t key;
    memcpy(&key, &rf, 4);
    pj[PJ_KEY] = (double)key;
    pj[PJ_DEPTH] = (double)rf;

    double r = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    double rho = sqrt(t[0] * t[0] + t[2] * t[2]);
    pj[PJ_R] = r;
    double J[6];
    if (v->model == 1) {
        /* pinhole (the perspective case of Sec. 3.1, Eq. 1): near / far planes on the float z
         * depth; centres outside the image widened by 30 % on each side are culled */
        if (!((double)rf > s->r_near && (double)rf < s->r_far)) return;
        double tz = t[2];
        double u = v->fx * t[0] / tz + v->cx, vv = v->fy * t[1] / tz + v->cy;
        if (!(u >= -0.3 * W && u <= 1.3 * W && vv >= -0.3 * H && vv <= 1.3 * H)) return;
        pj[PJ_PHI] = atan2(t[0], t[2]);
        pj[PJ_THETA] = atan2(-t[1], rho);
        pj[PJ_U] = u;
        pj[PJ_V] = vv;
        J[0] = v->fx / tz; J[1] = 0.0; J[2] = -v->fx * t[0] / (tz * tz);
        J[3] = 0.0; J[4] = v->fy / tz; J[5] = -v->fy * t[1] / (tz * tz);
        goto have_jacobian;
    }
    /* spherical-shell culling (Sec. 3.2) on the single-precision depth; poles culled */
    if (!((double)rf > s->r_near && (double)rf < s->r_far)) return;
    if (!(rho > 1e-4 * r)) return;

    /* spherical coordinates and ERP projection (Sec. 3.2, Eq. 4) */
    double phi = atan2(t[0], t[2]);
    double theta = atan2(-t[1], rho);
    pj[PJ_PHI] = phi;
    pj[PJ_THETA] = theta;
    pj[PJ_U] = (double)W / (2.0 * ORC_PI) * phi + (double)W / 2.0;
    pj[PJ_V] = -(double)H / ORC_PI * theta + (double)H / 2.0;

    /* T_mu = T_theta T_phi (Eq. 5) */
    double cp = cos(phi), sp = sin(phi), ct = cos(theta), st = sin(theta);
    double Tth[9] = {1, 0, 0, 0, ct, st, 0, -st, ct};
    double Tph[9] = {cp, 0, -sp, 0, 1, 0, sp, 0, cp};
    double Tmu[9];
    mat3_mul(Tth, Tph, Tmu);
    /* J_o (Eq. 6): unit-focal perspective Jacobian at (0, 0, |mu|), 2x3 */
    double Jo[6] = {1.0 / r, 0, 0, 0, 1.0 / r, 0};
    /* Q_o, S_o (Eq. 7) */
    double Qo[4] = {1.0 / ct, 0, 0, 1};
    double So[4] = {(double)W / (2.0 * ORC_PI), 0, 0, (double)H / ORC_PI};
    /* J_omni = S_o Q_o J_o T_mu (Eq. 8) */
    double SQ[4] = {So[0] * Qo[0] + So[1] * Qo[2], So[0] * Qo[1] + So[1] * Qo[3],
                    So[2] * Qo[0] + So[3] * Qo[2], So[2] * Qo[1] + So[3] * Qo[3]};
    double SQJ[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) SQJ[3 * i + j] = SQ[2 * i] * Jo[j] + SQ[2 * i + 1] * Jo[3 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += SQJ[3 * i + k] * Tmu[3 * k + j];
            J[3 * i + j] = acc;
        }
have_jacobian:
    memcpy(pj + PJ_J, J, sizeof(J));

    /* Sigma_2D = T Sigma T^T with T = J W (Sec. 3.2 / App. A.3), plus the dilation */
    double T[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = J[3 * i] * v->R[j] + J[3 * i + 1] * v->R[3 + j] + J[3 * i + 2] * v->R[6 + j];
    double TS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            TS[3 * i + j] = T[3 * i] * Sig[j] + T[3 * i + 1] * Sig[3 + j] + T[3 * i + 2] * Sig[6 + j];
    double A = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + s->dilation;
    double B = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    double C = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + s->dilation;
    pj[PJ_COV2] = A; pj[PJ_COV2 + 1] = B; pj[PJ_COV2 + 2] = C;
    double det = A * C - B * B;
    if (!(det > 0.0)) return;
    pj[PJ_CONIC] = C / det;
    pj[PJ_CONIC + 1] = -B / det;
    pj[PJ_CONIC + 2] = A / det;
    if (!(255.0 * opac > 1.0)) return;

    /* colour from real SH in the world-space view direction */
    double cam[3]; /* camera centre = -W^T t_wc */
    for (int j = 0; j < 3; ++j) cam[j] = -(v->R[j] * v->t[0] + v->R[3 + j] * v->t[1] + v->R[6 + j] * v->t[2]);
    double dv[3] = {mean[0] - cam[0], mean[1] - cam[1], mean[2] - cam[2]};
    double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int j = 0; j < 3; ++j) pj[PJ_DIR + j] = dv[j] / dn;
    double Y[16], dYt[16], dYp[16];
    double vp = atan2(dv[1], dv[0]);
    sh_basis(s->sh_degree, dv[2] / dn, sqrt(dv[0] * dv[0] + dv[1] * dv[1]) / dn, vp, Y, dYt, dYp);
    int K = (s->sh_degree + 1) * (s->sh_degree + 1);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + c] * Y[k];
        pj[PJ_CLAMP + c] = acc < 0.0 ? 1.0 : 0.0;
        pj[PJ_RGB + c] = acc < 0.0 ? 0.0 : acc;
    }
    pj[PJ_VALID] = 1.0;
}

int orc_project(int n, const double *means, const double *scales, const double *quats,
                const double *opacity, const double *sh, const orc_view *v, const orc_settings *s,
                double *pj)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        project_one(means + 3 * i, scales + 3 * i, quats + 4 * i, opacity[i],
                    sh + (size_t)3 * s->sh_coeffs * i, v, s, pj + (size_t)PJ_NFIELDS * i);
    return 0;
}

/* ---------------------------------------------------------------- global depth order */

typedef struct {
    uint32_t key;
    int id;
} key_id;

static int cmp_key_id(const void *a, const void *b)
{
    const key_id *x = (const key_id *)a, *y = (const key_id *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Compact copy of what a pixel needs, in global (depth, index) order. */
typedef struct {
    int id;
    double u, v, a, b, c, o, rgb[3];
} sorted_g;

static sorted_g *sort_visible(int n, const double *pj, int *m_out)
{
    key_id *ki = (key_id *)malloc(sizeof(key_id) * (n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const double *p = pj + (size_t)PJ_NFIELDS * i;
        if (p[PJ_VALID] != 0.0) {
            ki[m].key = (uint32_t)p[PJ_KEY];
            ki[m].id = i;
            ++m;
        }
    }
    qsort(ki, m, sizeof(key_id), cmp_key_id);
    sorted_g *g = (sorted_g *)malloc(sizeof(sorted_g) * (m > 0 ? m : 1));
    for (int k = 0; k < m; ++k) {
        const double *p = pj + (size_t)PJ_NFIELDS * ki[k].id;
        g[k].id = ki[k].id;
        g[k].u = p[PJ_U]; g[k].v = p[PJ_V];
        g[k].a = p[PJ_CONIC]; g[k].b = p[PJ_CONIC + 1]; g[k].c = p[PJ_CONIC + 2];
        g[k].o = p[PJ_OPAC];
        for (int c = 0; c < 3; ++c) g[k].rgb[c] = p[PJ_RGB + c];
    }
    free(ki);
    *m_out = m;
    return g;
}

/* ---------------------------------------------------------------- per-pixel blend */

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_MIN 1e-4

/* Offset from the Gaussian's centre to the pixel; for ERP views (W > 0) the horizontal part is
 * wrapped to [-W/2, W/2); pinhole views pass W = 0 (no wrap). */
static void pixel_offset(double px, double py, double u, double v, int W, double *dx, double *dy)
{
    double d = px - u;
    *dx = W > 0 ? d - (double)W * floor(d / (double)W + 0.5) : d;
    *dy = py - v;
}

/* One contributing Gaussian of a pixel, kept for the reverse pass. */
typedef struct {
    int k;                 /* index into the sorted list */
    double dx, dy, G, alpha, T; /* T = transmittance before this Gaussian */
    int clamped;
} contrib;

/* Eq. 2-3 at one pixel. margins[0] = min |ln(o G / (1/255))| over tested Gaussians,
 * margins[1] = min |ln(T' / 1e-4)| over the termination tests, margins[2] = min
 * |ln(o G / 0.99)| over contributing Gaussians; they let the tests flag pixels whose
 * discrete decisions sit within rounding of a threshold. */
static int blend_pixel(const sorted_g *g, int m, double px, double py, int W, const orc_settings *s,
                       double out[3], double *outT, double margins[3], contrib *list, int cap)
{
    double T = 1.0, C[3] = {0, 0, 0};
    double m0 = INFINITY, m1 = INFINITY, m2 = INFINITY;
    int nc = 0;
    for (int k = 0; k < m; ++k) {
        double dx, dy;
        pixel_offset(px, py, g[k].u, g[k].v, W, &dx, &dy);
        double power = -0.5 * (g[k].a * dx * dx + g[k].c * dy * dy) - g[k].b * dx * dy;
        double G = exp(power);
        double raw = g[k].o * G;
        if (raw > 0.0) {
            double lm = fabs(log(raw / ALPHA_MIN));
            if (lm < m0) m0 = lm;
        }
        double alpha = raw < ALPHA_MAX ? raw : ALPHA_MAX;
        if (alpha < ALPHA_MIN) continue;
        double Tn = T * (1.0 - alpha);
        double tm = fabs(log(Tn / T_MIN));
        if (tm < m1) m1 = tm;
        if (Tn < T_MIN) break;
        double cm = fabs(log(raw / ALPHA_MAX));
        if (cm < m2) m2 = cm;
        for (int c = 0; c < 3; ++c) C[c] += g[k].rgb[c] * alpha * T;
        if (list && nc < cap) {
            list[nc].k = k; list[nc].dx = dx; list[nc].dy = dy; list[nc].G = G;
            list[nc].alpha = alpha; list[nc].T = T; list[nc].clamped = raw >= ALPHA_MAX;
        }
        ++nc;
        T = Tn;
    }
    for (int c = 0; c < 3; ++c) out[c] = C[c] + T * s->bg[c];
    *outT = T;
    if (margins) { margins[0] = m0; margins[1] = m1; margins[2] = m2; }
    return nc;
}

/* Render the pixels listed in pix (flat y*W+x), or all pixels when pix == NULL.
 * color: [npix][3]; final_T, ncontrib: [npix]; margins: [npix][3] (may be NULL). */
int orc_render(int n, const double *means, const double *scales, const double *quats,
               const double *opacity, const double *sh, const orc_view *v, const orc_settings *s,
               int npix, const int32_t *pix, double *color, double *final_T, int32_t *ncontrib,
               double *margins)
{
    double *pj = (double *)malloc(sizeof(double) * PJ_NFIELDS * (size_t)(n > 0 ? n : 1));
    orc_project(n, means, scales, quats, opacity, sh, v, s, pj);
    int m;
    sorted_g *g = sort_visible(n, pj, &m);
    int total = pix ? npix : v->width * v->height;
#pragma omp parallel for schedule(dynamic, 8)
    for (int p = 0; p < total; ++p) {
        int flat = pix ? pix[p] : p;
        int x = flat % v->width, y = flat / v->width;
        double T;
        int nc = blend_pixel(g, m, x + s->pix_offset, y + s->pix_offset, v->model == 1 ? 0 : v->width, s,
                             color + 3 * (size_t)p,
                             &T, margins ? margins + 3 * (size_t)p : NULL, NULL, 0);
        final_T[p] = T;
        if (ncontrib) ncontrib[p] = nc;
    }
    free(g);
    free(pj);
    return 0;
}

/* ---------------------------------------------------------------- adjoint */

/* Per-Gaussian screen-space gradient accumulator layout. */
enum { G2_U = 0, G2_V, G2_A, G2_B, G2_C, G2_O, G2_R, G2_G, G2_BL, G2_N };

static void atomic_add(double *p, double x)
{
#pragma omp atomic
    *p += x;
}

/* Reverse pass of Eq. 3 at one pixel: accumulates dL/d(u, v, conic, opacity, rgb). With g2abs
 * non-NULL it also accumulates the absolute value of every pixel's contribution, the magnitude
 * that bounds the rounding error of any finite-precision evaluation of the same sums. */
static void add_contrib(double *acc, double *abs_acc, int c, double x)
{
    atomic_add(&acc[c], x);
    if (abs_acc) atomic_add(&abs_acc[c], fabs(x));
}

static void blend_pixel_adjoint(const sorted_g *g, int m, double px, double py, int W,
                                const orc_settings *s, const double *dLdC, double *g2, double *g2abs,
                                contrib *list, int cap)
{
    double out[3], Tf;
    int nc = blend_pixel(g, m, px, py, W, s, out, &Tf, NULL, list, cap);
    if (nc > cap) nc = cap; /* cap is sized to m, so this never truncates */
    /* B = colour blended behind the current Gaussian, including the background */
    double Bk[3] = {Tf * s->bg[0], Tf * s->bg[1], Tf * s->bg[2]};
    for (int q = nc - 1; q >= 0; --q) {
        const contrib *e = &list[q];
        const sorted_g *gk = &g[e->k];
        double a = e->alpha, T = e->T;
        double *acc = g2 + (size_t)G2_N * gk->id;
        double *aab = g2abs ? g2abs + (size_t)G2_N * gk->id : NULL;
        /* dC/drgb = alpha T */
        for (int c = 0; c < 3; ++c) add_contrib(acc, aab, G2_R + c, dLdC[c] * a * T);
        /* dC/dalpha = rgb T - B / (1 - alpha) */
        double dLda = 0.0;
        for (int c = 0; c < 3; ++c) dLda += dLdC[c] * (gk->rgb[c] * T - Bk[c] / (1.0 - a));
        for (int c = 0; c < 3; ++c) Bk[c] += gk->rgb[c] * a * T;
        if (e->clamped) continue; /* alpha = 0.99 does not depend on o or G */
        /* alpha = o G, G = exp(power) */
        add_contrib(acc, aab, G2_O, dLda * e->G);
        double dLdp = dLda * gk->o * e->G;
        double dx = e->dx, dy = e->dy;
        /* power = -(a dx^2 + c dy^2)/2 - b dx dy, dx = x - u, dy = y - v */
        add_contrib(acc, aab, G2_A, dLdp * (-0.5 * dx * dx));
        add_contrib(acc, aab, G2_B, dLdp * (-dx * dy));
        add_contrib(acc, aab, G2_C, dLdp * (-0.5 * dy * dy));
        add_contrib(acc, aab, G2_U, dLdp * (gk->a * dx + gk->b * dy));
        add_contrib(acc, aab, G2_V, dLdp * (gk->b * dx + gk->c * dy));
    }
}

/* Chain rule from the screen-space gradient of one Gaussian to its parameters (App. A.3). */
static void project_adjoint(const double *mean, const double *scale, const double *quat,
                            const double *sh, const orc_view *v, const orc_settings *s,
                            const double *pj, const double *g2, double *gm, double *gs, double *gq,
                            double *go, double *gsh)
{
    if (pj[PJ_VALID] == 0.0) return;
    const int W = v->width, H = v->height;
    double fx = (double)W / (2.0 * ORC_PI), fy = (double)H / ORC_PI;
    const double *J = pj + PJ_J;
    double A = pj[PJ_COV2], B = pj[PJ_COV2 + 1], C = pj[PJ_COV2 + 2];
    double D = A * C - B * B, D2 = D * D;

    *go += g2[G2_O];

    /* conic (a, b, c) = (C, -B, A) / D  ->  dL/d(A, B, C), B a single symmetric variable */
    double da = g2[G2_A], db = g2[G2_B], dc = g2[G2_C];
    double dA = da * (-C * C / D2) + db * (B * C / D2) + dc * (-B * B / D2);
    double dB = da * (2 * B * C / D2) + db * (-(A * C + B * B) / D2) + dc * (2 * A * B / D2);
    double dC = da * (-B * B / D2) + db * (A * B / D2) + dc * (-A * A / D2);

    /* T = J W; V = world Sigma */
    double T[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = J[3 * i] * v->R[j] + J[3 * i + 1] * v->R[3 + j] + J[3 * i + 2] * v->R[6 + j];
    const double *c3 = pj + PJ_COV3;
    double V[9] = {c3[0], c3[1], c3[2], c3[1], c3[3], c3[4], c3[2], c3[4], c3[5]};
    /* Eq. 11: dL/dT_1k = 2 (T_1 V)_k dA + (T_2 V)_k dB ; dL/dT_2k = 2 (T_2 V)_k dC + (T_1 V)_k dB */
    double T1V[3], T2V[3];
    for (int k = 0; k < 3; ++k) {
        T1V[k] = T[0] * V[k] + T[1] * V[3 + k] + T[2] * V[6 + k];
        T2V[k] = T[3] * V[k] + T[4] * V[3 + k] + T[5] * V[6 + k];
    }
    double dT[6];
    for (int k = 0; k < 3; ++k) {
        dT[k] = 2 * T1V[k] * dA + T2V[k] * dB;
        dT[3 + k] = 2 * T2V[k] * dC + T1V[k] * dB;
    }
    /* dL/dJ = dL/dT W^T */
    double dJ[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            dJ[3 * i + j] = dT[3 * i] * v->R[3 * j] + dT[3 * i + 1] * v->R[3 * j + 1] + dT[3 * i + 2] * v->R[3 * j + 2];
    /* dL/dSigma = T^T G T, G = [[dA, dB/2], [dB/2, dC]] */
    double G[4] = {dA, 0.5 * dB, 0.5 * dB, dC};
    double dSig[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) acc += T[3 * p + i] * G[2 * p + q] * T[3 * q + j];
            dSig[3 * i + j] = acc;
        }

    double dt[3];
    if (v->model == 1) {
        /* pinhole: u = fx tx/tz + cx, v = fy ty/tz + cy; J = [[fx/tz, 0, -fx tx/tz^2],
         * [0, fy/tz, -fy ty/tz^2]] (Eq. 1), differentiated w.r.t. t */
        const double *tp = pj + PJ_T;
        double tx = tp[0], ty = tp[1], tz = tp[2], iz = 1.0 / tz, iz2 = iz * iz, iz3 = iz2 * iz;
        double pfx = v->fx, pfy = v->fy;
        dt[0] = g2[G2_U] * pfx * iz - dJ[2] * pfx * iz2;
        dt[1] = g2[G2_V] * pfy * iz - dJ[5] * pfy * iz2;
        dt[2] = -g2[G2_U] * pfx * tx * iz2 - g2[G2_V] * pfy * ty * iz2 - dJ[0] * pfx * iz2
                + dJ[2] * 2.0 * pfx * tx * iz3 - dJ[4] * pfy * iz2 + dJ[5] * 2.0 * pfy * ty * iz3;
        goto have_dt;
    }
    /* J_omni as a function of (r, theta, phi):
     *   J11 = fx cos(phi) / (r cos(theta)), J13 = -fx sin(phi) / (r cos(theta)),
     *   J21 = fy sin(theta) sin(phi) / r, J22 = fy cos(theta) / r, J23 = fy sin(theta) cos(phi) / r */
    double r = pj[PJ_R], th = pj[PJ_THETA], ph = pj[PJ_PHI];
    double ct = cos(th), st = sin(th), cp = cos(ph), sp = sin(ph);
    double J11 = J[0], J13 = J[2], J21 = J[3], J22 = J[4], J23 = J[5];
    double dLdr = -(dJ[0] * J11 + dJ[2] * J13 + dJ[3] * J21 + dJ[4] * J22 + dJ[5] * J23) / r;
    double dLdth = dJ[0] * J11 * (st / ct) + dJ[2] * J13 * (st / ct) + dJ[3] * fy * ct * sp / r
                 - dJ[4] * fy * st / r + dJ[5] * fy * ct * cp / r;
    double dLdph = dJ[0] * J13 + dJ[2] * (-J11) + dJ[3] * J23 + dJ[5] * (-J21);
    /* mean path, Eq. 4: u = fx phi + W/2, v = -fy theta + H/2 */
    dLdph += g2[G2_U] * fx;
    dLdth += g2[G2_V] * (-fy);
    /* (r, theta, phi) as functions of t */
    const double *t = pj + PJ_T;
    double rho2 = t[0] * t[0] + t[2] * t[2], rho = sqrt(rho2), r2 = r * r;
    double drdt[3] = {t[0] / r, t[1] / r, t[2] / r};
    double dphdt[3] = {t[2] / rho2, 0.0, -t[0] / rho2};
    double dthdt[3] = {t[0] * t[1] / (r2 * rho), -rho / r2, t[2] * t[1] / (r2 * rho)};
    for (int k = 0; k < 3; ++k) dt[k] = dLdr * drdt[k] + dLdth * dthdt[k] + dLdph * dphdt[k];
have_dt:
    /* t = W mu + t_wc  ->  dL/dmu = W^T dL/dt */
    for (int j = 0; j < 3; ++j) gm[j] += v->R[j] * dt[0] + v->R[3 + j] * dt[1] + v->R[6 + j] * dt[2];

    /* colour: rgb_c = max(0, sum_k sh_kc Y_k(d) + 0.5) */
    double cam[3];
    for (int j = 0; j < 3; ++j) cam[j] = -(v->R[j] * v->t[0] + v->R[3 + j] * v->t[1] + v->R[6 + j] * v->t[2]);
    double dv[3] = {mean[0] - cam[0], mean[1] - cam[1], mean[2] - cam[2]};
    double sxy2 = dv[0] * dv[0] + dv[1] * dv[1], sxy = sqrt(sxy2);
    double n2 = sxy2 + dv[2] * dv[2];
    double nn = sqrt(n2), vp = atan2(dv[1], dv[0]);
    double Y[16], dYt[16], dYp[16];
    sh_basis(s->sh_degree, dv[2] / nn, sxy / nn, vp, Y, dYt, dYp);
    int K = (s->sh_degree + 1) * (s->sh_degree + 1);
    double dLdvt = 0.0, dLdvp = 0.0;
    for (int c = 0; c < 3; ++c) {
        if (pj[PJ_CLAMP + c] != 0.0) continue;
        double gc = g2[G2_R + c];
        for (int k = 0; k < K; ++k) {
            gsh[3 * k + c] += gc * Y[k];
            dLdvt += gc * sh[3 * k + c] * dYt[k];
            dLdvp += gc * sh[3 * k + c] * dYp[k];
        }
    }
    if (sxy > 1e-100 * nn) {
        /* vt = atan2(sqrt(x^2 + y^2), z), vp = atan2(y, x) of the unnormalised direction */
        double dvtdv[3] = {dv[0] * dv[2] / (n2 * sxy), dv[1] * dv[2] / (n2 * sxy), -sxy / n2};
        double dvpdv[3] = {-dv[1] / sxy2, dv[0] / sxy2, 0.0};
        for (int j = 0; j < 3; ++j) gm[j] += dLdvt * dvtdv[j] + dLdvp * dvpdv[j];
    } else {
        /* direction on the z axis (to 1e-100), where the (vt, vp) chart is singular. The colour
         * is smooth on the sphere, so its gradient there is the limit along +x (vp = 0) and
         * along +y (vp = pi/2); at either pole d vt / dx = d vt / dy = 1 / z, and moving along z
         * leaves the direction unchanged. */
        double Yq[16], dYtq[16], dYpq[16];
        for (int a = 0; a < 2; ++a) {
            sh_basis(s->sh_degree, dv[2] > 0.0 ? 1.0 : -1.0, 0.0, a == 0 ? 0.0 : 0.5 * ORC_PI, Yq, dYtq, dYpq);
            double D = 0.0;
            for (int c = 0; c < 3; ++c) {
                if (pj[PJ_CLAMP + c] != 0.0) continue;
                for (int k = 0; k < K; ++k) D += g2[G2_R + c] * sh[3 * k + c] * dYtq[k];
            }
            gm[a] += D / dv[2];
        }
    }

    /* Sigma = M M^T, M = R diag(s)  ->  dL/dM = (dSig + dSig^T) M */
    double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    double q[4] = {quat[0] / qn, quat[1] / qn, quat[2] / qn, quat[3] / qn};
    double R[9], M[9];
    quat_to_rot(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * scale[j];
    double dM[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += (dSig[3 * i + k] + dSig[3 * k + i]) * M[3 * k + j];
            dM[3 * i + j] = acc;
        }
    double dR[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            gs[j] += dM[3 * i + j] * R[3 * i + j];
            dR[3 * i + j] = dM[3 * i + j] * scale[j];
        }
    double P[4][9];
    quat_to_rot_partials(q, P);
    double dqn[4];
    for (int k = 0; k < 4; ++k) {
        double acc = 0;
        for (int e = 0; e < 9; ++e) acc += dR[e] * P[k][e];
        dqn[k] = acc;
    }
    /* q_hat = q / |q| */
    double qd = q[0] * dqn[0] + q[1] * dqn[1] + q[2] * dqn[2] + q[3] * dqn[3];
    for (int k = 0; k < 4; ++k) gq[k] += (dqn[k] - q[k] * qd) / qn;
}

/* Adjoint of orc_render for a loss with dL/dcolor given at the listed pixels.
 * Gradients are ACCUMULATED into gm [n][3], gs [n][3], gq [n][4], go [n], gsh [n][K][3].
 * g2_out (optional) receives the per-Gaussian screen-space gradient [n][9], g2abs_out (optional)
 * the sum over pixels of the absolute values of its contributions [n][9]. */
int orc_backward(int n, const double *means, const double *scales, const double *quats,
                 const double *opacity, const double *sh, const orc_view *v, const orc_settings *s,
                 int npix, const int32_t *pix, const double *dLdC, double *gm, double *gs, double *gq,
                 double *go, double *gsh, double *g2_out, double *g2abs_out)
{
    double *pj = (double *)malloc(sizeof(double) * PJ_NFIELDS * (size_t)(n > 0 ? n : 1));
    orc_project(n, means, scales, quats, opacity, sh, v, s, pj);
    int m;
    sorted_g *g = sort_visible(n, pj, &m);
    double *g2 = (double *)calloc((size_t)G2_N * (n > 0 ? n : 1), sizeof(double));
    double *g2abs = g2abs_out ? (double *)calloc((size_t)G2_N * (n > 0 ? n : 1), sizeof(double)) : NULL;
    int total = pix ? npix : v->width * v->height;
#pragma omp parallel
    {
        contrib *list = (contrib *)malloc(sizeof(contrib) * (m > 0 ? m : 1));
#pragma omp for schedule(dynamic, 8)
        for (int p = 0; p < total; ++p) {
            const double *d = dLdC + 3 * (size_t)p;
            if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) continue;
            int flat = pix ? pix[p] : p;
            int x = flat % v->width, y = flat / v->width;
            blend_pixel_adjoint(g, m, x + s->pix_offset, y + s->pix_offset, v->model == 1 ? 0 : v->width, s, d, g2,
                                g2abs, list, m);
        }
        free(list);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        project_adjoint(means + 3 * i, scales + 3 * i, quats + 4 * i, sh + (size_t)3 * s->sh_coeffs * i, v, s,
                        pj + (size_t)PJ_NFIELDS * i, g2 + (size_t)G2_N * i, gm + 3 * i, gs + 3 * i, gq + 4 * i,
                        go + i, gsh + (size_t)3 * s->sh_coeffs * i);
    if (g2_out) memcpy(g2_out, g2, sizeof(double) * G2_N * (size_t)n);
    if (g2abs_out) memcpy(g2abs_out, g2abs, sizeof(double) * G2_N * (size_t)n);
    free(g2abs);
    free(g2);
    free(g);
    free(pj);
    return 0;
}

/* The chain rule alone (App. A.3): parameter gradients from given per-Gaussian screen-space
 * gradients g2 [n][9] (dL/du, dL/dv, dL/da, dL/db, dL/dc, dL/do, dL/dr, dL/dg, dL/db) of one view,
 * ACCUMULATED into gm, gs, gq, go, gsh as in orc_backward. It lets a test feed the same
 * screen-space gradients to two chain-rule implementations. */
int orc_chain(int n, const double *means, const double *scales, const double *quats, const double *opacity,
              const double *sh, const orc_view *v, const orc_settings *s, const double *g2, double *gm,
              double *gs, double *gq, double *go, double *gsh)
{
    double *pj = (double *)malloc(sizeof(double) * PJ_NFIELDS * (size_t)(n > 0 ? n : 1));
    orc_project(n, means, scales, quats, opacity, sh, v, s, pj);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        project_adjoint(means + 3 * i, scales + 3 * i, quats + 4 * i, sh + (size_t)3 * s->sh_coeffs * i, v, s,
                        pj + (size_t)PJ_NFIELDS * i, g2 + (size_t)G2_N * i, gm + 3 * i, gs + 3 * i, gq + 4 * i,
                        go + i, gsh + (size_t)3 * s->sh_coeffs * i);
    free(pj);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
