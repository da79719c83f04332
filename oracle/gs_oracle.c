/*
 * gs_oracle.c -- FP64 CPU oracle of the Turbo-GS dilated 3DGS rasterizer hot path.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load it; the product path never does. It is written
 * for a reader checking it against the paper by eye: one Gaussian or one
 * pixel at a time, in double precision, no blocking or fusion beyond what the
 * method states. OpenMP only splits independent Gaussians / tiles.
 *
 * Constants that the paper does not print are readings (each one is marked
 * "reading:" below):
 *   low-pass term 0.3 px^2 added to the 2D covariance diagonal (Sec. 3.1 says a
 *   low-pass filter "following 3DGS"); the 0.1 floor under the eigenvalue
 *   discriminant; alpha clamp 0.99, alpha skip 1/255 and transmittance stop 1e-4
 *   (the early-stop rule); Jacobian clamp at 1.3 x the half field of view.
 */
#include "gs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* reading: low-pass term of the 2D covariance (hr px^2) */
static const double LOWPASS = 0.3;
/* reading: floor of the discriminant in the largest-eigenvalue formula */
static const double DISC_FLOOR = 0.1;
/* early-stop rule: alpha < 1/255 is skipped, alpha is clamped to 0.99, and the
 * walk stops before an entry that would take transmittance below 1e-4 */
static const double ALPHA_MIN = 1.0 / 255.0;
static const double ALPHA_MAX = 0.99;
static const double T_STOP = 1e-4;
/* reading: t_x/t_z and t_y/t_z are clamped to 1.3 x the half field of view
 * before the Jacobian is formed */
static const double CLAMP_FOV = 1.3;

/* margins for ambiguity flags (FP32 rounding of the GPU path stays far below) */
static const double MARGIN_RADIUS = 1e-5;   /* relative, on 3 sqrt(lambda) */
static const double MARGIN_RECT = 2e-4;     /* absolute, in tile units */
static const double MARGIN_REL = 1e-5;      /* relative, generic */
static const double MARGIN_ALPHA = 1e-4;    /* relative, alpha gates */
static const double MARGIN_TSTOP = 1e-3;    /* relative, transmittance stop */

static int ceil_div(int a, int b) { return (a + b - 1) / b; }

void orc_grid(const OrcCamera* cam, const OrcDilation* dil,
              int32_t* w_ds, int32_t* h_ds, int32_t* tiles_x, int32_t* tiles_y)
{
    /* Sec. 3.1: the d*d offsets partition the hr image, so the rendered lattice
     * for offset o has ceil((W - o)/d) columns (reading for d not dividing W). */
    int w = ceil_div(cam->width - dil->ox, dil->d);
    int h = ceil_div(cam->height - dil->oy, dil->d);
    if (w_ds) *w_ds = w;
    if (h_ds) *h_ds = h;
    if (tiles_x) *tiles_x = ceil_div(w, dil->tile);
    if (tiles_y) *tiles_y = ceil_div(h, dil->tile);
}

/* ------------------------------------------------------------------------- */
/* Spherical harmonics (Sec. 3: view-dependent colour from SH coefficients).  */
/* Real SH from the associated Legendre recurrence with Condon-Shortley phase: */
/*   Y_l0 = K_l0 Q_l^0(z),                                                    */
/*   Y_lm = sqrt2 K_lm Q_l^m(z) Re((x+iy)^m),  Y_l,-m = ... Im((x+iy)^m),     */
/*   K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),                                */
/* where Q_l^m = P_l^m / (1 - z^2)^{m/2} is a polynomial in z. The derivative */
/* with respect to (x, y, z) is carried along (forward mode).                 */
/* ------------------------------------------------------------------------- */

#define ORC_MAX_DEG 3
#define ORC_MAX_COEFS ((ORC_MAX_DEG + 1) * (ORC_MAX_DEG + 1))

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* val[k] = Y_k(x, y, z); grad[3k + j] = dY_k/d(x, y, z)_j (grad nullable). */
static void sh_basis_grad(int deg, double x, double y, double z, double* val, double* grad)
{
    /* C_m + i S_m = (x + i y)^m with partial derivatives */
    double C[ORC_MAX_DEG + 1], S[ORC_MAX_DEG + 1];
    double dC[ORC_MAX_DEG + 1][2], dS[ORC_MAX_DEG + 1][2];  /* d/dx, d/dy */
    C[0] = 1.0; S[0] = 0.0;
    dC[0][0] = dC[0][1] = dS[0][0] = dS[0][1] = 0.0;
    for (int m = 1; m <= deg; ++m) {
        C[m] = C[m - 1] * x - S[m - 1] * y;
        S[m] = S[m - 1] * x + C[m - 1] * y;
        dC[m][0] = C[m - 1] + x * dC[m - 1][0] - y * dS[m - 1][0];
        dC[m][1] = x * dC[m - 1][1] - S[m - 1] - y * dS[m - 1][1];
        dS[m][0] = S[m - 1] + x * dS[m - 1][0] + y * dC[m - 1][0];
        dS[m][1] = x * dS[m - 1][1] + C[m - 1] + y * dC[m - 1][1];
    }
    for (int m = 0; m <= deg; ++m) {
        /* Q_m^m = (-1)^m (2m-1)!!, Q_{m+1}^m = (2m+1) z Q_m^m,
         * (l-m) Q_l^m = (2l-1) z Q_{l-1}^m - (l+m-1) Q_{l-2}^m */
        double q_prev2 = 0.0, dq_prev2 = 0.0;
        double dfact = 1.0;
        for (int i = 1; i <= 2 * m - 1; i += 2) dfact *= i;
        double q_prev = (m % 2 ? -1.0 : 1.0) * dfact, dq_prev = 0.0;
        for (int l = m; l <= deg; ++l) {
            double q, dq;
            if (l == m) {
                q = q_prev; dq = dq_prev;
            } else if (l == m + 1) {
                q = (2 * m + 1) * z * q_prev;
                dq = (2 * m + 1) * (q_prev + z * dq_prev);
                q_prev2 = q_prev; dq_prev2 = dq_prev;
                q_prev = q; dq_prev = dq;
            } else {
                q = ((2 * l - 1) * z * q_prev - (l + m - 1) * q_prev2) / (l - m);
                dq = ((2 * l - 1) * (q_prev + z * dq_prev) - (l + m - 1) * dq_prev2) / (l - m);
                q_prev2 = q_prev; dq_prev2 = dq_prev;
                q_prev = q; dq_prev = dq;
            }
            double K = sqrt((2 * l + 1) / (4.0 * ORC_PI) * factorial(l - m) / factorial(l + m));
            if (m == 0) {
                int k = l * l + l;
                val[k] = K * q;
                if (grad) { grad[3 * k] = 0.0; grad[3 * k + 1] = 0.0; grad[3 * k + 2] = K * dq; }
            } else {
                double c = sqrt(2.0) * K;
                int kp = l * l + l + m, kn = l * l + l - m;
                val[kp] = c * q * C[m];
                val[kn] = c * q * S[m];
                if (grad) {
                    grad[3 * kp] = c * q * dC[m][0];
                    grad[3 * kp + 1] = c * q * dC[m][1];
                    grad[3 * kp + 2] = c * dq * C[m];
                    grad[3 * kn] = c * q * dS[m][0];
                    grad[3 * kn + 1] = c * q * dS[m][1];
                    grad[3 * kn + 2] = c * dq * S[m];
                }
            }
        }
    }
}

void orc_sh_basis(int32_t deg, const double dir[3], double* out)
{
    sh_basis_grad(deg, dir[0], dir[1], dir[2], out, NULL);
}

/* ------------------------------------------------------------------------- */
/* Projection (Sec. 3 covariance, Sec. 3.1 projection and dilated binning).   */
/* ------------------------------------------------------------------------- */

/* Rotation matrix of the unit quaternion (w, x, y, z), row-major. */
static void quat_to_rot(double w, double x, double y, double z, double R[9])
{
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static double near_int_dist(double v) { return fabs(v - nearbyint(v)); }

/* Everything the forward projection of one Gaussian produces, kept for the
 * backward pass which recomputes it. */
typedef struct {
    int culled;
    double s[3], qn[4], qnorm, Rq[9], M[9], Sigma[9];
    double t[3], u, v, uc, vc;
    int clamp_x, clamp_y;
    double J[6], Tm[6];
    double a, b, c, det;
    double conic[3];
    double lambda, r3;
    int radius;
    double p[2];
    double dir[3], vlen, vvec[3];
    double basis[ORC_MAX_COEFS];
    double rgb_raw[3], rgb[3];
    double opacity;
    int rect[4];
    int64_t tiles;
    uint32_t flags;
} OrcProj;

static void project_one(const OrcCamera* cam, const OrcDilation* dil, int deg,
                        const double* mean, const double* log_scale, const double* quat,
                        double opacity_logit, const double* sh, OrcProj* P)
{
    memset(P, 0, sizeof(*P));
    int ncoef = (deg + 1) * (deg + 1);

    /* activations: s = exp(log s), unit quaternion, sigmoid opacity */
    for (int j = 0; j < 3; ++j) P->s[j] = exp(log_scale[j]);
    P->qnorm = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    if (!(P->qnorm > 0.0)) { P->culled = 1; P->flags |= ORC_FLAG_CULLED; return; }
    for (int j = 0; j < 4; ++j) P->qn[j] = quat[j] / P->qnorm;
    P->opacity = 1.0 / (1.0 + exp(-opacity_logit));

    /* Sigma = R S S^T R^T with M = R S */
    quat_to_rot(P->qn[0], P->qn[1], P->qn[2], P->qn[3], P->Rq);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[3 * i + j] = P->Rq[3 * i + j] * P->s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P->M[3 * i + k] * P->M[3 * j + k];
            P->Sigma[3 * i + j] = acc;
        }

    /* camera space; near-plane cull (reading: t_z <= z_near is culled) */
    for (int i = 0; i < 3; ++i)
        P->t[i] = cam->R[3 * i] * mean[0] + cam->R[3 * i + 1] * mean[1] + cam->R[3 * i + 2] * mean[2] + cam->T[i];
    if (fabs(P->t[2] - cam->z_near) < MARGIN_REL * fabs(cam->z_near) + 1e-12) P->flags |= ORC_FLAG_NEAR;
    if (P->t[2] <= cam->z_near) { P->culled = 1; P->flags |= ORC_FLAG_CULLED; return; }
    double tz = P->t[2];

    /* Jacobian of the perspective map with the hr (original) focal lengths,
     * with the clamped view-space tangent (reading) */
    double limx = CLAMP_FOV * 0.5 * cam->width / cam->fx;
    double limy = CLAMP_FOV * 0.5 * cam->height / cam->fy;
    P->u = P->t[0] / tz;
    P->v = P->t[1] / tz;
    P->clamp_x = fabs(P->u) > limx;
    P->clamp_y = fabs(P->v) > limy;
    P->uc = P->clamp_x ? (P->u > 0 ? limx : -limx) : P->u;
    P->vc = P->clamp_y ? (P->v > 0 ? limy : -limy) : P->v;
    if (fabs(fabs(P->u) - limx) < MARGIN_REL * limx || fabs(fabs(P->v) - limy) < MARGIN_REL * limy)
        P->flags |= ORC_FLAG_CLAMP;
    double txc = P->uc * tz, tyc = P->vc * tz;
    P->J[0] = cam->fx / tz; P->J[1] = 0.0;           P->J[2] = -cam->fx * txc / (tz * tz);
    P->J[3] = 0.0;          P->J[4] = cam->fy / tz;  P->J[5] = -cam->fy * tyc / (tz * tz);

    /* Sigma' = J W Sigma W^T J^T + low-pass */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P->J[3 * i + k] * cam->R[3 * k + j];
            P->Tm[3 * i + j] = acc;
        }
    double S2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += P->Tm[3 * i + k] * P->Sigma[3 * k + l] * P->Tm[3 * j + l];
            S2[2 * i + j] = acc;
        }
    P->a = S2[0] + LOWPASS;
    P->b = 0.5 * (S2[1] + S2[2]);
    P->c = S2[3] + LOWPASS;
    P->det = P->a * P->c - P->b * P->b;
    if (!(P->det > 0.0)) { P->culled = 1; P->flags |= ORC_FLAG_CULLED; return; }
    P->conic[0] = P->c / P->det;
    P->conic[1] = -P->b / P->det;
    P->conic[2] = P->a / P->det;

    /* 3-sigma radius in hr pixels from the largest eigenvalue */
    double mid = 0.5 * (P->a + P->c);
    double disc = mid * mid - P->det;
    P->lambda = mid + sqrt(disc > DISC_FLOOR ? disc : DISC_FLOOR);
    P->r3 = 3.0 * sqrt(P->lambda);
    P->radius = (int)ceil(P->r3);
    if (near_int_dist(P->r3) < MARGIN_RADIUS * P->r3) P->flags |= ORC_FLAG_RADIUS;

    /* hr image-plane centre (unclamped) */
    P->p[0] = cam->fx * P->u + cam->cx;
    P->p[1] = cam->fy * P->v + cam->cy;

    /* downsampled centre and radius (Eq. 3-4); reading: lattice-aligned centre
     * (p - o)/d by default, (p - (d-1)/2)/d in the paper-literal mode */
    double d = dil->d;
    double pdx, pdy;
    if (dil->center_mode == 0) {
        pdx = (P->p[0] - dil->ox) / d;
        pdy = (P->p[1] - dil->oy) / d;
    } else {
        pdx = (P->p[0] - 0.5 * (d - 1)) / d;
        pdy = (P->p[1] - 0.5 * (d - 1)) / d;
    }
    double rds = P->radius / d;
    int tiles_x, tiles_y;
    orc_grid(cam, dil, NULL, NULL, &tiles_x, &tiles_y);
    /* reading: tile tx is touched iff [pdx - rds, pdx + rds] meets
     * [tile*tx, tile*(tx+1)), i.e. tx in [floor((pdx-rds)/tile), floor((pdx+rds)/tile)] */
    double bx0 = (pdx - rds) / dil->tile, bx1 = (pdx + rds) / dil->tile;
    double by0 = (pdy - rds) / dil->tile, by1 = (pdy + rds) / dil->tile;
    if (near_int_dist(bx0) < MARGIN_RECT || near_int_dist(bx1) < MARGIN_RECT ||
        near_int_dist(by0) < MARGIN_RECT || near_int_dist(by1) < MARGIN_RECT)
        P->flags |= ORC_FLAG_RECT;
    double fx0 = floor(bx0), fx1 = floor(bx1), fy0 = floor(by0), fy1 = floor(by1);
    if (fx0 < 0) fx0 = 0;
    if (fy0 < 0) fy0 = 0;
    if (fx1 > tiles_x - 1) fx1 = tiles_x - 1;
    if (fy1 > tiles_y - 1) fy1 = tiles_y - 1;
    if (P->radius <= 0 || fx0 > fx1 || fy0 > fy1) {
        P->culled = 1; P->flags |= ORC_FLAG_CULLED;
        P->rect[0] = 0; P->rect[1] = 0; P->rect[2] = -1; P->rect[3] = -1;
        return;
    }
    P->rect[0] = (int)fx0; P->rect[1] = (int)fy0; P->rect[2] = (int)fx1; P->rect[3] = (int)fy1;
    P->tiles = (int64_t)(fx1 - fx0 + 1) * (int64_t)(fy1 - fy0 + 1);

    /* view-dependent colour: dir = normalize(mean - camera centre), rgb =
     * max(0, sum_k Y_k(dir) sh_k + 0.5) (reading: the +0.5 offset and clamp) */
    double cc[3];
    for (int j = 0; j < 3; ++j)
        cc[j] = -(cam->R[j] * cam->T[0] + cam->R[3 + j] * cam->T[1] + cam->R[6 + j] * cam->T[2]);
    for (int j = 0; j < 3; ++j) P->vvec[j] = mean[j] - cc[j];
    P->vlen = sqrt(P->vvec[0] * P->vvec[0] + P->vvec[1] * P->vvec[1] + P->vvec[2] * P->vvec[2]);
    for (int j = 0; j < 3; ++j) P->dir[j] = P->vvec[j] / P->vlen;
    sh_basis_grad(deg, P->dir[0], P->dir[1], P->dir[2], P->basis, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < ncoef; ++k) acc += P->basis[k] * sh[3 * k + ch];
        P->rgb_raw[ch] = acc + 0.5;
        P->rgb[ch] = P->rgb_raw[ch] > 0.0 ? P->rgb_raw[ch] : 0.0;
        if (fabs(P->rgb_raw[ch]) < MARGIN_REL) P->flags |= ORC_FLAG_RGB;
    }
}

int64_t orc_project(int32_t n, int32_t sh_degree,
                    const double* means, const double* log_scales, const double* quats,
                    const double* opacity_logits, const double* sh,
                    const OrcCamera* cam, const OrcDilation* dil,
                    double* xy, double* conic, double* opacity, double* rgb, double* depth,
                    double* cov2d, int32_t* radius, int32_t* rect, int64_t* tiles_touched,
                    uint32_t* flags)
{
    int ncoef = (sh_degree + 1) * (sh_degree + 1);
    int64_t visible = 0;
#pragma omp parallel for schedule(static) reduction(+ : visible)
    for (int32_t i = 0; i < n; ++i) {
        OrcProj P;
        project_one(cam, dil, sh_degree, means + 3 * (int64_t)i, log_scales + 3 * (int64_t)i,
                    quats + 4 * (int64_t)i, opacity_logits[i], sh + (int64_t)i * ncoef * 3, &P);
        if (xy) { xy[2 * (int64_t)i] = P.p[0]; xy[2 * (int64_t)i + 1] = P.p[1]; }
        if (conic) for (int j = 0; j < 3; ++j) conic[3 * (int64_t)i + j] = P.conic[j];
        if (opacity) opacity[i] = P.opacity;
        if (rgb) for (int j = 0; j < 3; ++j) rgb[3 * (int64_t)i + j] = P.rgb[j];
        if (depth) depth[i] = P.t[2];
        if (cov2d) { cov2d[3 * (int64_t)i] = P.a; cov2d[3 * (int64_t)i + 1] = P.b; cov2d[3 * (int64_t)i + 2] = P.c; }
        if (radius) radius[i] = P.culled ? 0 : P.radius;
        if (rect) {
            if (P.culled) { rect[4 * (int64_t)i] = 0; rect[4 * (int64_t)i + 1] = 0; rect[4 * (int64_t)i + 2] = -1; rect[4 * (int64_t)i + 3] = -1; }
            else for (int j = 0; j < 4; ++j) rect[4 * (int64_t)i + j] = P.rect[j];
        }
        if (tiles_touched) tiles_touched[i] = P.culled ? 0 : P.tiles;
        if (flags) flags[i] = P.flags;
        if (!P.culled) visible += 1;
    }
    return visible;
}

/* ------------------------------------------------------------------------- */
/* Binning: tile|depth keys, sort, ranges (Sec. 3 tile-based rasterizer).     */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t key; uint32_t val; } OrcPair;

static int cmp_pair(const void* pa, const void* pb)
{
    const OrcPair* a = (const OrcPair*)pa;
    const OrcPair* b = (const OrcPair*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

int64_t orc_bin(int32_t n, const int32_t* rect, const int64_t* tiles_touched,
                const uint32_t* depth_bits, int32_t tiles_x, int32_t tiles_y,
                uint64_t* keys, uint32_t* vals, uint32_t* ranges)
{
    int64_t total = 0;
    for (int32_t i = 0; i < n; ++i) total += tiles_touched[i];
    OrcPair* pairs = (OrcPair*)malloc((size_t)(total > 0 ? total : 1) * sizeof(OrcPair));
    int64_t k = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (tiles_touched[i] <= 0) continue;
        const int32_t* rc = rect + 4 * (int64_t)i;
        for (int ty = rc[1]; ty <= rc[3]; ++ty)
            for (int tx = rc[0]; tx <= rc[2]; ++tx) {
                uint64_t tile_id = (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
                pairs[k].key = (tile_id << 32) | (uint64_t)depth_bits[i];
                pairs[k].val = (uint32_t)i;
                ++k;
            }
    }
    qsort(pairs, (size_t)k, sizeof(OrcPair), cmp_pair);
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    for (int64_t t = 0; t < 2 * ntiles; ++t) ranges[t] = 0;
    for (int64_t j = 0; j < k; ++j) {
        keys[j] = pairs[j].key;
        vals[j] = pairs[j].val;
        uint64_t tile = pairs[j].key >> 32;
        if (j == 0 || (pairs[j - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)j;
        if (j == k - 1 || (pairs[j + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(j + 1);
    }
    free(pairs);
    return k;
}

int64_t orc_bin_tiles(int32_t n, const int32_t* rect, const uint32_t* depth_bits,
                      int32_t tiles_x, int32_t n_tiles, const int32_t* tile_ids,
                      uint32_t* vals, uint32_t* ranges)
{
    int64_t* counts = (int64_t*)calloc((size_t)(n_tiles > 0 ? n_tiles : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t k = 0; k < n_tiles; ++k) {
        int tx = tile_ids[k] % tiles_x, ty = tile_ids[k] / tiles_x;
        int64_t c = 0;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t* rc = rect + 4 * (int64_t)i;
            if (rc[2] < rc[0]) continue;
            if (tx >= rc[0] && tx <= rc[2] && ty >= rc[1] && ty <= rc[3]) ++c;
        }
        counts[k] = c;
    }
    int64_t total = 0;
    for (int32_t k = 0; k < n_tiles; ++k) total += counts[k];
    if (vals) {
        int64_t start = 0;
        for (int32_t k = 0; k < n_tiles; ++k) {
            ranges[2 * k] = (uint32_t)start;
            ranges[2 * k + 1] = (uint32_t)(start + counts[k]);
            start += counts[k];
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t k = 0; k < n_tiles; ++k) {
            int tx = tile_ids[k] % tiles_x, ty = tile_ids[k] / tiles_x;
            OrcPair* pairs = (OrcPair*)malloc((size_t)(counts[k] > 0 ? counts[k] : 1) * sizeof(OrcPair));
            int64_t c = 0;
            for (int32_t i = 0; i < n; ++i) {
                const int32_t* rc = rect + 4 * (int64_t)i;
                if (rc[2] < rc[0]) continue;
                if (tx >= rc[0] && tx <= rc[2] && ty >= rc[1] && ty <= rc[3]) {
                    pairs[c].key = depth_bits[i];
                    pairs[c].val = (uint32_t)i;
                    ++c;
                }
            }
            qsort(pairs, (size_t)c, sizeof(OrcPair), cmp_pair);
            for (int64_t j = 0; j < c; ++j) vals[ranges[2 * k] + j] = pairs[j].val;
            free(pairs);
        }
    } else if (ranges) {
        for (int32_t k = 0; k < n_tiles; ++k) { ranges[2 * k] = 0; ranges[2 * k + 1] = (uint32_t)counts[k]; }
    }
    free(counts);
    return total;
}

/* ------------------------------------------------------------------------- */
/* Blending (Eq. 2) of the strided hr pixels of the downsampled image (Eq. 5). */
/* ------------------------------------------------------------------------- */

/* One blended entry of a pixel, kept for the backward pass. */
typedef struct { uint32_t g; double alpha, T, G, dx, dy; int clamped; } OrcBlend;

/* Walk one pixel front to back. Returns the number of blended entries written
 * to blend (capacity cap); outputs colour, final transmittance, last position,
 * ambiguity and counts. */
static int64_t blend_pixel(double x, double y, const double* xy, const double* conic,
                           const double* opacity, const double* rgb, const double* depth,
                           const uint32_t* vals, uint32_t start, uint32_t end, const double bg[3],
                           double C[3], double* T_out, uint32_t* last_out, int* amb,
                           uint64_t* n_eval, uint64_t* n_blend, OrcBlend* blend)
{
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    uint32_t last = 0;
    int64_t nb = 0;
    double prev_depth = -1.0;
    *amb = 0;
    for (uint32_t j = start; j < end; ++j) {
        uint32_t g = vals[j];
        ++*n_eval;
        double dx = x - xy[2 * (int64_t)g], dy = y - xy[2 * (int64_t)g + 1];
        const double* q = conic + 3 * (int64_t)g;
        double power = -0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy;
        if (power > 0.0) continue;
        double G = exp(power);
        double a_raw = opacity[g] * G;
        double alpha = a_raw < ALPHA_MAX ? a_raw : ALPHA_MAX;
        if (fabs(a_raw - ALPHA_MIN) < MARGIN_ALPHA * ALPHA_MIN) *amb = 1;
        if (fabs(a_raw - ALPHA_MAX) < MARGIN_ALPHA * ALPHA_MAX) *amb = 1;
        if (alpha < ALPHA_MIN) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - T_STOP) < MARGIN_TSTOP * T_STOP) *amb = 1;
        if (Tn < T_STOP) break;
        /* equal FP32 depth keys are ordered by index; near-equal ones may
         * reorder under FP32 projection, which changes the blend */
        if (depth && prev_depth >= 0.0 && fabs(depth[g] - prev_depth) < 1e-6 * prev_depth) *amb = 1;
        if (depth) prev_depth = depth[g];
        if (blend) {
            blend[nb].g = g; blend[nb].alpha = alpha; blend[nb].T = T; blend[nb].G = G;
            blend[nb].dx = dx; blend[nb].dy = dy; blend[nb].clamped = !(a_raw < ALPHA_MAX);
        }
        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * (int64_t)g + ch] * alpha * T;
        T = Tn;
        last = j - start + 1;
        ++nb;
        ++*n_blend;
    }
    for (int ch = 0; ch < 3; ++ch) C[ch] += T * bg[ch];
    *T_out = T;
    *last_out = last;
    return nb;
}

static void tile_of(int32_t k, int32_t n_tiles, const int32_t* tile_ids, const uint32_t* ranges,
                    int32_t* tile, uint32_t* start, uint32_t* end)
{
    (void)n_tiles;
    int32_t t = tile_ids ? tile_ids[k] : k;
    *tile = t;
    *start = ranges[2 * (int64_t)k];
    *end = ranges[2 * (int64_t)k + 1];
}

void orc_render_fwd(const double* xy, const double* conic, const double* opacity,
                    const double* rgb, const double* depth,
                    const uint32_t* vals, const uint32_t* ranges,
                    int32_t n_tiles, const int32_t* tile_ids,
                    const OrcCamera* cam, const OrcDilation* dil, const double bg[3],
                    double* img, double* t_final, uint32_t* last, uint8_t* ambiguous,
                    uint64_t* counts)
{
    int32_t w_ds, h_ds, tiles_x, tiles_y;
    orc_grid(cam, dil, &w_ds, &h_ds, &tiles_x, &tiles_y);
    int32_t nt = tile_ids ? n_tiles : tiles_x * tiles_y;
    uint64_t tot_eval = 0, tot_blend = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : tot_eval, tot_blend)
    for (int32_t k = 0; k < nt; ++k) {
        int32_t tile; uint32_t start, end;
        tile_of(k, nt, tile_ids, ranges, &tile, &start, &end);
        int tx = tile % tiles_x, ty = tile / tiles_x;
        for (int v = ty * dil->tile; v < (ty + 1) * dil->tile && v < h_ds; ++v)
            for (int u = tx * dil->tile; u < (tx + 1) * dil->tile && u < w_ds; ++u) {
                /* Eq. 5 / Sec. 3.1: ds pixel (u, v) is the hr pixel (d u + ox, d v + oy) */
                double x = (double)dil->d * u + dil->ox, y = (double)dil->d * v + dil->oy;
                double C[3], T; uint32_t lst; int amb;
                uint64_t ne = 0, nb = 0;
                blend_pixel(x, y, xy, conic, opacity, rgb, depth, vals, start, end, bg,
                            C, &T, &lst, &amb, &ne, &nb, NULL);
                int64_t pix = (int64_t)v * w_ds + u;
                for (int ch = 0; ch < 3; ++ch) img[3 * pix + ch] = C[ch];
                if (t_final) t_final[pix] = T;
                if (last) last[pix] = lst;
                if (ambiguous) ambiguous[pix] = (uint8_t)amb;
                tot_eval += ne;
                tot_blend += nb;
            }
    }
    if (counts) { counts[0] += tot_eval; counts[1] += tot_blend; }
}

static void atomic_add(double* p, double v)
{
#pragma omp atomic
    *p += v;
}

void orc_render_bwd(const double* xy, const double* conic, const double* opacity,
                    const double* rgb,
                    const uint32_t* vals, const uint32_t* ranges,
                    int32_t n_tiles, const int32_t* tile_ids,
                    const OrcCamera* cam, const OrcDilation* dil, const double bg[3],
                    const double* dl_dimg,
                    double* dxy, double* dconic, double* dopacity, double* drgb)
{
    int32_t w_ds, h_ds, tiles_x, tiles_y;
    orc_grid(cam, dil, &w_ds, &h_ds, &tiles_x, &tiles_y);
    int32_t nt = tile_ids ? n_tiles : tiles_x * tiles_y;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t k = 0; k < nt; ++k) {
        int32_t tile; uint32_t start, end;
        tile_of(k, nt, tile_ids, ranges, &tile, &start, &end);
        int tx = tile % tiles_x, ty = tile / tiles_x;
        OrcBlend* blend = (OrcBlend*)malloc((size_t)(end - start + 1) * sizeof(OrcBlend));
        for (int v = ty * dil->tile; v < (ty + 1) * dil->tile && v < h_ds; ++v)
            for (int u = tx * dil->tile; u < (tx + 1) * dil->tile && u < w_ds; ++u) {
                double x = (double)dil->d * u + dil->ox, y = (double)dil->d * v + dil->oy;
                double C[3], T_final; uint32_t lst; int amb;
                uint64_t ne = 0, nbl = 0;
                int64_t nb = blend_pixel(x, y, xy, conic, opacity, rgb, NULL, vals, start, end, bg,
                                         C, &T_final, &lst, &amb, &ne, &nbl, blend);
                int64_t pix = (int64_t)v * w_ds + u;
                const double* gC = dl_dimg + 3 * pix;
                /* S = colour accumulated behind the current entry, starting with
                 * the background seen through the final transmittance */
                double S[3] = { T_final * bg[0], T_final * bg[1], T_final * bg[2] };
                for (int64_t i = nb - 1; i >= 0; --i) {
                    const OrcBlend* e = &blend[i];
                    const double* c = rgb + 3 * (int64_t)e->g;
                    double w = e->alpha * e->T;
                    double dalpha = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        atomic_add(&drgb[3 * (int64_t)e->g + ch], w * gC[ch]);
                        dalpha += gC[ch] * (e->T * c[ch] - S[ch] / (1.0 - e->alpha));
                        S[ch] += c[ch] * w;
                    }
                    if (e->clamped) continue;  /* alpha = 0.99 does not depend on o or G */
                    double o = opacity[e->g];
                    atomic_add(&dopacity[e->g], e->G * dalpha);
                    double dpower = e->G * o * dalpha;
                    const double* q = conic + 3 * (int64_t)e->g;
                    /* power = -1/2 (A dx^2 + C dy^2) - B dx dy, dx = x - p_x */
                    atomic_add(&dconic[3 * (int64_t)e->g], -0.5 * e->dx * e->dx * dpower);
                    atomic_add(&dconic[3 * (int64_t)e->g + 1], -e->dx * e->dy * dpower);
                    atomic_add(&dconic[3 * (int64_t)e->g + 2], -0.5 * e->dy * e->dy * dpower);
                    atomic_add(&dxy[2 * (int64_t)e->g], dpower * (q[0] * e->dx + q[1] * e->dy));
                    atomic_add(&dxy[2 * (int64_t)e->g + 1], dpower * (q[2] * e->dy + q[1] * e->dx));
                }
            }
        free(blend);
    }
}

double orc_loss_l1(const OrcCamera* cam, const OrcDilation* dil, const double* img,
                   const double* target, double* dl_dimg)
{
    int32_t w_ds, h_ds;
    orc_grid(cam, dil, &w_ds, &h_ds, NULL, NULL);
    double inv = 1.0 / (3.0 * (double)w_ds * (double)h_ds);
    double L = 0.0;
    for (int v = 0; v < h_ds; ++v)
        for (int u = 0; u < w_ds; ++u) {
            int64_t hx = (int64_t)dil->d * u + dil->ox, hy = (int64_t)dil->d * v + dil->oy;
            int64_t pix = (int64_t)v * w_ds + u;
            for (int ch = 0; ch < 3; ++ch) {
                double r = img[3 * pix + ch] - target[3 * (hy * cam->width + hx) + ch];
                L += fabs(r) * inv;
                if (dl_dimg) dl_dimg[3 * pix + ch] = (r > 0.0 ? inv : (r < 0.0 ? -inv : 0.0));
            }
        }
    return L;
}

/* ------------------------------------------------------------------------- */
/* Projection backward: chain rule through conic, Sigma', J, Sigma(R, S),     */
/* the image-plane centre and the SH direction.                               */
/* ------------------------------------------------------------------------- */

void orc_project_bwd(int32_t n, int32_t sh_degree,
                     const double* means, const double* log_scales, const double* quats,
                     const double* opacity_logits, const double* sh,
                     const OrcCamera* cam, const OrcDilation* dil,
                     const double* dxy, const double* dconic, const double* dopacity,
                     const double* drgb,
                     double* d_means, double* d_log_scales, double* d_quats,
                     double* d_opacity_logits, double* d_sh)
{
    int ncoef = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double* gm = d_means + 3 * (int64_t)i;
        double* gs = d_log_scales + 3 * (int64_t)i;
        double* gq = d_quats + 4 * (int64_t)i;
        double* gsh = d_sh + (int64_t)i * ncoef * 3;
        for (int j = 0; j < 3; ++j) { gm[j] = 0.0; gs[j] = 0.0; }
        for (int j = 0; j < 4; ++j) gq[j] = 0.0;
        for (int j = 0; j < 3 * ncoef; ++j) gsh[j] = 0.0;
        d_opacity_logits[i] = 0.0;

        const double* mean = means + 3 * (int64_t)i;
        const double* shi = sh + (int64_t)i * ncoef * 3;
        OrcProj P;
        project_one(cam, dil, sh_degree, mean, log_scales + 3 * (int64_t)i, quats + 4 * (int64_t)i,
                    opacity_logits[i], shi, &P);
        if (P.culled) continue;
        double tz = P.t[2];

        /* opacity = sigmoid(logit) */
        d_opacity_logits[i] = dopacity[i] * P.opacity * (1.0 - P.opacity);

        /* colour: rgb = max(0, sum_k Y_k(dir) sh_k + 0.5) */
        double basis[ORC_MAX_COEFS], bgrad[3 * ORC_MAX_COEFS];
        sh_basis_grad(sh_degree, P.dir[0], P.dir[1], P.dir[2], basis, bgrad);
        double ddir[3] = { 0.0, 0.0, 0.0 };
        for (int ch = 0; ch < 3; ++ch) {
            if (!(P.rgb_raw[ch] > 0.0)) continue;
            double g = drgb[3 * (int64_t)i + ch];
            for (int k = 0; k < ncoef; ++k) {
                gsh[3 * k + ch] = basis[k] * g;
                for (int j = 0; j < 3; ++j) ddir[j] += g * shi[3 * k + ch] * bgrad[3 * k + j];
            }
        }
        /* dir = v / |v|, v = mean - camera centre */
        double dd = ddir[0] * P.dir[0] + ddir[1] * P.dir[1] + ddir[2] * P.dir[2];
        for (int j = 0; j < 3; ++j) gm[j] += (ddir[j] - P.dir[j] * dd) / P.vlen;

        /* conic (A, B, C) = (c, -b, a) / (ac - b^2) -> gradient w.r.t. (a, b, c) of Sigma' */
        double a = P.a, b = P.b, c = P.c, D = P.det, D2 = D * D;
        double gA = dconic[3 * (int64_t)i], gB = dconic[3 * (int64_t)i + 1], gC = dconic[3 * (int64_t)i + 2];
        double ga = gA * (-c * c / D2) + gB * (b * c / D2) + gC * (-b * b / D2);
        double gb = gA * (2 * b * c / D2) + gB * (-(a * c + b * b) / D2) + gC * (2 * a * b / D2);
        double gc = gA * (-b * b / D2) + gB * (a * b / D2) + gC * (-a * a / D2);
        /* symmetric matrix gradient of Sigma' (b is the shared off-diagonal) */
        double G2[4] = { ga, 0.5 * gb, 0.5 * gb, gc };

        /* Sigma' = Tm Sigma Tm^T: dL/dSigma = Tm^T G2 Tm, dL/dTm = 2 G2 Tm Sigma */
        double GS[9];
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                double acc = 0.0;
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) acc += P.Tm[3 * p + k] * G2[2 * p + q] * P.Tm[3 * q + l];
                GS[3 * k + l] = acc;
            }
        double GT[6];
        for (int p = 0; p < 2; ++p)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int q = 0; q < 2; ++q)
                    for (int l = 0; l < 3; ++l) acc += 2.0 * G2[2 * p + q] * P.Tm[3 * q + l] * P.Sigma[3 * l + k];
                GT[3 * p + k] = acc;
            }
        /* Tm = J R_cam: dL/dJ = dL/dTm R_cam^T */
        double GJ[6];
        for (int p = 0; p < 2; ++p)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int l = 0; l < 3; ++l) acc += GT[3 * p + l] * cam->R[3 * k + l];
                GJ[3 * p + k] = acc;
            }
        /* J(t): J00 = fx/tz, J02 = -fx txc/tz^2, J11 = fy/tz, J12 = -fy tyc/tz^2,
         * txc = tx unclamped, or +-lim tz when clamped (then J02 = -+fx lim / tz) */
        double dt[3] = { 0.0, 0.0, 0.0 };
        double fx = cam->fx, fy = cam->fy;
        double txc = P.uc * tz, tyc = P.vc * tz;
        dt[2] += GJ[0] * (-fx / (tz * tz)) + GJ[4] * (-fy / (tz * tz));
        if (P.clamp_x) {
            dt[2] += GJ[2] * (fx * txc / (tz * tz * tz));
        } else {
            dt[0] += GJ[2] * (-fx / (tz * tz));
            dt[2] += GJ[2] * (2.0 * fx * txc / (tz * tz * tz));
        }
        if (P.clamp_y) {
            dt[2] += GJ[5] * (fy * tyc / (tz * tz * tz));
        } else {
            dt[1] += GJ[5] * (-fy / (tz * tz));
            dt[2] += GJ[5] * (2.0 * fy * tyc / (tz * tz * tz));
        }
        /* p = (fx tx/tz + cx, fy ty/tz + cy) */
        double gpx = dxy[2 * (int64_t)i], gpy = dxy[2 * (int64_t)i + 1];
        dt[0] += gpx * fx / tz;
        dt[1] += gpy * fy / tz;
        dt[2] += -gpx * fx * P.t[0] / (tz * tz) - gpy * fy * P.t[1] / (tz * tz);
        /* t = R_cam mean + T */
        for (int j = 0; j < 3; ++j)
            gm[j] += cam->R[j] * dt[0] + cam->R[3 + j] * dt[1] + cam->R[6 + j] * dt[2];

        /* Sigma = M M^T, M = R S: dL/dM = 2 GS M (GS symmetric) */
        double GM[9];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int l = 0; l < 3; ++l) acc += 2.0 * GS[3 * k + l] * P.M[3 * l + j];
                GM[3 * k + j] = acc;
            }
        double GR[9];
        for (int j = 0; j < 3; ++j) {
            double gsj = 0.0;
            for (int k = 0; k < 3; ++k) {
                gsj += GM[3 * k + j] * P.Rq[3 * k + j];
                GR[3 * k + j] = GM[3 * k + j] * P.s[j];
            }
            gs[j] = gsj * P.s[j];  /* s = exp(log s) */
        }
        /* R(w, x, y, z): derivative of each entry with respect to each component */
        double w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
        double gqn[4];
        gqn[0] = 2 * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
        gqn[1] = 2 * (y * GR[1] + z * GR[2] + y * GR[3] - 2 * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2 * x * GR[8]);
        gqn[2] = 2 * (-2 * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2 * y * GR[8]);
        gqn[3] = 2 * (-2 * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2 * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
        /* qn = q / |q| */
        double qd = gqn[0] * P.qn[0] + gqn[1] * P.qn[1] + gqn[2] * P.qn[2] + gqn[3] * P.qn[3];
        for (int j = 0; j < 4; ++j) gq[j] = (gqn[j] - P.qn[j] * qd) / P.qnorm;
    }
}

/* ------------------------------------------------------------------------- */
/* Densification statistics (Sec. 3.3) and Adam (Sec. 4.1).                   */
/* ------------------------------------------------------------------------- */

void orc_densify_stats(int32_t n, const int64_t* tiles_touched, const double* dxy,
                       const double* drgb, double* pos_acc, double* col_acc,
                       int32_t* count)
{
    for (int32_t i = 0; i < n; ++i) {
        if (tiles_touched[i] <= 0) continue;
        const double* g = dxy + 2 * (int64_t)i;
        const double* c = drgb + 3 * (int64_t)i;
        pos_acc[i] += sqrt(g[0] * g[0] + g[1] * g[1]);
        col_acc[i] += sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        count[i] += 1;
    }
}

void orc_adam(int64_t numel, int32_t row_width, double* param, const double* grad,
              double* m, double* v, double lr, double beta1, double beta2, double eps,
              int32_t step, const uint8_t* row_mask)
{
    double bc1 = 1.0 - pow(beta1, step);
    double bc2 = 1.0 - pow(beta2, step);
    for (int64_t e = 0; e < numel; ++e) {
        if (row_mask && !row_mask[e / row_width]) continue;
        double g = grad[e];
        m[e] = beta1 * m[e] + (1.0 - beta1) * g;
        v[e] = beta2 * v[e] + (1.0 - beta2) * g * g;
        double mhat = m[e] / bc1;
        double vhat = v[e] / bc2;
        param[e] -= lr * mhat / (sqrt(vhat) + eps);
    }
}
