/*
 * ProbeSDF per-ray render and its adjoint: a plain, slow FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library: everything below is written from the paper's equations.
 *
 * What it computes, per ray (ProbeSDF, Sec. 3.1-3.3):
 *   - N colour samples and N+1 SDF points evenly spaced over the ray's
 *     segment inside the grid box (Eq. 8 needs s_{i+1} for the last alpha);
 *   - SDF s and its analytic trilinear gradient g at every point (Sec. 3.1
 *     explicit SDF grid; the normal of Eq. 13 is n = g/|g|);
 *   - spatial features F_s: trilinear blend of per-node features;
 *   - angular features F_a: real spherical harmonics of the reflected
 *     direction r = 2(n.v)n - v (or v itself), with coefficients blended
 *     trilinearly from the 8 surrounding probes (Eqs. 5-7);
 *   - Fresnel inputs (1 - n.v)^k, k = 1..K (Eq. 4);
 *   - a 2-hidden-layer ReLU MLP with sigmoid output (Sec. 4);
 *   - NeuS opacities and front-to-back compositing (Eqs. 8-10).
 * The adjoint is the exact reverse-mode derivative of the same steps.
 *
 * Readings of the paper taken here (the paper is silent on them):
 *   - Sample positions are computed in FP32 with a fixed, correctly rounded
 *     operation sequence, because they decide integer cell indices; the
 *     CUDA path computes the identical bits.  Everything after the cell
 *     index and fraction is FP64.
 *   - Both grids are node-aligned on one box: u = (x - bmin) * (R-1)/(bmax-bmin).
 *   - The normal guard is n = g / sqrt(|g|^2 + eps^2), eps = 1e-12.
 *   - The alpha clip max(., 0) of Eq. 9 passes no gradient at a tie.
 *   - v = -d; rays_d is taken as a unit vector as given.
 *   - SH: real orthonormal basis, no Condon-Shortley phase, ordered by
 *     degree and then m = -deg..deg; l is 1-indexed (l^2 coefficients).
 *
 * Parity pins live in tests/test_oracle_pins.py: closed forms, invariants,
 * a library routine for the SH basis and central finite differences.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "probesdf_oracle.h"

#define ORC_EPS_NORMAL 1e-12

/* ------------------------------------------------------------------------ */
/* Sample positions: FP32, correctly rounded, no contraction (compiled with */
/* -ffp-contract=off).                                                       */
/* ------------------------------------------------------------------------ */

/* Slab intersection of the ray with the box.  Returns 1 on a hit and sets
 * [tn, tf] with tn = max(t_enter, 0). */
static int ray_box_f32(const float o[3], const float d[3], const float bmin[3],
                       const float bmax[3], float* tn, float* tf)
{
    float t_enter = -INFINITY, t_exit = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < bmin[a] || o[a] > bmax[a]) return 0;
            continue;
        }
        float t0 = (bmin[a] - o[a]) / d[a];
        float t1 = (bmax[a] - o[a]) / d[a];
        float lo = t0 < t1 ? t0 : t1;
        float hi = t0 < t1 ? t1 : t0;
        if (lo > t_enter) t_enter = lo;
        if (hi < t_exit) t_exit = hi;
    }
    *tn = t_enter > 0.0f ? t_enter : 0.0f;
    *tf = t_exit;
    return *tf > *tn;
}

/* Grid coordinate of a point along one axis and its cell: the cell index is
 * floor(u) clamped to [0, R-2]; the fraction u - i is exact in FP32. */
static void locate_f32(const float x[3], const float bmin[3], const float sc[3],
                       const int32_t dims[3], int idx[3], double frac[3])
{
    for (int a = 0; a < 3; ++a) {
        float u = (x[a] - bmin[a]) * sc[a];
        float fl = floorf(u);
        float hi = (float)(dims[a] - 2);
        if (!(fl >= 0.0f)) fl = 0.0f; /* also maps NaN to cell 0: indices stay in bounds */
        if (fl > hi) fl = hi;
        idx[a] = (int)fl;
        frac[a] = (double)(u - fl);
    }
}

static void grid_scale_f32(const int32_t dims[3], const float bmin[3], const float bmax[3],
                           float sc[3])
{
    for (int a = 0; a < 3; ++a) sc[a] = (float)(dims[a] - 1) / (bmax[a] - bmin[a]);
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degrees 0..3 (l = 1..4, 1-indexed as in Eq. 5). */
/* Normalisation sqrt((2d+1)/(4 pi) * (d-|m|)!/(d+|m|)!), times sqrt(2) for  */
/* m != 0, written as Cartesian polynomials on the unit sphere.              */
/* ------------------------------------------------------------------------ */

void orc_sh_eval(int32_t l, const double r[3], double* Y)
{
    const double x = r[0], y = r[1], z = r[2];
    const double pi = M_PI;
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (l < 2) return;
    const double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = c1 * y;
    Y[2] = c1 * z;
    Y[3] = c1 * x;
    if (l < 3) return;
    const double c2a = 0.5 * sqrt(15.0 / pi);
    const double c20 = 0.25 * sqrt(5.0 / pi);
    const double c22 = 0.25 * sqrt(15.0 / pi);
    Y[4] = c2a * x * y;
    Y[5] = c2a * y * z;
    Y[6] = c20 * (3.0 * z * z - 1.0);
    Y[7] = c2a * x * z;
    Y[8] = c22 * (x * x - y * y);
    if (l < 4) return;
    const double c33 = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double c32 = 0.5 * sqrt(105.0 / pi);
    const double c31 = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double c30 = 0.25 * sqrt(7.0 / pi);
    const double c32b = 0.25 * sqrt(105.0 / pi);
    Y[9] = c33 * y * (3.0 * x * x - y * y);
    Y[10] = c32 * x * y * z;
    Y[11] = c31 * y * (5.0 * z * z - 1.0);
    Y[12] = c30 * z * (5.0 * z * z - 3.0);
    Y[13] = c31 * x * (5.0 * z * z - 1.0);
    Y[14] = c32b * z * (x * x - y * y);
    Y[15] = c33 * x * (x * x - 3.0 * y * y);
}

/* Partial derivatives dY_j/dr_a of the same polynomials: dY[j*3 + a]. */
void orc_sh_grad(int32_t l, const double r[3], double* dY)
{
    const double x = r[0], y = r[1], z = r[2];
    const double pi = M_PI;
    memset(dY, 0, sizeof(double) * 3 * (size_t)(l * l));
    if (l < 2) return;
    const double c1 = sqrt(3.0 / (4.0 * pi));
    dY[1 * 3 + 1] = c1;
    dY[2 * 3 + 2] = c1;
    dY[3 * 3 + 0] = c1;
    if (l < 3) return;
    const double c2a = 0.5 * sqrt(15.0 / pi);
    const double c20 = 0.25 * sqrt(5.0 / pi);
    const double c22 = 0.25 * sqrt(15.0 / pi);
    dY[4 * 3 + 0] = c2a * y;  dY[4 * 3 + 1] = c2a * x;
    dY[5 * 3 + 1] = c2a * z;  dY[5 * 3 + 2] = c2a * y;
    dY[6 * 3 + 2] = c20 * 6.0 * z;
    dY[7 * 3 + 0] = c2a * z;  dY[7 * 3 + 2] = c2a * x;
    dY[8 * 3 + 0] = c22 * 2.0 * x;  dY[8 * 3 + 1] = -c22 * 2.0 * y;
    if (l < 4) return;
    const double c33 = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double c32 = 0.5 * sqrt(105.0 / pi);
    const double c31 = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double c30 = 0.25 * sqrt(7.0 / pi);
    const double c32b = 0.25 * sqrt(105.0 / pi);
    dY[9 * 3 + 0] = c33 * 6.0 * x * y;
    dY[9 * 3 + 1] = c33 * (3.0 * x * x - 3.0 * y * y);
    dY[10 * 3 + 0] = c32 * y * z;  dY[10 * 3 + 1] = c32 * x * z;  dY[10 * 3 + 2] = c32 * x * y;
    dY[11 * 3 + 1] = c31 * (5.0 * z * z - 1.0);  dY[11 * 3 + 2] = c31 * 10.0 * y * z;
    dY[12 * 3 + 2] = c30 * (15.0 * z * z - 3.0);
    dY[13 * 3 + 0] = c31 * (5.0 * z * z - 1.0);  dY[13 * 3 + 2] = c31 * 10.0 * x * z;
    dY[14 * 3 + 0] = c32b * 2.0 * x * z;  dY[14 * 3 + 1] = -c32b * 2.0 * y * z;
    dY[14 * 3 + 2] = c32b * (x * x - y * y);
    dY[15 * 3 + 0] = c33 * (3.0 * x * x - 3.0 * y * y);
    dY[15 * 3 + 1] = -c33 * 6.0 * x * y;
}

/* ------------------------------------------------------------------------ */
/* Per-sample state                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    float t;                       /* distance along the ray (FP32 value) */
    int ci[3];                     /* SDF cell */
    double cf[3];                  /* fraction inside the SDF cell */
    int pi_[3];                    /* probe cell */
    double pf[3];                  /* fraction inside the probe cell */
    double s;                      /* SDF value */
    double g[3];                   /* trilinear gradient, world units */
    double rho;                    /* sqrt(|g|^2 + eps^2) */
    double n[3], r[3], ndv;
    double Y[ORC_MAX_L2];
    double bhat[ORC_MAX_L2 * ORC_MAX_NA];   /* probe-blended coefficients */
    double x[ORC_MAX_IN];          /* MLP input [F_s, F_a, fresnel] */
    double z1[ORC_MAX_W], h1[ORC_MAX_W], z2[ORC_MAX_W], h2[ORC_MAX_W];
    double z3[3], C[3];
} orc_sample;

static inline size_t node_index(const int32_t dims[3], int ix, int iy, int iz)
{
    return ((size_t)iz * (size_t)dims[1] + (size_t)iy) * (size_t)dims[0] + (size_t)ix;
}

/* Trilinear weight of corner (cx,cy,cz) and its derivative in cell units. */
static void corner_weight(const double f[3], int cx, int cy, int cz, double* w, double dw[3])
{
    const double wx = cx ? f[0] : 1.0 - f[0], dx = cx ? 1.0 : -1.0;
    const double wy = cy ? f[1] : 1.0 - f[1], dy = cy ? 1.0 : -1.0;
    const double wz = cz ? f[2] : 1.0 - f[2], dz = cz ? 1.0 : -1.0;
    *w = wx * wy * wz;
    if (dw) {
        dw[0] = dx * wy * wz;
        dw[1] = wx * dy * wz;
        dw[2] = wx * wy * dz;
    }
}

static inline double relu(double z) { return z > 0.0 ? z : 0.0; }
static inline double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }
/* log Phi_tau(s) with Phi the logistic function (Eq. 10), in a stable form. */
static inline double log_phi(double tau, double s)
{
    const double z = -tau * s; /* log Phi = -softplus(z) */
    return -((z > 0.0 ? z : 0.0) + log1p(exp(-fabs(z))));
}

static int mlp_n_in(const orc_model* m) { return m->n_s + m->n_a + m->n_fresnel; }

/* Tile tri-plane spatial features (Sec. 3.1, Sec. 4): the grid's cells are cut
 * into tiles of 16^3; each tile holds three 16 x 16 planes of n_s channels,
 * orthogonal to x, y and z, and F_s = F_x (.) F_y (.) F_z, each factor a
 * bilinear lookup in its plane at the point's two in-plane coordinates.  A
 * plane's 16 texels per axis sit at the centres of the tile's 16 cells; a
 * point's texel coordinate is clamped to the tile's texels.  The tile and
 * texel of a coordinate are exact functions of the FP32 grid coordinate u
 * (u / 16 and u - 16 t are exact). */
typedef struct {
    size_t plane0;     /* offset of the tile's first plane (in values) */
    int i[3];          /* texel index along x, y, z (0..14) */
    double f[3];       /* fraction to the next texel */
    double b[3][ORC_MAX_NS];  /* the three bilinear lookups per channel */
} tri_at;

static int n_tiles(int32_t R) { return (R - 1 + ORC_TILE - 1) / ORC_TILE; }

static size_t texel(int plane, int r, int c, int ns)
{
    return (((size_t)plane * ORC_TILE + (size_t)r) * ORC_TILE + (size_t)c) * (size_t)ns;
}

static void triplane_locate(const orc_model* m, const int ci[3], const double cf[3], tri_at* T)
{
    int t[3];
    for (int a = 0; a < 3; ++a) {
        const double u = (double)ci[a] + cf[a];
        const int nt = n_tiles(m->R[a]);
        int ta = (int)floor(u / ORC_TILE);
        if (ta > nt - 1) ta = nt - 1;
        if (ta < 0) ta = 0;
        double tau = u - (double)ORC_TILE * ta - 0.5;
        if (tau < 0.0) tau = 0.0;
        if (tau > ORC_TILE - 1) tau = ORC_TILE - 1;
        int i = (int)floor(tau);
        if (i > ORC_TILE - 2) i = ORC_TILE - 2;
        t[a] = ta;
        T->i[a] = i;
        T->f[a] = tau - i;
    }
    const size_t tile = ((size_t)t[2] * n_tiles(m->R[1]) + t[1]) * n_tiles(m->R[0]) + t[0];
    T->plane0 = tile * 3 * ORC_TILE * ORC_TILE * (size_t)m->n_s;
}

/* Bilinear weights of a plane lookup at (row axis, column axis). */
static void bilerp_w(const tri_at* T, int ra, int ca, double w[4])
{
    const double fr = T->f[ra], fc = T->f[ca];
    w[0] = (1 - fr) * (1 - fc);
    w[1] = (1 - fr) * fc;
    w[2] = fr * (1 - fc);
    w[3] = fr * fc;
}

/* plane p: 0 is [z][y], 1 is [z][x], 2 is [y][x] */
static const int kPlaneRow[3] = {2, 2, 1}, kPlaneCol[3] = {1, 0, 0};

static void triplane_features(const orc_model* m, tri_at* T, double* fs)
{
    const int ns = m->n_s;
    for (int p = 0; p < 3; ++p) {
        const int ra = kPlaneRow[p], ca = kPlaneCol[p];
        double w[4];
        bilerp_w(T, ra, ca, w);
        const int r = T->i[ra], c = T->i[ca];
        const double* P = m->planes + T->plane0;
        for (int q = 0; q < ns; ++q)
            T->b[p][q] = w[0] * P[texel(p, r, c, ns) + q] + w[1] * P[texel(p, r, c + 1, ns) + q] +
                         w[2] * P[texel(p, r + 1, c, ns) + q] +
                         w[3] * P[texel(p, r + 1, c + 1, ns) + q];
    }
    for (int q = 0; q < ns; ++q) fs[q] = T->b[0][q] * T->b[1][q] * T->b[2][q];
}

/* Colour inputs after the spatial features (Sec. 3.1-3.2): normal from S->g
 * (Eq. 13, guarded against 0/0), the SH lookup direction (r = 2(n.v)n - v, or v),
 * the probe-blended angular features of the probe cell in S->pi_, S->pf
 * (Eqs. 5-7) and the Fresnel inputs (Eq. 4), into S->x after the n_s features. */
static void angular_inputs(const orc_model* m, const orc_params* p, const double v[3],
                           orc_sample* S)
{
    const int ns = m->n_s;
    const double gg = S->g[0] * S->g[0] + S->g[1] * S->g[1] + S->g[2] * S->g[2];
    S->rho = sqrt(gg + ORC_EPS_NORMAL * ORC_EPS_NORMAL);
    for (int a = 0; a < 3; ++a) S->n[a] = S->g[a] / S->rho;
    S->ndv = S->n[0] * v[0] + S->n[1] * v[1] + S->n[2] * v[2];
    for (int a = 0; a < 3; ++a)
        S->r[a] = (p->dir_mode == ORC_DIR_VIEW) ? v[a] : 2.0 * S->ndv * S->n[a] - v[a];

    /* Angular features, Eqs. 5-7: bhat_j = sum_i w_i b_ij, F_a = sum_j bhat_j Y_j. */
    const int L2 = m->sh_l * m->sh_l, na = m->n_a;
    orc_sh_eval(m->sh_l, S->r, S->Y);
    for (int k = 0; k < L2 * na; ++k) S->bhat[k] = 0.0;
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        double w;
        corner_weight(S->pf, cx, cy, cz, &w, NULL);
        const size_t pn = node_index(m->P, S->pi_[0] + cx, S->pi_[1] + cy, S->pi_[2] + cz);
        const double* b = m->probes + pn * (size_t)(L2 * na);
        for (int k = 0; k < L2 * na; ++k) S->bhat[k] += w * b[k];
    }
    for (int ch = 0; ch < na; ++ch) {
        double fa = 0.0;
        for (int j = 0; j < L2; ++j) fa += S->bhat[j * na + ch] * S->Y[j];
        S->x[ns + ch] = fa;
    }
    /* Fresnel inputs (1 - n.v)^k, k = 1..K (Eq. 4). */
    for (int k = 1; k <= m->n_fresnel; ++k) S->x[ns + na + k - 1] = pow(1.0 - S->ndv, (double)k);
}

/* Nearest binary16 value of v (ties to even): 11 significant bits, so the
 * spacing in [2^(e-1), 2^e) is 2^(e-11); below the smallest normal 2^-14 the
 * spacing stays 2^-24 (subnormals).  nearbyint rounds in the default
 * to-nearest-even mode. */
double orc_round_f16(double v)
{
    if (!(fabs(v) > 0.0) || isinf(v)) return v;
    int e;
    frexp(v, &e);
    int q = e - 11;
    if (q < -24) q = -24;
    const double r = ldexp(nearbyint(ldexp(v, -q)), q);
    return fabs(r) > 65504.0 ? copysign(INFINITY, v) : r;
}

/* Colour MLP on S->x: two ReLU layers and a sigmoid output (Sec. 4).  With
 * f16 the inputs of layers 1 and 2 are rounded to binary16 first and kept so
 * (the adjoint's weight gradients use the rounded values). */
static void mlp_colour(const orc_model* m, orc_sample* S, double* margin, int f16)
{
    const int W = m->width, nin = mlp_n_in(m);
    const double* W1 = m->mlp;
    const double* b1 = W1 + W * nin;
    const double* W2 = b1 + W;
    const double* b2 = W2 + W * W;
    const double* W3 = b2 + W;
    const double* b3 = W3 + 3 * W;
    if (f16)
        for (int i = 0; i < nin; ++i) S->x[i] = orc_round_f16(S->x[i]);
    for (int o2 = 0; o2 < W; ++o2) {
        double z = b1[o2], mag = fabs(b1[o2]);
        for (int i = 0; i < nin; ++i) {
            z += W1[o2 * nin + i] * S->x[i];
            mag += fabs(W1[o2 * nin + i] * S->x[i]);
        }
        S->z1[o2] = z;
        S->h1[o2] = f16 ? orc_round_f16(relu(z)) : relu(z);
        if (margin && mag > 0.0 && fabs(z) / mag < *margin) *margin = fabs(z) / mag;
    }
    for (int o2 = 0; o2 < W; ++o2) {
        double z = b2[o2], mag = fabs(b2[o2]);
        for (int i = 0; i < W; ++i) {
            z += W2[o2 * W + i] * S->h1[i];
            mag += fabs(W2[o2 * W + i] * S->h1[i]);
        }
        S->z2[o2] = z;
        S->h2[o2] = relu(z);
        if (margin && mag > 0.0 && fabs(z) / mag < *margin) *margin = fabs(z) / mag;
    }
    for (int c = 0; c < 3; ++c) {
        double z = b3[c];
        for (int i = 0; i < W; ++i) z += W3[c * W + i] * S->h2[i];
        S->z3[c] = z;
        S->C[c] = sigmoid(z);
    }
}

/* Point geometry (positions, cells, SDF value and gradient, spatial
 * features).  `color` also asks for the rest of the colour inputs. */
static void eval_point(const orc_model* m, const orc_params* p, const float o[3],
                       const float d[3], float t, int color, orc_sample* S, double* margin)
{
    float sc[3], scp[3], x[3];
    grid_scale_f32(m->R, m->bmin, m->bmax, sc);
    grid_scale_f32(m->P, m->bmin, m->bmax, scp);
    for (int a = 0; a < 3; ++a) x[a] = fmaf(t, d[a], o[a]);
    S->t = t;
    locate_f32(x, m->bmin, sc, m->R, S->ci, S->cf);

    S->s = 0.0;
    S->g[0] = S->g[1] = S->g[2] = 0.0;
    const int ns = m->n_s;
    for (int q = 0; q < ns; ++q) S->x[q] = 0.0;
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        double w, dw[3];
        corner_weight(S->cf, cx, cy, cz, &w, dw);
        const size_t nd = node_index(m->R, S->ci[0] + cx, S->ci[1] + cy, S->ci[2] + cz);
        const double sv = m->sdf[nd];
        S->s += w * sv;
        for (int a = 0; a < 3; ++a) S->g[a] += sv * dw[a] * (double)sc[a];
        if (color && m->feat_layout == ORC_FEAT_NODES)
            for (int q = 0; q < ns; ++q) S->x[q] += w * m->feat[nd * (size_t)ns + q];
    }
    if (p->sdf_fp32) {
        /* the same value rounded as a FP32 evaluation rounds it: corner weights
         * as products of (1 - f) and f in FP32, then a fused multiply-add per
         * corner in corner order (the fractions are exact in FP32) */
        const float fx = (float)S->cf[0], fy = (float)S->cf[1], fz = (float)S->cf[2];
        const float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
        float s32 = 0.0f;
        for (int c = 0; c < 8; ++c) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
            const float w32 = wx[cx] * wy[cy] * wz[cz];
            const size_t nd = node_index(m->R, S->ci[0] + cx, S->ci[1] + cy, S->ci[2] + cz);
            s32 = fmaf(w32, (float)m->sdf[nd], s32);
        }
        S->s = (double)s32;
    }
    if (!color) return;
    if (m->feat_layout == ORC_FEAT_TRIPLANE) {
        tri_at T;
        triplane_locate(m, S->ci, S->cf, &T);
        triplane_features(m, &T, S->x);
    }

    double v[3];
    for (int a = 0; a < 3; ++a) v[a] = -(double)d[a];
    locate_f32(x, m->bmin, scp, m->P, S->pi_, S->pf);
    angular_inputs(m, p, v, S);
    mlp_colour(m, S, margin, p->mlp_f16);
}

/* Sample distances of one ray.  Returns 0 for a ray that misses the box. */
static int ray_samples(const orc_model* m, const orc_params* p, const float* o, const float* d,
                       const float* t_given, float* t)
{
    const int N = p->n_samples;
    if (t_given) {
        for (int k = 0; k <= N; ++k) t[k] = t_given[k];
        return t[N] > t[0];
    }
    float tn, tf;
    if (!ray_box_f32(o, d, m->bmin, m->bmax, &tn, &tf)) return 0;
    const float dt = (tf - tn) / (float)N;
    for (int k = 0; k <= N; ++k) t[k] = fmaf((float)k, dt, tn);
    return 1;
}

/* Forward of one ray.  Fills S[0..N], lam[0..N-1] (log(1 - alpha_k)),
 * logT[0..N], clipped[0..N-1]. */
typedef struct {
    orc_sample* S;
    float* t;
    double *lam, *logT, *alpha, *w;
    int* unclipped;
} ray_work;

static int forward_ray(const orc_model* m, const orc_params* p, const float* o, const float* d,
                       const float* t_given, ray_work* rw, double out_rgb[3], double* out_depth,
                       double* out_wsum, double* out_logT, double* margin)
{
    const int N = p->n_samples;
    if (!ray_samples(m, p, o, d, t_given, rw->t)) {
        for (int c = 0; c < 3; ++c) out_rgb[c] = p->bg[c];
        *out_depth = 0.0;
        *out_wsum = 0.0;
        *out_logT = 0.0;
        return 0;
    }
    for (int k = 0; k <= N; ++k) eval_point(m, p, o, d, rw->t[k], k < N, &rw->S[k], margin);

    /* NeuS opacity (Eqs. 9-10) in log space:
     *   log(1 - alpha_k) = min(log Phi(s_{k+1}) - log Phi(s_k), 0),
     * transmittance T_k = prod_{j<k} (1 - alpha_j) (Eq. 8). */
    double rgb[3] = {0, 0, 0}, depth = 0.0, wsum = 0.0;
    rw->logT[0] = 0.0;
    for (int k = 0; k < N; ++k) {
        const double l0 = log_phi(p->tau, rw->S[k].s), l1 = log_phi(p->tau, rw->S[k + 1].s);
        const double diff = l1 - l0;
        rw->unclipped[k] = diff < 0.0;
        rw->lam[k] = diff < 0.0 ? diff : 0.0;
        if (margin) {
            const double mag = fabs(l0) + fabs(l1);
            if (mag > 0.0 && fabs(diff) / mag < *margin) *margin = fabs(diff) / mag;
        }
        rw->alpha[k] = -expm1(rw->lam[k]);
        rw->logT[k + 1] = rw->logT[k] + rw->lam[k];
        rw->w[k] = exp(rw->logT[k]) * rw->alpha[k];
        for (int c = 0; c < 3; ++c) rgb[c] += rw->w[k] * rw->S[k].C[c];
        depth += rw->w[k] * (double)rw->t[k];
        wsum += rw->w[k];
    }
    const double TN = exp(rw->logT[N]);
    for (int c = 0; c < 3; ++c) out_rgb[c] = rgb[c] + TN * p->bg[c];
    *out_depth = depth;
    *out_wsum = wsum;
    *out_logT = rw->logT[N];
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Gradient accumulation                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double* g_sdf;     /* [R^3]         (shared; atomic when threaded) */
    double* g_feat;    /* [R^3][n_s]    (shared; atomic when threaded) */
    double* g_probe;   /* [P^3][L2][na] (private per thread) */
    double* g_mlp;     /* [params]      (private per thread) */
    int atomic;
} grad_sink;

static void add_f64(double* p, double v, int atomic)
{
    if (!atomic) {
        *p += v;
        return;
    }
    uint64_t* q = (uint64_t*)p;
    uint64_t old = __atomic_load_n(q, __ATOMIC_RELAXED), nw;
    for (;;) {
        double cur, nv;
        memcpy(&cur, &old, 8);
        nv = cur + v;
        memcpy(&nw, &nv, 8);
        if (__atomic_compare_exchange_n(q, &old, nw, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) break;
    }
}

/* Adjoint of one ray; the forward state is in rw. */
static void backward_ray(const orc_model* m, const orc_params* p, const float* d, ray_work* rw,
                         const double drgb[3], double ddepth, double dwsum, grad_sink* gs)
{
    const int N = p->n_samples, W = m->width, nin = mlp_n_in(m);
    const int ns = m->n_s, na = m->n_a, L2 = m->sh_l * m->sh_l, K = m->n_fresnel;
    const double* W1 = m->mlp;
    const double* b1 = W1 + W * nin;
    const double* W2 = b1 + W;
    const double* b2 = W2 + W * W;
    const double* W3 = b2 + W;
    (void)b2;
    double* gW1 = gs->g_mlp;
    double* gb1 = gW1 + W * nin;
    double* gW2 = gb1 + W;
    double* gb2 = gW2 + W * W;
    double* gW3 = gb2 + W;
    double* gb3 = gW3 + 3 * W;
    float sc[3];
    grid_scale_f32(m->R, m->bmin, m->bmax, sc);

    /* dL/dlam_k with the suffix recurrence
     *   Shat_{N-1} = G_bg,  Shat_k = alpha_{k+1} G_{k+1} + (1 - alpha_{k+1}) Shat_{k+1},
     *   dL/dalpha_k = T_k (G_k - Shat_k),  dalpha/dlam = -(1 - alpha) = -T_{k+1}/T_k. */
    double* G = (double*)malloc(sizeof(double) * (size_t)N);
    double* dlam = (double*)malloc(sizeof(double) * (size_t)N);
    double* ds = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    for (int k = 0; k < N; ++k)
        G[k] = drgb[0] * rw->S[k].C[0] + drgb[1] * rw->S[k].C[1] + drgb[2] * rw->S[k].C[2] +
               ddepth * (double)rw->t[k] + dwsum;
    const double Gbg = drgb[0] * p->bg[0] + drgb[1] * p->bg[1] + drgb[2] * p->bg[2];
    double Shat = Gbg;
    for (int k = N - 1; k >= 0; --k) {
        if (k < N - 1) Shat = rw->alpha[k + 1] * G[k + 1] + (1.0 - rw->alpha[k + 1]) * Shat;
        dlam[k] = rw->unclipped[k] ? -exp(rw->logT[k + 1]) * (G[k] - Shat) : 0.0;
    }
    /* lam_k = logPhi(s_{k+1}) - logPhi(s_k);  dlogPhi/ds = tau * (1 - Phi(s)). */
    for (int k = 0; k <= N; ++k) {
        double dl = 0.0;
        if (k < N) dl -= dlam[k];
        if (k > 0) dl += dlam[k - 1];
        ds[k] = dl * p->tau * sigmoid(p->tau * rw->S[k].s * -1.0);
    }

    for (int k = 0; k <= N; ++k) {
        orc_sample* S = &rw->S[k];
        double dg[3] = {0, 0, 0};
        double dx[ORC_MAX_IN];
        if (k < N) {
            /* Colour path: rgb += w_k C_k. */
            double dz3[3], dh2[ORC_MAX_W], dz2[ORC_MAX_W], dh1[ORC_MAX_W], dz1[ORC_MAX_W];
            for (int c = 0; c < 3; ++c) dz3[c] = rw->w[k] * drgb[c] * S->C[c] * (1.0 - S->C[c]);
            for (int c = 0; c < 3; ++c) {
                gb3[c] += dz3[c];
                for (int i = 0; i < W; ++i) gW3[c * W + i] += dz3[c] * S->h2[i];
            }
            for (int i = 0; i < W; ++i) {
                double a = 0.0;
                for (int c = 0; c < 3; ++c) a += W3[c * W + i] * dz3[c];
                dh2[i] = a;
                dz2[i] = S->z2[i] > 0.0 ? a : 0.0;
            }
            for (int o2 = 0; o2 < W; ++o2) {
                gb2[o2] += dz2[o2];
                for (int i = 0; i < W; ++i) gW2[o2 * W + i] += dz2[o2] * S->h1[i];
            }
            for (int i = 0; i < W; ++i) {
                double a = 0.0;
                for (int o2 = 0; o2 < W; ++o2) a += W2[o2 * W + i] * dz2[o2];
                dh1[i] = a;
                dz1[i] = S->z1[i] > 0.0 ? a : 0.0;
            }
            for (int o2 = 0; o2 < W; ++o2) {
                gb1[o2] += dz1[o2];
                for (int i = 0; i < nin; ++i) gW1[o2 * nin + i] += dz1[o2] * S->x[i];
            }
            for (int i = 0; i < nin; ++i) {
                double a = 0.0;
                for (int o2 = 0; o2 < W; ++o2) a += W1[o2 * nin + i] * dz1[o2];
                dx[i] = a;
            }
            (void)dh2;
            (void)dh1;

            /* Probe coefficients and the reflected direction (Eqs. 6-7). */
            double dY[ORC_MAX_L2];
            for (int j = 0; j < L2; ++j) {
                double a = 0.0;
                for (int ch = 0; ch < na; ++ch) a += S->bhat[j * na + ch] * dx[ns + ch];
                dY[j] = a;
            }
            for (int c = 0; c < 8; ++c) {
                const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
                double w;
                corner_weight(S->pf, cx, cy, cz, &w, NULL);
                const size_t pn =
                    node_index(m->P, S->pi_[0] + cx, S->pi_[1] + cy, S->pi_[2] + cz);
                double* gb = gs->g_probe + pn * (size_t)(L2 * na);
                for (int j = 0; j < L2; ++j)
                    for (int ch = 0; ch < na; ++ch) gb[j * na + ch] += w * S->Y[j] * dx[ns + ch];
            }
            double dYdr[ORC_MAX_L2 * 3], dr[3] = {0, 0, 0};
            orc_sh_grad(m->sh_l, S->r, dYdr);
            for (int j = 0; j < L2; ++j)
                for (int a = 0; a < 3; ++a) dr[a] += dY[j] * dYdr[j * 3 + a];

            double v[3], dn[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a) v[a] = -(double)d[a];
            if (p->dir_mode != ORC_DIR_VIEW) {
                /* r = 2 (n.v) n - v */
                const double drn = dr[0] * S->n[0] + dr[1] * S->n[1] + dr[2] * S->n[2];
                for (int a = 0; a < 3; ++a) dn[a] += 2.0 * drn * v[a] + 2.0 * S->ndv * dr[a];
            }
            /* Fresnel: f_k = (1 - n.v)^k. */
            double dndv = 0.0;
            for (int kk = 1; kk <= K; ++kk)
                dndv -= dx[ns + na + kk - 1] * (double)kk * pow(1.0 - S->ndv, (double)(kk - 1));
            for (int a = 0; a < 3; ++a) dn[a] += dndv * v[a];
            /* n = g / rho: dg = (dn - n (n.dn)) / rho. */
            const double ndn = S->n[0] * dn[0] + S->n[1] * dn[1] + S->n[2] * dn[2];
            for (int a = 0; a < 3; ++a) dg[a] = (dn[a] - S->n[a] * ndn) / S->rho;
        }
        /* Scatter into the SDF nodes (alpha path and normal path) and features. */
        for (int c = 0; c < 8; ++c) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
            double w, dw[3];
            corner_weight(S->cf, cx, cy, cz, &w, dw);
            const size_t nd = node_index(m->R, S->ci[0] + cx, S->ci[1] + cy, S->ci[2] + cz);
            double gsdf = ds[k] * w;
            if (k < N)
                for (int a = 0; a < 3; ++a) gsdf += dg[a] * dw[a] * (double)sc[a];
            add_f64(&gs->g_sdf[nd], gsdf, gs->atomic);
            if (k < N && m->feat_layout == ORC_FEAT_NODES)
                for (int q = 0; q < ns; ++q)
                    add_f64(&gs->g_feat[nd * (size_t)ns + q], w * dx[q], gs->atomic);
        }
        if (k < N && m->feat_layout == ORC_FEAT_TRIPLANE) {
            /* F_s = b0 b1 b2 per channel: each plane's lookup gets dF_s times the
             * other two, spread over its 4 texels by the bilinear weights */
            tri_at T;
            triplane_locate(m, S->ci, S->cf, &T);
            double fs[ORC_MAX_NS];
            triplane_features(m, &T, fs);
            for (int p2 = 0; p2 < 3; ++p2) {
                const int ra = kPlaneRow[p2], ca = kPlaneCol[p2];
                double w4[4];
                bilerp_w(&T, ra, ca, w4);
                const int r = T.i[ra], c = T.i[ca];
                const size_t o4[4] = {texel(p2, r, c, ns), texel(p2, r, c + 1, ns),
                                      texel(p2, r + 1, c, ns), texel(p2, r + 1, c + 1, ns)};
                for (int q = 0; q < ns; ++q) {
                    double other = 1.0;
                    for (int p3 = 0; p3 < 3; ++p3)
                        if (p3 != p2) other *= T.b[p3][q];
                    for (int e = 0; e < 4; ++e)
                        add_f64(&gs->g_feat[T.plane0 + o4[e] + q], w4[e] * other * dx[q],
                                gs->atomic);
                }
            }
        }
    }
    free(G);
    free(dlam);
    free(ds);
}

/* ------------------------------------------------------------------------ */
/* Threaded drivers                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_model* m;
    const orc_params* p;
    int64_t n_rays;
    const float *o, *d, *t_given;
    double *rgb, *depth, *wsum, *logT, *margin;
    const double *drgb, *ddepth, *dwsum;
    grad_sink sink;
    int64_t* next;
    int backward;
    double* g_probe_priv;
    double* g_mlp_priv;
} job;

static int64_t n_mlp_params(const orc_model* m)
{
    const int W = m->width, nin = mlp_n_in(m);
    return (int64_t)W * nin + W + (int64_t)W * W + W + 3 * W + 3;
}

static int64_t n_probe_values(const orc_model* m)
{
    return (int64_t)m->P[0] * m->P[1] * m->P[2] * m->sh_l * m->sh_l * m->n_a;
}

static void alloc_work(const orc_params* p, ray_work* rw)
{
    const int N = p->n_samples;
    rw->S = (orc_sample*)malloc(sizeof(orc_sample) * (size_t)(N + 1));
    rw->t = (float*)malloc(sizeof(float) * (size_t)(N + 1));
    rw->lam = (double*)malloc(sizeof(double) * (size_t)N);
    rw->logT = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    rw->alpha = (double*)malloc(sizeof(double) * (size_t)N);
    rw->w = (double*)malloc(sizeof(double) * (size_t)N);
    rw->unclipped = (int*)malloc(sizeof(int) * (size_t)N);
}

static void free_work(ray_work* rw)
{
    free(rw->S);
    free(rw->t);
    free(rw->lam);
    free(rw->logT);
    free(rw->alpha);
    free(rw->w);
    free(rw->unclipped);
}

static void* worker(void* arg)
{
    job* jb = (job*)arg;
    ray_work rw;
    alloc_work(jb->p, &rw);
    const int N = jb->p->n_samples;
    for (;;) {
        const int64_t r0 = __atomic_fetch_add(jb->next, 16, __ATOMIC_RELAXED);
        if (r0 >= jb->n_rays) break;
        const int64_t r1 = r0 + 16 < jb->n_rays ? r0 + 16 : jb->n_rays;
        for (int64_t r = r0; r < r1; ++r) {
            double rgb[3], depth, wsum, logT, margin = INFINITY;
            const float* tg = jb->t_given ? jb->t_given + r * (N + 1) : NULL;
            const int hit = forward_ray(jb->m, jb->p, jb->o + 3 * r, jb->d + 3 * r, tg, &rw, rgb,
                                        &depth, &wsum, &logT, jb->margin ? &margin : NULL);
            if (!jb->backward) {
                for (int c = 0; c < 3; ++c) jb->rgb[3 * r + c] = rgb[c];
                jb->depth[r] = depth;
                jb->wsum[r] = wsum;
                jb->logT[r] = logT;
                if (jb->margin) jb->margin[r] = margin;
            } else if (hit) {
                const double dd = jb->ddepth ? jb->ddepth[r] : 0.0;
                const double dw = jb->dwsum ? jb->dwsum[r] : 0.0;
                backward_ray(jb->m, jb->p, jb->d + 3 * r, &rw, jb->drgb + 3 * r, dd, dw, &jb->sink);
            }
        }
    }
    free_work(&rw);
    return NULL;
}

static int run_jobs(job* proto, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    int64_t next = 0;
    job* jobs = (job*)calloc((size_t)n_threads, sizeof(job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    const int64_t np = n_probe_values(proto->m), nm = n_mlp_params(proto->m);
    for (int i = 0; i < n_threads; ++i) {
        jobs[i] = *proto;
        jobs[i].next = &next;
        jobs[i].sink.atomic = n_threads > 1;
        if (proto->backward && n_threads > 1) {
            jobs[i].g_probe_priv = (double*)calloc((size_t)np, sizeof(double));
            jobs[i].g_mlp_priv = (double*)calloc((size_t)nm, sizeof(double));
            jobs[i].sink.g_probe = jobs[i].g_probe_priv;
            jobs[i].sink.g_mlp = jobs[i].g_mlp_priv;
        }
    }
    if (n_threads == 1) {
        worker(&jobs[0]);
    } else {
        for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, worker, &jobs[i]);
        for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    }
    if (proto->backward && n_threads > 1) {
        for (int i = 0; i < n_threads; ++i) {
            for (int64_t k = 0; k < np; ++k) proto->sink.g_probe[k] += jobs[i].g_probe_priv[k];
            for (int64_t k = 0; k < nm; ++k) proto->sink.g_mlp[k] += jobs[i].g_mlp_priv[k];
            free(jobs[i].g_probe_priv);
            free(jobs[i].g_mlp_priv);
        }
    }
    free(jobs);
    free(th);
    return 0;
}

static int check_model(const orc_model* m, const orc_params* p)
{
    if (!m || !p) return -1;
    if (m->n_s < 0 || m->n_s > ORC_MAX_NS || m->n_a < 1 || m->n_a > ORC_MAX_NA) return -2;
    if (m->sh_l < 1 || m->sh_l > 4 || m->n_fresnel < 0 || m->n_fresnel > ORC_MAX_K) return -2;
    if (m->width < 1 || m->width > ORC_MAX_W || mlp_n_in(m) > ORC_MAX_IN) return -2;
    for (int a = 0; a < 3; ++a)
        if (m->R[a] < 2 || m->P[a] < 2 || !(m->bmax[a] > m->bmin[a])) return -2;
    if (p->n_samples < 1) return -2;
    if (m->feat_layout == ORC_FEAT_TRIPLANE ? !m->planes
                                            : (m->feat_layout != ORC_FEAT_NODES ||
                                               (m->n_s > 0 && !m->feat)))
        return -2;
    return 0;
}

int32_t orc_render_forward(const orc_model* m, const orc_params* p, int64_t n_rays,
                           const float* rays_o, const float* rays_d, const float* t_samples,
                           double* rgb, double* depth, double* wsum, double* logT_final,
                           double* margin, int32_t n_threads)
{
    const int err = check_model(m, p);
    if (err) return err;
    job jb;
    memset(&jb, 0, sizeof(jb));
    jb.m = m;
    jb.p = p;
    jb.n_rays = n_rays;
    jb.o = rays_o;
    jb.d = rays_d;
    jb.t_given = t_samples;
    jb.rgb = rgb;
    jb.depth = depth;
    jb.wsum = wsum;
    jb.logT = logT_final;
    jb.margin = margin;
    return run_jobs(&jb, n_threads);
}

int32_t orc_render_backward(const orc_model* m, const orc_params* p, int64_t n_rays,
                            const float* rays_o, const float* rays_d, const float* t_samples,
                            const double* d_rgb, const double* d_depth, const double* d_wsum,
                            double* g_sdf, double* g_feat, double* g_probe, double* g_mlp,
                            int32_t n_threads)
{
    const int err = check_model(m, p);
    if (err) return err;
    job jb;
    memset(&jb, 0, sizeof(jb));
    jb.m = m;
    jb.p = p;
    jb.n_rays = n_rays;
    jb.o = rays_o;
    jb.d = rays_d;
    jb.t_given = t_samples;
    jb.drgb = d_rgb;
    jb.ddepth = d_depth;
    jb.dwsum = d_wsum;
    jb.backward = 1;
    jb.sink.g_sdf = g_sdf;
    jb.sink.g_feat = g_feat;
    jb.sink.g_probe = g_probe;
    jb.sink.g_mlp = g_mlp;
    return run_jobs(&jb, n_threads);
}

int32_t orc_render_trace(const orc_model* m, const orc_params* p, const float* o, const float* d,
                         const float* t_samples, float* t, double* s, double* w, double* C,
                         double* normal)
{
    const int err = check_model(m, p);
    if (err) return err;
    ray_work rw;
    alloc_work(p, &rw);
    double rgb[3], depth, wsum, logT;
    const int hit = forward_ray(m, p, o, d, t_samples, &rw, rgb, &depth, &wsum, &logT, NULL);
    const int N = p->n_samples;
    for (int k = 0; k <= N; ++k) {
        t[k] = hit ? rw.t[k] : 0.0f;
        s[k] = hit ? rw.S[k].s : 0.0;
    }
    for (int k = 0; k < N; ++k) {
        w[k] = hit ? rw.w[k] : 0.0;
        for (int c = 0; c < 3; ++c) {
            C[3 * k + c] = hit ? rw.S[k].C[c] : 0.0;
            normal[3 * k + c] = hit ? rw.S[k].n[c] : 0.0;
        }
    }
    free_work(&rw);
    return hit;
}

int32_t orc_point_eval(const orc_model* m, const orc_params* p, const float o[3],
                       const float d[3], float t, double* s, double g[3], double* mlp_in,
                       double C[3])
{
    const int err = check_model(m, p);
    if (err) return err;
    orc_sample S;
    eval_point(m, p, o, d, t, 1, &S, NULL);
    *s = S.s;
    for (int a = 0; a < 3; ++a) g[a] = S.g[a];
    for (int i = 0; i < mlp_n_in(m); ++i) mlp_in[i] = S.x[i];
    for (int c = 0; c < 3; ++c) C[c] = S.C[c];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Learned sample proposal.  Not part of the paper: a per-ray MLP predicts  */
/* how the render's weight is spread over B equal bins of the ray's segment */
/* in the box, and the samples are placed at quantiles of that density.     */
/* ------------------------------------------------------------------------ */

/* Coarse occupancy: cell c of res cells along an axis covers the fine nodes
 * floor(c (R-1) / res) .. ceil((c+1) (R-1) / res); it is occupied (1) when
 * the smallest |s| over those nodes is below `threshold`. */
int32_t orc_occupancy(const orc_model* m, const int32_t res[3], double threshold, double* occ)
{
    for (int a = 0; a < 3; ++a)
        if (res[a] < 1) return -2;
    for (int cz = 0; cz < res[2]; ++cz)
        for (int cy = 0; cy < res[1]; ++cy)
            for (int cx = 0; cx < res[0]; ++cx) {
                const int c[3] = {cx, cy, cz};
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    const int64_t span = (int64_t)(m->R[a] - 1);
                    lo[a] = (int)((c[a] * span) / res[a]);
                    hi[a] = (int)(((c[a] + 1) * span + res[a] - 1) / res[a]);
                    if (hi[a] > m->R[a] - 1) hi[a] = m->R[a] - 1;
                }
                double mn = INFINITY;
                for (int iz = lo[2]; iz <= hi[2]; ++iz)
                    for (int iy = lo[1]; iy <= hi[1]; ++iy)
                        for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                            const double v = fabs(m->sdf[node_index(m->R, ix, iy, iz)]);
                            if (v < mn) mn = v;
                        }
                occ[((size_t)cz * res[1] + cy) * res[0] + cx] = mn < threshold ? 1.0 : 0.0;
            }
    return 0;
}

/* Occupancy features of a ray: the segment [t_n, t_f] is cut into B n_sub
 * equal sub-intervals whose centres are looked up in the occupancy cell that
 * contains them.  frac[b] is the occupied share of bin b's n_sub points,
 * *first the position (j + 1/2) / (B n_sub) of the first occupied point j
 * (1 when none is) and step[b] = clamp(B *first - b, 0, 1) the share of bin b
 * that lies before it.  The positions and cell indices decide integers, so they
 * are computed in FP32 with the roundings the kernel uses (FP contraction off,
 * fmaf a fused multiply-add). */
static void ray_occupancy(const orc_model* m, const orc_proposal* pr, const float o[3],
                          const float d[3], float tn, float tf, double* frac, double* first,
                          double* step)
{
    const int B = pr->n_bins, S = pr->n_sub;
    const float seg = (tf - tn) / (float)(B * S);
    float inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = (float)pr->occ_res[a] / (m->bmax[a] - m->bmin[a]);
    *first = 1.0;
    for (int b = 0; b < B; ++b) {
        int count = 0;
        for (int j = 0; j < S; ++j) {
            const float t = fmaf((float)(b * S + j) + 0.5f, seg, tn);
            int c[3];
            for (int a = 0; a < 3; ++a) {
                const float x = fmaf(t, d[a], o[a]);
                float u = (x - m->bmin[a]) * inv[a];
                u = fminf(fmaxf(u, 0.0f), (float)(pr->occ_res[a] - 1));
                c[a] = (int)floorf(u);
            }
            const size_t cell = ((size_t)c[2] * pr->occ_res[1] + c[1]) * pr->occ_res[0] + c[0];
            if (pr->occ[cell] > 0.5) {
                if (*first == 1.0) *first = (b * S + j + 0.5) / (B * S);
                ++count;
            }
        }
        frac[b] = (double)count / S;
    }
    for (int b = 0; b < B; ++b) {
        const double v = B * *first - b;
        step[b] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
}

typedef struct {
    int hit;
    float tn, tf;
    double x[ORC_MAX_IN], z1[ORC_MAX_W], h1[ORC_MAX_W], z2[ORC_MAX_W], h2[ORC_MAX_W];
    double logit[ORC_MAX_IN], p[ORC_MAX_IN];
} prop_state;

/* Proposal MLP input [(o - centre)/extent, d, first occupied position,
 * occupied fraction of the B bins, share of each bin before the first
 * occupied point]
 * -> W -> W -> B logits (ReLU hidden layers), softmax. */
static void proposal_eval(const orc_model* m, const orc_proposal* pr, const float* o,
                          const float* d, prop_state* st)
{
    const int B = pr->n_bins, W = pr->width, nin = 7 + 2 * B;
    st->hit = ray_box_f32(o, d, m->bmin, m->bmax, &st->tn, &st->tf);
    for (int a = 0; a < 3; ++a) {
        const double c = 0.5 * ((double)m->bmin[a] + (double)m->bmax[a]);
        const double e = (double)m->bmax[a] - (double)m->bmin[a];
        st->x[a] = ((double)o[a] - c) / e;
        st->x[3 + a] = (double)d[a];
    }
    if (st->hit) {
        ray_occupancy(m, pr, o, d, st->tn, st->tf, st->x + 7, st->x + 6, st->x + 7 + B);
    } else {
        st->x[6] = 1.0;
        for (int b = 0; b < B; ++b) {
            st->x[7 + b] = 0.0;
            st->x[7 + B + b] = 1.0;
        }
    }
    const double* W1 = pr->params;
    const double* b1 = W1 + W * nin;
    const double* W2 = b1 + W;
    const double* b2 = W2 + W * W;
    const double* W3 = b2 + W;
    const double* b3 = W3 + B * W;
    for (int u = 0; u < W; ++u) {
        double z = b1[u];
        for (int i = 0; i < nin; ++i) z += W1[u * nin + i] * st->x[i];
        st->z1[u] = z;
        st->h1[u] = relu(z);
    }
    for (int u = 0; u < W; ++u) {
        double z = b2[u];
        for (int i = 0; i < W; ++i) z += W2[u * W + i] * st->h1[i];
        st->z2[u] = z;
        st->h2[u] = relu(z);
    }
    double mx = -INFINITY;
    for (int b = 0; b < B; ++b) {
        double z = b3[b];
        for (int i = 0; i < W; ++i) z += W3[b * W + i] * st->h2[i];
        st->logit[b] = z;
        if (z > mx) mx = z;
    }
    double sum = 0.0;
    for (int b = 0; b < B; ++b) {
        st->p[b] = exp(st->logit[b] - mx);
        sum += st->p[b];
    }
    for (int b = 0; b < B; ++b) st->p[b] /= sum;
}

/* Samples at the quantiles k / n_out, k = 0..n_out, of the piecewise-constant
 * density q over B equal bins of [t_n, t_f]: the sample's bin is where the
 * running sum of q first passes k / n_out, and it sits at the matching
 * fraction of that bin. */
static void place_quantiles(double tn, double tf, const double* q, int B, int n_out, double* t)
{
    const double db = (tf - tn) / B;
    for (int k = 0; k <= n_out; ++k) {
        const double u = (double)k / n_out;
        double c = 0.0;
        int b = 0;
        while (b < B - 1 && c + q[b] <= u) {
            c += q[b];
            ++b;
        }
        double frac = (u - c) / q[b];
        if (frac > 1.0) frac = 1.0;
        t[k] = tn + (b + frac) * db;
    }
    t[0] = tn;
    t[n_out] = tf;
}

int32_t orc_proposal_forward(const orc_model* m, const orc_proposal* pr, int64_t n_rays,
                             const float* rays_o, const float* rays_d, int32_t n_out,
                             double* logits, double* probs, double* t_samples, double* margin)
{
    const int B = pr->n_bins;
    if (B < 1 || 7 + 2 * B > ORC_MAX_IN || pr->width < 1 || pr->width > ORC_MAX_W || n_out < 1 ||
        pr->n_sub < 1)
        return -2;
    prop_state st;
    for (int64_t r = 0; r < n_rays; ++r) {
        proposal_eval(m, pr, rays_o + 3 * r, rays_d + 3 * r, &st);
        if (margin) {
            /* smallest |pre-activation| of a hidden unit: how far the ray is
             * from a ReLU kink, where FP32 and FP64 may switch a unit apart */
            double mg = INFINITY;
            for (int u = 0; u < pr->width; ++u) {
                if (fabs(st.z1[u]) < mg) mg = fabs(st.z1[u]);
                if (fabs(st.z2[u]) < mg) mg = fabs(st.z2[u]);
            }
            margin[r] = mg;
        }
        /* mixed density p' = (1 - mix) p + mix r: r puts a quarter of the mix
         * share on every bin and three quarters evenly on the bins that hold
         * an occupied point or neighbour a bin that does (all of it uniformly
         * when none does); p' is uniform when its peak is below theta */
        double near[ORC_MAX_IN], nr = 0.0;
        for (int b = 0; b < B; ++b) {
            const int nb = st.x[7 + b] > 0.0 || (b > 0 && st.x[6 + b] > 0.0) ||
                           (b + 1 < B && st.x[8 + b] > 0.0);
            near[b] = nb ? 1.0 : 0.0;
            nr += near[b];
        }
        double q[ORC_MAX_IN], qmax = 0.0;
        for (int b = 0; b < B; ++b) {
            const double rb = nr > 0.0 ? 0.75 * near[b] / nr + 0.25 / B : 1.0 / B;
            q[b] = (1.0 - pr->mix) * st.p[b] + pr->mix * rb;
            if (q[b] > qmax) qmax = q[b];
        }
        if (qmax < pr->theta)
            for (int b = 0; b < B; ++b) q[b] = 1.0 / B;
        for (int b = 0; b < B; ++b) {
            if (logits) logits[r * B + b] = st.logit[b];
            if (probs) probs[r * B + b] = q[b];
        }
        if (!t_samples) continue;
        double* t = t_samples + r * (n_out + 1);
        if (!st.hit) {
            for (int k = 0; k <= n_out; ++k) t[k] = 0.0;
            continue;
        }
        place_quantiles(st.tn, st.tf, q, B, n_out, t);
    }
    return 0;
}

int32_t orc_place_samples(const orc_model* m, int64_t n_rays, const float* rays_o,
                          const float* rays_d, const double* q, int32_t n_bins, int32_t n_out,
                          double* t_samples)
{
    if (n_bins < 1 || n_out < 1) return -2;
    for (int64_t r = 0; r < n_rays; ++r) {
        float tn, tf;
        double* t = t_samples + r * (n_out + 1);
        if (!ray_box_f32(rays_o + 3 * r, rays_d + 3 * r, m->bmin, m->bmax, &tn, &tf)) {
            for (int k = 0; k <= n_out; ++k) t[k] = 0.0;
            continue;
        }
        place_quantiles(tn, tf, q + r * n_bins, n_bins, n_out, t);
    }
    return 0;
}

/* Per-bin sums of the uniform render's weights w_k (the proposal's target). */
int32_t orc_weight_histogram(const orc_model* m, const orc_params* p, int64_t n_rays,
                             const float* rays_o, const float* rays_d, int32_t n_bins,
                             double* hist, int32_t n_threads)
{
    (void)n_threads;
    const int err = check_model(m, p);
    if (err) return err;
    const int N = p->n_samples;
    if (n_bins < 1 || N % n_bins) return -2;
    ray_work rw;
    alloc_work(p, &rw);
    for (int64_t r = 0; r < n_rays; ++r) {
        double rgb[3], depth, wsum, logT;
        const int hit = forward_ray(m, p, rays_o + 3 * r, rays_d + 3 * r, NULL, &rw, rgb, &depth,
                                    &wsum, &logT, NULL);
        for (int b = 0; b < n_bins; ++b) hist[r * n_bins + b] = 0.0;
        if (!hit) continue;
        for (int k = 0; k < N; ++k) hist[r * n_bins + k / (N / n_bins)] += rw.w[k];
    }
    free_work(&rw);
    return 0;
}

/* Loss of a ray: the cross-entropy of the weight histogram against the
 * proposal's softmax, weighted by the ray's weight mass,
 * loss_r = -sum_b hist_b log p_b (rays with mass below min_mass skipped);
 * gradients of scale * sum_r loss_r with respect to the proposal parameters
 * (d loss / d logit_b = mass p_b - hist_b). */
int32_t orc_proposal_backward(const orc_model* m, const orc_proposal* pr, int64_t n_rays,
                              const float* rays_o, const float* rays_d, const double* hist,
                              double min_mass, double scale, double* g_params, double* loss)
{
    const int B = pr->n_bins, W = pr->width, nin = 7 + 2 * B;
    const double* W1 = pr->params;
    const double* b1 = W1 + W * nin;
    const double* W2 = b1 + W;
    const double* b2 = W2 + W * W;
    const double* W3 = b2 + W;
    (void)b1;
    (void)b2;
    double* gW1 = g_params;
    double* gb1 = gW1 + W * nin;
    double* gW2 = gb1 + W;
    double* gb2 = gW2 + W * W;
    double* gW3 = gb2 + W;
    double* gb3 = gW3 + B * W;
    prop_state st;
    for (int64_t r = 0; r < n_rays; ++r) {
        if (loss) loss[r] = 0.0;
        double mass = 0.0;
        for (int b = 0; b < B; ++b) mass += hist[r * B + b];
        if (!(mass >= min_mass)) continue;
        proposal_eval(m, pr, rays_o + 3 * r, rays_d + 3 * r, &st);
        double dl[ORC_MAX_IN], dh2[ORC_MAX_W], dz2[ORC_MAX_W], dh1[ORC_MAX_W], dz1[ORC_MAX_W];
        double ce = 0.0;
        for (int b = 0; b < B; ++b) {
            ce -= hist[r * B + b] * log(st.p[b]);
            dl[b] = scale * (mass * st.p[b] - hist[r * B + b]);
        }
        if (loss) loss[r] = ce;
        for (int b = 0; b < B; ++b) {
            gb3[b] += dl[b];
            for (int i = 0; i < W; ++i) gW3[b * W + i] += dl[b] * st.h2[i];
        }
        for (int i = 0; i < W; ++i) {
            double a = 0.0;
            for (int b = 0; b < B; ++b) a += W3[b * W + i] * dl[b];
            dh2[i] = a;
            dz2[i] = st.z2[i] > 0.0 ? a : 0.0;
        }
        for (int u = 0; u < W; ++u) {
            gb2[u] += dz2[u];
            for (int i = 0; i < W; ++i) gW2[u * W + i] += dz2[u] * st.h1[i];
        }
        for (int i = 0; i < W; ++i) {
            double a = 0.0;
            for (int u = 0; u < W; ++u) a += W2[u * W + i] * dz2[u];
            dh1[i] = a;
            dz1[i] = st.z1[i] > 0.0 ? a : 0.0;
        }
        for (int u = 0; u < W; ++u) {
            gb1[u] += dz1[u];
            for (int i = 0; i < nin; ++i) gW1[u * nin + i] += dz1[u] * st.x[i];
        }
        (void)dh1;
        (void)dh2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Two-pass inference (the paper's viewer: "shading" assigns a colour to    */
/* every voxel for the current view, then "render" samples the SDF and the  */
/* colour field along the rays; Sec. "Performance Analysis", Tab. 8).        */
/* ------------------------------------------------------------------------ */

/* Colour of node nd (Rx Ry Rz order) seen from cam, or 0 outside the band. */
static void shade_node(const orc_model* m, const orc_params* p, const double cam[3], double band,
                       size_t nd, orc_sample* S, double C[3])
{
    const int i[3] = {(int)(nd % (size_t)m->R[0]), (int)((nd / (size_t)m->R[0]) % (size_t)m->R[1]),
                      (int)(nd / ((size_t)m->R[0] * (size_t)m->R[1]))};
    const double s = m->sdf[nd];
    if (!(fabs(s) < band)) { /* outside the band: not shaded */
        C[0] = C[1] = C[2] = 0.0;
        return;
    }
    double h[3];
    for (int a = 0; a < 3; ++a)
        h[a] = ((double)m->bmax[a] - (double)m->bmin[a]) / (double)(m->R[a] - 1);
    /* SDF gradient at the node: central differences, one-sided on the faces */
    for (int a = 0; a < 3; ++a) {
        int ip[3] = {i[0], i[1], i[2]}, im[3] = {i[0], i[1], i[2]};
        ip[a] = i[a] + 1 < m->R[a] ? i[a] + 1 : i[a];
        im[a] = i[a] > 0 ? i[a] - 1 : 0;
        const double sp = m->sdf[node_index(m->R, ip[0], ip[1], ip[2])];
        const double sm = m->sdf[node_index(m->R, im[0], im[1], im[2])];
        S->g[a] = (sp - sm) / ((double)(ip[a] - im[a]) * h[a]);
    }
    /* direction from the node to the camera */
    double v[3], len = 0.0;
    for (int a = 0; a < 3; ++a) {
        v[a] = cam[a] - ((double)m->bmin[a] + (double)i[a] * h[a]);
        len += v[a] * v[a];
    }
    len = sqrt(len);
    for (int a = 0; a < 3; ++a) v[a] /= len;
    /* spatial features at the node */
    if (m->feat_layout == ORC_FEAT_TRIPLANE) {
        int ci[3];
        double cf[3];
        for (int a = 0; a < 3; ++a) {
            ci[a] = i[a] < m->R[a] - 1 ? i[a] : m->R[a] - 2;
            cf[a] = (double)(i[a] - ci[a]);
        }
        tri_at T;
        triplane_locate(m, ci, cf, &T);
        triplane_features(m, &T, S->x);
    } else {
        for (int q = 0; q < m->n_s; ++q) S->x[q] = m->feat[nd * (size_t)m->n_s + q];
    }
    /* probe cell of the node: u = i (P - 1) / (R - 1) */
    for (int a = 0; a < 3; ++a) {
        const double u = (double)i[a] * (double)(m->P[a] - 1) / (double)(m->R[a] - 1);
        int pi = (int)floor(u);
        if (pi > m->P[a] - 2) pi = m->P[a] - 2;
        if (pi < 0) pi = 0;
        S->pi_[a] = pi;
        S->pf[a] = u - (double)pi;
    }
    angular_inputs(m, p, v, S);
    mlp_colour(m, S, NULL, p->mlp_f16);
    for (int c = 0; c < 3; ++c) C[c] = S->C[c];
}

int32_t orc_shade_nodes(const orc_model* m, const orc_params* p, const double cam[3],
                        double band, double* colours)
{
    const int rc = check_model(m, p);
    if (rc) return rc;
    if (!cam || !colours) return -1;
    orc_sample* S = (orc_sample*)calloc(1, sizeof(orc_sample));
    if (!S) return -3;
    const size_t n = (size_t)m->R[0] * (size_t)m->R[1] * (size_t)m->R[2];
    for (size_t nd = 0; nd < n; ++nd) shade_node(m, p, cam, band, nd, S, colours + 3 * nd);
    free(S);
    return 0;
}

int32_t orc_shade_node_list(const orc_model* m, const orc_params* p, const double cam[3],
                            double band, int64_t n, const int64_t* nodes, double* colours)
{
    const int rc = check_model(m, p);
    if (rc) return rc;
    if (!cam || n < 0 || (n > 0 && (!nodes || !colours))) return -1;
    const int64_t total = (int64_t)m->R[0] * m->R[1] * m->R[2];
    for (int64_t k = 0; k < n; ++k)
        if (nodes[k] < 0 || nodes[k] >= total) return -1;
    orc_sample* S = (orc_sample*)calloc(1, sizeof(orc_sample));
    if (!S) return -3;
    for (int64_t k = 0; k < n; ++k)
        shade_node(m, p, cam, band, (size_t)nodes[k], S, colours + 3 * k);
    free(S);
    return 0;
}

int32_t orc_render_colour_field(const orc_model* m, const orc_params* p, const double* colours,
                                int64_t n_rays, const float* rays_o, const float* rays_d,
                                const float* t_samples, double* rgb, double* depth, double* wsum)
{
    const int rc = check_model(m, p);
    if (rc) return rc;
    if (n_rays < 0 || (n_rays > 0 && (!colours || !rays_o || !rays_d || !rgb || !depth || !wsum)))
        return -1;
    const int N = p->n_samples;
    float* t = (float*)malloc(sizeof(float) * (size_t)(N + 1));
    double* s = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    double* col = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    orc_sample* S = (orc_sample*)calloc(1, sizeof(orc_sample));
    if (!t || !s || !col || !S) {
        free(t), free(s), free(col), free(S);
        return -3;
    }
    for (int64_t r = 0; r < n_rays; ++r) {
        const float* o = rays_o + 3 * r;
        const float* d = rays_d + 3 * r;
        const float* tg = t_samples ? t_samples + r * (int64_t)(N + 1) : NULL;
        if (!ray_samples(m, p, o, d, tg, t)) {
            for (int c = 0; c < 3; ++c) rgb[3 * r + c] = p->bg[c];
            depth[r] = wsum[r] = 0.0;
            continue;
        }
        /* SDF at the N + 1 points; colour of sample k: trilinear blend of the
         * node colours of the cell holding point k */
        for (int k = 0; k <= N; ++k) {
            eval_point(m, p, o, d, t[k], 0, S, NULL);
            s[k] = S->s;
            if (k == N) break;
            for (int c = 0; c < 3; ++c) col[3 * k + c] = 0.0;
            for (int q = 0; q < 8; ++q) {
                const int cx = q & 1, cy = (q >> 1) & 1, cz = (q >> 2) & 1;
                double w;
                corner_weight(S->cf, cx, cy, cz, &w, NULL);
                const size_t nd = node_index(m->R, S->ci[0] + cx, S->ci[1] + cy, S->ci[2] + cz);
                for (int c = 0; c < 3; ++c) col[3 * k + c] += w * colours[3 * nd + c];
            }
        }
        /* NeuS opacity and compositing (Eqs. 8-10), as in the per-sample render */
        double acc[3] = {0, 0, 0}, dep = 0.0, ws = 0.0, logT = 0.0;
        for (int k = 0; k < N; ++k) {
            const double diff = log_phi(p->tau, s[k + 1]) - log_phi(p->tau, s[k]);
            const double lam = diff < 0.0 ? diff : 0.0;
            const double w = exp(logT) * -expm1(lam);
            for (int c = 0; c < 3; ++c) acc[c] += w * col[3 * k + c];
            dep += w * (double)t[k];
            ws += w;
            logT += lam;
        }
        const double TN = exp(logT);
        for (int c = 0; c < 3; ++c) rgb[3 * r + c] = acc[c] + TN * p->bg[c];
        depth[r] = dep;
        wsum[r] = ws;
    }
    free(t), free(s), free(col), free(S);
    return 0;
}
