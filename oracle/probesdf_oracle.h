/*
 * FP64 CPU oracle of the ProbeSDF per-ray render and adjoint.
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.
 */
#ifndef PROBESDF_ORACLE_H
#define PROBESDF_ORACLE_H

#include <stdint.h>

#define ORC_MAX_NS 16
#define ORC_MAX_NA 16
#define ORC_MAX_K 8
#define ORC_MAX_L2 16
#define ORC_MAX_W 64
#define ORC_MAX_IN 48

#define ORC_DIR_REFLECT 0
#define ORC_DIR_VIEW 1

typedef struct orc_model {
    int32_t R[3];          /* SDF / feature nodes per axis (x, y, z) */
    float bmin[3];         /* grid box, FP32 as the kernel sees it */
    float bmax[3];
    int32_t n_s;           /* spatial features per node */
    const double* sdf;     /* [Rz][Ry][Rx] */
    const double* feat;    /* [Rz][Ry][Rx][n_s] */
    int32_t P[3];          /* probe nodes per axis, same box */
    int32_t sh_l;          /* SH order l (1-indexed): l*l coefficients */
    int32_t n_a;           /* angular feature channels */
    const double* probes;  /* [Pz][Py][Px][l*l][n_a] */
    int32_t width;         /* MLP hidden width W */
    int32_t n_fresnel;     /* K: Fresnel powers 1..K */
    const double* mlp;     /* W1[W][n_in] b1[W] W2[W][W] b2[W] W3[3][W] b3[3] */
    int32_t feat_layout;   /* ORC_FEAT_NODES: feat per node; ORC_FEAT_TRIPLANE: planes */
    const double* planes;  /* [tz][ty][tx][3][16][16][n_s]: per 16^3 tile, the planes
                              orthogonal to x ([z][y]), y ([z][x]) and z ([y][x]) */
} orc_model;

#define ORC_FEAT_NODES 0
#define ORC_FEAT_TRIPLANE 1
#define ORC_TILE 16

typedef struct orc_params {
    double tau;            /* NeuS logistic scale */
    int32_t n_samples;     /* N colour samples, N+1 SDF points */
    int32_t dir_mode;      /* ORC_DIR_REFLECT or ORC_DIR_VIEW */
    double bg[3];          /* background colour */
    int32_t sdf_fp32;      /* 1: the SDF value at a point by the FP32 sequence of the
                              render kernels (weights and fused multiply-adds in FP32,
                              corner order x fastest) instead of FP64; only tests that
                              isolate FP32 rounding of s set it */
    int32_t mlp_f16;       /* 1: the colour MLP's layer-1 and layer-2 inputs (the input
                              vector and the first hidden activations) rounded to the
                              nearest binary16 value before their products, as a
                              reduced-precision FP16 evaluation stores them; products,
                              sums, the output layer and the adjoint stay FP64 (the
                              adjoint treats the rounding as the identity) */
} orc_params;

/* v rounded to the nearest IEEE binary16 value (ties to even), returned as a
 * double; magnitudes that round beyond the largest finite binary16 value give
 * +-inf; zeros, infinities and NaN are returned unchanged. */
double orc_round_f16(double v);

void orc_sh_eval(int32_t l, const double r[3], double* Y);
void orc_sh_grad(int32_t l, const double r[3], double* dY);

int32_t orc_render_forward(const orc_model* m, const orc_params* p, int64_t n_rays,
                           const float* rays_o, const float* rays_d, const float* t_samples,
                           double* rgb, double* depth, double* wsum, double* logT_final,
                           double* margin, int32_t n_threads);

int32_t orc_render_backward(const orc_model* m, const orc_params* p, int64_t n_rays,
                            const float* rays_o, const float* rays_d, const float* t_samples,
                            const double* d_rgb, const double* d_depth, const double* d_wsum,
                            double* g_sdf, double* g_feat, double* g_probe, double* g_mlp,
                            int32_t n_threads);

int32_t orc_render_trace(const orc_model* m, const orc_params* p, const float* o, const float* d,
                         const float* t_samples, float* t, double* s, double* w, double* C,
                         double* normal);

int32_t orc_point_eval(const orc_model* m, const orc_params* p, const float o[3],
                       const float d[3], float t, double* s, double g[3], double* mlp_in,
                       double C[3]);

/* ---- Learned sample proposal (not in the paper: places the render's
 * samples where a small per-ray MLP expects the surface) ---- */

typedef struct orc_proposal {
    int32_t occ_res[3];     /* coarse occupancy cells along x, y, z (over the grid box) */
    const double* occ;      /* [res_z][res_y][res_x] in {0, 1} */
    int32_t width;          /* hidden width */
    int32_t n_bins;         /* bins of [t_n, t_f] */
    int32_t n_sub;          /* occupancy look-ups per bin */
    const double* params;   /* W1[W][7+2B] b1[W] W2[W][W] b2[W] W3[B][W] b3[B] */
    double mix;             /* p' = (1 - mix) softmax + mix / B */
    double theta;           /* uniform fallback if max p' < theta */
} orc_proposal;

int32_t orc_occupancy(const orc_model* m, const int32_t res[3], double threshold, double* occ);
int32_t orc_proposal_forward(const orc_model* m, const orc_proposal* pr, int64_t n_rays,
                             const float* rays_o, const float* rays_d, int32_t n_out,
                             double* logits, double* probs, double* t_samples, double* margin);
int32_t orc_place_samples(const orc_model* m, int64_t n_rays, const float* rays_o,
                          const float* rays_d, const double* q, int32_t n_bins, int32_t n_out,
                          double* t_samples);
int32_t orc_weight_histogram(const orc_model* m, const orc_params* p, int64_t n_rays,
                             const float* rays_o, const float* rays_d, int32_t n_bins,
                             double* hist, int32_t n_threads);
int32_t orc_proposal_backward(const orc_model* m, const orc_proposal* pr, int64_t n_rays,
                              const float* rays_o, const float* rays_d, const double* hist,
                              double min_mass, double scale, double* g_params, double* loss);

/* Two-pass inference.  orc_shade_nodes: colours [Rz][Ry][Rx][3] of every node
 * for a camera at cam: nodes with |s| < band get the MLP colour of the node
 * (gradient by central differences, one-sided on the faces; v towards the
 * camera; the node's own features or its tri-plane features; probes
 * interpolated at the node), the others 0.  orc_render_colour_field: the
 * NeuS march of orc_render_forward with the colour of sample k the trilinear
 * blend of `colours` over the cell holding point k. */
int32_t orc_shade_nodes(const orc_model* m, const orc_params* p, const double cam[3],
                        double band, double* colours);
/* orc_shade_nodes for the listed nodes only (linear indices, x fastest). */
int32_t orc_shade_node_list(const orc_model* m, const orc_params* p, const double cam[3],
                            double band, int64_t n, const int64_t* nodes, double* colours);
int32_t orc_render_colour_field(const orc_model* m, const orc_params* p, const double* colours,
                                int64_t n_rays, const float* rays_o, const float* rays_d,
                                const float* t_samples, double* rgb, double* depth, double* wsum);

#endif
