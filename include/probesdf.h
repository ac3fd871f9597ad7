/*
 * probesdf.h — C ABI of the GB300 (sm_103a) ProbeSDF per-ray render library.
 *
 * The library evaluates the appearance and rendering model of ProbeSDF
 * ("Light Field Probes For Neural Surface Reconstruction", CVPR 2025) for a
 * batch of camera rays, and its adjoint:
 *   - an explicit SDF grid, read by trilinear interpolation, with the normal
 *     taken from the SDF gradient (Sec. 3, Eq. 13);
 *   - spatial features F_s interpolated from the same grid nodes, or the
 *     product of three bilinear lookups in per-tile tri-planes (Sec. 3.1,
 *     Sec. 4); the grid dense or stored as sparse 16^3-node bricks;
 *   - angular features F_a: spherical-harmonic coefficients stored on a
 *     coarse probe grid, blended trilinearly and evaluated in the reflected
 *     (or view) direction (Sec. 3.2, Eqs. 5-7);
 *   - Fresnel inputs (1 - n.v)^k (Sec. 3.1, Eq. 4);
 *   - a 2-hidden-layer ReLU MLP with a sigmoid output (Sec. 4);
 *   - NeuS opacities and front-to-back alpha compositing of colour, depth
 *     and accumulated weight (Sec. 3.3, Eqs. 8-10).
 * Beside the render: the grid-level training terms (Gaussian smoothing of the
 * raw SDF, Eikonal / normal / feature / probe smoothness, Eqs. 11-15) and an
 * Adam step; the two-pass inference of the paper's viewer (per-view node
 * colours, then a march over the colour field); and a learned sample proposal
 * (not in the paper).
 *
 * Conventions for every entry point:
 *   - Every pointer marked "device" is a CUDA device pointer owned by the
 *     caller, contiguous, 16-byte aligned, and valid on `stream` for the
 *     duration of the work enqueued by the call.  The library never frees or
 *     retains device memory and allocates no device memory.
 *   - Handles (psdf_grid, psdf_probes, psdf_mlp) are small host structs that
 *     hold a copy of the descriptor and a NON-owning device pointer to the
 *     parameter values.  Destroying a handle frees only the host struct.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are asynchronous with respect to the host.
 *   - Errors found on the host (bad descriptor, null or misaligned pointer,
 *     unsupported combination) return immediately with a negative status and
 *     enqueue nothing.  A failing CUDA launch returns PSDF_ERR_CUDA; the
 *     cudaError_t is available from psdf_last_cuda_error() on the same host
 *     thread.  No C++ exception crosses this boundary.
 *   - Nothing here synchronises the stream.
 *
 * Axes: dims[0..2] are the node counts along x, y, z; arrays are stored with
 * x fastest ([z][y][x]).  Both grids span the same box and are node-aligned:
 * node i along an axis sits at box_min + i (box_max - box_min) / (dims - 1).
 */
#ifndef PROBESDF_H
#define PROBESDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t psdf_status;

#define PSDF_OK 0
#define PSDF_ERR_INVALID_ARG -1   /* null pointer, negative count, bad enum */
#define PSDF_ERR_BAD_SHAPE -2     /* a dimension outside the supported range */
#define PSDF_ERR_BAD_DTYPE -3     /* a dtype enum the call does not take */
#define PSDF_ERR_MISALIGNED -4    /* a device pointer not 16-byte aligned */
#define PSDF_ERR_CUDA -5          /* a CUDA call failed; see psdf_last_cuda_error */
#define PSDF_ERR_UNSUPPORTED -6   /* a valid but not compiled-in combination */

#define PSDF_F32 0
#define PSDF_BF16 1
#define PSDF_F16 2

#define PSDF_DIR_REFLECT 0  /* F_a looked up with r = 2(n.v)n - v (Sec. 3.1) */
#define PSDF_DIR_VIEW 1     /* F_a looked up with v, for retro-reflective materials (Sec. 3.1) */

#define PSDF_GRID_VALUES 0
#define PSDF_GRID_GRAD 1

#define PSDF_FEAT_NODES 0     /* n_feat features stored at every grid node */
#define PSDF_FEAT_TRIPLANE 1  /* tile tri-planes (Sec. 3.1): per 16^3-cell tile, three
                                 16 x 16 planes; F_s = F_x * F_y * F_z per channel */
#define PSDF_TILE 16

/* SDF + spatial-feature grid (Sec. 3, "explicit SDF grid"; Sec. 3.1 F_s). */
typedef struct psdf_grid_desc {
    int32_t dims[3];     /* nodes along x, y, z; each in [2, 4096], product < 2^31 */
    float box_min[3];    /* world-space box spanned by the nodes */
    float box_max[3];    /* box_max > box_min on every axis */
    int32_t n_feat;      /* spatial features per node (n_s); 3 is compiled in */
    int32_t feat_dtype;  /* PSDF_F32 or PSDF_BF16 (storage of the features; SDF stays FP32) */
    int32_t feat_layout; /* PSDF_FEAT_NODES, or PSDF_FEAT_TRIPLANE (FP32 features only):
                            the cells form tiles of 16^3 (tiles_a = ceil((dims_a - 1) / 16));
                            a tile holds three planes of 16 x 16 texels, orthogonal to x
                            (indexed [z][y]), y ([z][x]) and z ([y][x]), texel (r, c) at the
                            centre of the tile's cell row r, column c; a point's spatial
                            feature c is the product of the three planes' bilinear lookups
                            at its in-plane coordinates (texel coordinate clamped to the
                            tile) */
    int32_t n_bricks;    /* 0: dense.  > 0: sparse (FP32 node features only): the nodes
                            form bricks of 16^3 (dims must be multiples of 16) and only
                            n_bricks of them are stored; see psdf_grid_bytes */
    float empty_sdf;     /* sparse: the SDF value of every node of a brick that is not
                            stored (> 0: empty space outside the surface); its features
                            are 0.  A sample whose 8 corners all lie in such bricks has
                            s = empty_sdf exactly.  Sparse grids are read by the render
                            forward and adjoint, the occupancy build, the weight histogram,
                            node shading, the colour-field march, the SDF smoothing
                            and its adjoint, and the SDF regularisers */
} psdf_grid_desc;

/* Light-field probe grid (Sec. 3.2): l*l SH coefficients of n_a channels. */
typedef struct psdf_probe_desc {
    int32_t dims[3];     /* probe nodes along x, y, z over the grid's box; each >= 2 */
    int32_t sh_l;        /* SH order l, 1-indexed as in Eq. 5 (l*l coefficients); 3 compiled
                            in, and 4 (16 coefficients, Sec. 4) with 4 channels and width 32 */
    int32_t n_ang;       /* angular channels n_a; 4 and 8 compiled in */
    int32_t dtype;       /* PSDF_F32 or PSDF_F16 (storage of the coefficients) */
} psdf_probe_desc;

/* Colour MLP (Sec. 4): n_in -> width -> width -> 3, ReLU, ReLU, sigmoid.
 * n_in = n_s + n_a + n_fresnel; parameters packed row-major as
 * W1[width][n_in] b1[width] W2[width][width] b2[width] W3[3][width] b3[3]. */
typedef struct psdf_mlp_desc {
    int32_t n_in;
    int32_t width;       /* 16 and 32 compiled in */
    int32_t dtype;       /* arithmetic: PSDF_F32 (FP32-equivalent: FP16 hi/lo split on the
                            tensor cores, FP32 accumulation) or PSDF_F16 (FP16 operands, FP32
                            accumulation); the parameters are FP32 in memory either way */
} psdf_mlp_desc;

typedef struct psdf_render_params {
    float tau;           /* NeuS logistic scale of Eq. 10, > 0 */
    int32_t n_samples;   /* N colour samples per ray (N+1 SDF points), in [1, 4096] */
    int32_t dir_mode;    /* PSDF_DIR_REFLECT or PSDF_DIR_VIEW */
    int32_t n_fresnel;   /* K: inputs (1 - n.v)^1..K (Eq. 4 uses powers of 1 - n.v); 3 compiled in */
    float bg[3];         /* background colour added with the final transmittance */
    int32_t n_bins;      /* 0: t_samples (if given) are sample distances; B in [1, 32]:
                            t_samples are per-bin densities (see psdf_render_forward) */
} psdf_render_params;

typedef struct psdf_grid psdf_grid;
typedef struct psdf_probes psdf_probes;
typedef struct psdf_mlp psdf_mlp;

/* Human-readable text of a status code (static storage). */
const char* psdf_status_string(psdf_status status);

/* cudaError_t (as int) of the last call on this host thread that returned
 * PSDF_ERR_CUDA; 0 if none. */
int32_t psdf_last_cuda_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t psdf_version(void);

/* Synchronises `stream`, then reads and clears the device status word of the
 * current device into *flags: 0 = no device-side error since the last call;
 * bit 0 = a kernel gave up waiting for its tensor-core work (the kernel
 * stopped early; its outputs are not valid).  Kernels never trap: they
 * record the condition here and return. */
psdf_status psdf_device_status(void* stream, int32_t* flags);

/* How many times each kernel launched afterwards from this host thread polls
 * a tensor-core completion (an mbarrier phase) before it gives up, records
 * bit 0 of the device status word, frees its tensor memory and returns
 * (after one more wait of the default length for the work already issued).
 * Default 2^24; 0xFFFFFFFF restores it.  A small value makes the waits run
 * out on purpose (a test of that path: every output of such a launch is then
 * invalid); the default is long enough that a wait only runs out when the
 * tensor core stops answering.  Thread-local, like psdf_last_cuda_error. */
psdf_status psdf_set_wait_polls(uint32_t polls);
uint32_t psdf_wait_polls(void);

/* Bytes of the packed grid values and of the grid gradient buffer.
 * Values, PSDF_F32 features: one 16-byte record {sdf, f0, f1, f2} per node.
 * Values, PSDF_BF16 features: an FP32 SDF array, then (at the next 16-byte
 * boundary) one 8-byte record {f0, f1, f2, 0} of BF16 per node.
 * Gradient (either case): one FP32 record {dsdf, df0, df1, df2} per node.
 * PSDF_FEAT_TRIPLANE, values and gradient alike: an FP32 SDF array, then (at the
 * next 16-byte boundary) the planes: [tz][ty][tx][3][16][16] texels of 16 bytes
 * {f0, f1, f2, 0}.
 * Sparse (n_bricks > 0), values and gradient alike: the brick table, int32
 * [Bz][By][Bx] (B_a = dims_a / 16; entry = the brick's slot in 0..n_bricks-1,
 * or -1 when it is not stored; padded to 16 bytes), then n_bricks blocks of
 * 16^3 FP32 node records {sdf, f0, f1, f2}, x fastest inside a block.  The
 * caller writes the table (the gradient buffer's table region is unused); each
 * slot in [0, n_bricks) may appear at most once (two entries naming one slot
 * would alias one record block: pack would write it from two threads at once
 * and the adjoint would add both bricks' gradients into it).  The library does
 * not check this: the table stays in device memory.
 * Node order is x fastest. */
psdf_status psdf_grid_bytes(const psdf_grid_desc* desc, size_t* values_bytes, size_t* grad_bytes);

/* Handle over caller-owned packed values (device, psdf_grid_bytes bytes). */
psdf_status psdf_grid_create(const psdf_grid_desc* desc, const void* values, psdf_grid** out);
void psdf_grid_destroy(psdf_grid* grid);

/* Dense <-> packed conversion on `stream`.
 * pack:   sdf (device, FP32 [Rz][Ry][Rx]) and feat (device, FP32
 *         [Rz][Ry][Rx][n_feat], or for tri-planes [tz][ty][tx][3][16][16][n_feat])
 *         -> packed values (device, values_bytes); BF16 features are rounded to
 *         nearest even.
 * unpack: packed values (which = PSDF_GRID_VALUES) or a gradient buffer
 *         (PSDF_GRID_GRAD) -> the dense arrays (either may be NULL).
 * Sparse grids: `packed` must already hold the brick table; pack copies the
 * stored bricks' nodes out of the dense arrays, unpack writes the stored
 * bricks and fills the others with {empty_sdf, 0, 0, 0} (values) or zeros
 * (gradient).  The table is read on the host side of neither call: it stays
 * in device memory. */
psdf_status psdf_grid_pack(const psdf_grid_desc* desc, const float* sdf, const float* feat,
                           void* packed, void* stream);
psdf_status psdf_grid_unpack(const psdf_grid_desc* desc, int32_t which, const void* packed,
                             float* sdf, float* feat, void* stream);

/* Probe coefficients (device, [Pz][Py][Px][l*l][n_a], FP32 or FP16 per the
 * descriptor); the layout is the caller's, no packing. */
psdf_status psdf_probes_create(const psdf_probe_desc* desc, const void* coeffs,
                               psdf_probes** out);
void psdf_probes_destroy(psdf_probes* probes);

/* MLP parameters (device, FP32, packed as in psdf_mlp_desc). */
psdf_status psdf_mlp_param_count(const psdf_mlp_desc* desc, int64_t* count);
psdf_status psdf_mlp_create(const psdf_mlp_desc* desc, const void* params, psdf_mlp** out);
void psdf_mlp_destroy(psdf_mlp* mlp);

/* Forward render (Eqs. 4-10, Sec. 4) of n_rays rays.
 *   rays_o, rays_d : device FP32 [n_rays][3]; rays_d must be unit length
 *                    (used as given; t is then a distance).
 *   t_samples      : NULL for N evenly spaced samples over the ray's segment
 *                    inside the box (slab test, t >= 0), or device FP32
 *                    [n_rays][N+1] of increasing sample distances (a ray with
 *                    t[N] <= t[0] is treated as a miss), or, when
 *                    params->n_bins = B > 0, device FP32 [n_rays][B] densities
 *                    q_b of B equal bins of the box segment [t_n, t_f] (as
 *                    psdf_proposal_forward returns in `probs`, summing to 1,
 *                    each > 0): sample k sits at the quantile k / N,
 *                    t_k = t_n + (b + (k/N - c_b) / q_b) (t_f - t_n) / B with
 *                    c_b = q_0 + .. + q_{b-1} and b the last bin with c_b <= k/N
 *                    (t_0 = t_n, t_N = t_f) -- the distances
 *                    psdf_proposal_forward writes to its t_samples.
 *   rgb            : device FP32 [n_rays][3] = sum_k w_k C_k + T_N bg
 *   depth          : device FP32 [n_rays]    = sum_k w_k t_k
 *   wsum           : device FP32 [n_rays]    = sum_k w_k
 *   logT_final     : device FP32 [n_rays]    = log T_N, needed by the backward
 *   n_live         : device int32 [n_rays] or NULL: 1 + the index of the ray's
 *                    last sample with a nonzero opacity alpha_k (0 when none
 *                    is, or the ray misses); lets the backward skip the
 *                    samples after it, whose adjoint terms are all zero
 * Rays that miss the box give rgb = bg and zeros elsewhere.  n_rays = 0 is a
 * valid no-op. */
psdf_status psdf_render_forward(const psdf_grid* grid, const psdf_probes* probes,
                                const psdf_mlp* mlp, const psdf_render_params* params,
                                const float* rays_o, const float* rays_d,
                                const float* t_samples, int64_t n_rays, float* rgb,
                                float* depth, float* wsum, float* logT_final, int32_t* n_live,
                                void* stream);

/* Adjoint of psdf_render_forward (Sec. 3.3-3.4: gradients for the SDF
 * values, spatial features, probe coefficients and MLP weights).  The
 * per-sample activations are recomputed, not stored.
 *   d_rgb          : device FP32 [n_rays][3] (required)
 *   d_depth, d_wsum: device FP32 [n_rays] or NULL (= zero)
 *   logT_final     : the forward's output for the same inputs
 *   n_live         : the forward's n_live for the same inputs, or NULL (every
 *                    sample of every ray is visited)
 *   grad_grid      : device FP32, grad_bytes of psdf_grid_bytes, {dsdf, df0..2} per node
 *   grad_probes    : device FP32 [Pz][Py][Px][l*l][n_a] (FP32 whatever the storage)
 *   grad_mlp       : device FP32 [psdf_mlp_param_count]
 * Gradients are ACCUMULATED (+=) with atomics, so their summation order is
 * not fixed; zero them first for a fresh gradient.  All three gradient
 * pointers are required. */
psdf_status psdf_render_backward(const psdf_grid* grid, const psdf_probes* probes,
                                 const psdf_mlp* mlp, const psdf_render_params* params,
                                 const float* rays_o, const float* rays_d,
                                 const float* t_samples, int64_t n_rays, const float* d_rgb,
                                 const float* d_depth, const float* d_wsum,
                                 const float* logT_final, const int32_t* n_live,
                                 float* grad_grid, float* grad_probes, float* grad_mlp,
                                 void* stream);

/* Resident CTAs per SM that psdf_render_forward / psdf_render_backward launch
 * with for these objects (each CTA renders 4 rays at a time).  Host query,
 * no kernel is launched. */
psdf_status psdf_render_occupancy(const psdf_grid* grid, const psdf_probes* probes,
                                  const psdf_mlp* mlp, const psdf_render_params* params,
                                  int32_t* forward_ctas_per_sm, int32_t* backward_ctas_per_sm);

/* ---------------------------------------------------------------------------
 * Optimiser.  The paper trains its grids, probes and MLP with Adam (Sec. 3.4);
 * this is the update of Kingma & Ba (2015, Algorithm 1) with bias correction:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)
 * (evaluated as lr_t m / (sqrt(v) + eps_t), lr_t and eps_t folded on the host).
 *   param, grad, m, v : device FP32 [n], m and v zero before step 1
 *   step              : 1-based update count (>= 1)
 *   clear_grad        : nonzero to zero grad in the same pass (the render's
 *                       and the proposal's backward calls accumulate)
 * Elementwise and in place; the four arrays must not overlap.
 * ------------------------------------------------------------------------- */

psdf_status psdf_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr,
                           float beta1, float beta2, float eps, int32_t step, int32_t clear_grad,
                           void* stream);

/* ---------------------------------------------------------------------------
 * Two-pass inference (the paper's viewer; Tab. 8 times its two kernels:
 * "shading" assigns every voxel a colour for the current view, "render"
 * samples the SDF and that colour field along the rays).  Per frame:
 * psdf_shade_nodes for the view's camera, then psdf_render_colour_field for
 * its rays.  The colour field is device memory of psdf_colour_field_bytes:
 * one 8-byte record {r, g, b, 0} of FP16 per grid node, x fastest.
 * ------------------------------------------------------------------------- */

psdf_status psdf_colour_field_bytes(const psdf_grid_desc* desc, size_t* bytes);

/* Colour of every node seen from a pinhole camera at `camera` (host FP32
 * [3], world units).  Nodes with |s| < band get the colour model's output
 * at the node: normal from the SDF gradient by central differences over the
 * node's neighbours (one-sided on the grid's faces; Eq. 13), v the unit
 * vector from the node to the camera, r per params->dir_mode, the node's own
 * spatial features (tri-planes: the lookup at the node), probes interpolated
 * at the node (Eqs. 5-7), Fresnel inputs (Eq. 4), the MLP (Sec. 4).  The other
 * nodes get 0.  Of params only dir_mode and n_fresnel are used (the rest must
 * be valid).  band >= 0 (0 shades nothing; +inf shades every node).  Every
 * record of `colours` is written.  A sparse grid's colour field is still one
 * record per node of the full grid; a node of a brick that is not stored
 * has s = empty_sdf and zero features. */
psdf_status psdf_shade_nodes(const psdf_grid* grid, const psdf_probes* probes,
                             const psdf_mlp* mlp, const psdf_render_params* params,
                             const float camera[3], float band, void* colours, void* stream);

/* The NeuS march of psdf_render_forward (same sample distances -- uniform,
 * explicit or from bin densities --, opacities and compositing, Eqs. 8-10)
 * with sample k's colour the trilinear blend of the colour field over the
 * 8 nodes of the SDF cell holding point k, in place of the colour model.
 * Outputs rgb [n_rays][3], depth, wsum [n_rays] as in psdf_render_forward.
 * Of params dir_mode and n_fresnel are not used. */
psdf_status psdf_render_colour_field(const psdf_grid* grid, const void* colours,
                                     const psdf_render_params* params, const float* rays_o,
                                     const float* rays_d, const float* t_samples,
                                     int64_t n_rays, float* rgb, float* depth, float* wsum,
                                     void* stream);

/* ---------------------------------------------------------------------------
 * Grid-level training terms (Sec. 3.3, Eqs. 11-15).  The trained SDF
 * parameter is a raw grid s_hat (device FP32 [Rz][Ry][Rx], x fastest, the
 * caller's); the grid the renderer reads holds its smoothing s = G(s_hat),
 * G the normalised 5^3 Gaussian (separable, 5 taps per axis, standard
 * deviation one node spacing, edge nodes replicated).  One training step:
 *   psdf_sdf_smooth -> render forward/backward -> psdf_grid_regularizers
 *   (+ psdf_probe_smoothness) -> psdf_sdf_smooth_adjoint (accumulate) ->
 *   psdf_adam_step on s_hat, the features, the probes and the MLP.
 * Finite differences: grad s at a node is the central difference over its
 * two neighbours per axis (node spacing h_a = (box_max - box_min) / (dims - 1)),
 * defined at interior nodes only.  All calls run on `stream`, launch without
 * synchronising and allocate nothing.
 * ------------------------------------------------------------------------- */

/* s = G(s_hat) written into the SDF slot of packed grid values (the layout of
 * psdf_grid_bytes; the features are not touched).  sdf_hat and the packed
 * values must not overlap.
 * Sparse grids (n_bricks > 0): s_hat is device FP32 [n_bricks][16][16][16],
 * the stored bricks in slot order, x fastest inside a brick.  G is that of the
 * full grid in which every node of an absent brick holds empty_sdf (in s_hat
 * and s alike); s is written at the stored nodes only, the table is read from
 * packed_values. */
psdf_status psdf_sdf_smooth(const psdf_grid_desc* desc, const float* sdf_hat, void* packed_values,
                            void* stream);

/* d_sdf_hat (+)= G^T dsdf: the SDF slot of a gradient buffer (psdf_grid_bytes'
 * grad layout) taken back through the smoothing.  accumulate = 0 overwrites
 * d_sdf_hat (device FP32 [Rz][Ry][Rx]), nonzero adds to it.
 * Sparse grids: d_sdf_hat is [n_bricks][16][16][16] as s_hat above; the brick
 * table is read from the gradient buffer's copy (so a caller that zeroes the
 * buffer zeroes its records, not the table), and the nodes of absent bricks
 * carry no gradient (their s is fixed). */
psdf_status psdf_sdf_smooth_adjoint(const psdf_grid_desc* desc, const void* grad_grid,
                                    float* d_sdf_hat, int32_t accumulate, void* stream);

/* The per-voxel terms on s = the SDF of packed_values, and the tri-plane term:
 *   L_sdf      = sum_i |s_i - s_hat_i|^2                         (Eq. 11)
 *   L_Eik      = sum_interior (||grad s|| - 1)^2                  (Eq. 12)
 *   L_normal   = sum_interior sum_a ||n(i + e_a) - n(i)||^2 over the axes whose
 *                neighbour is interior, n = grad s / sqrt(||grad s||^2 + 1e-24) (Eq. 13)
 *   L_features = sum over the tile planes of the squared forward differences
 *                between neighbouring texels, rows and columns     (Eq. 14)
 * The gradient of lam_sdf L_sdf + lam_eik L_Eik + lam_normal L_normal, each
 * voxel's term scaled by w_i = (1 + 5 |s_i|)^-1 (held fixed, not differentiated;
 * Sec. 3.3), is ADDED to the SDF slot of grad_grid (w.r.t. s) and
 * to d_sdf_hat (w.r.t. s_hat directly); lam_features * L_features' gradient is
 * added to the planes of grad_grid.  lam_features > 0 needs PSDF_FEAT_TRIPLANE
 * (PSDF_ERR_UNSUPPORTED otherwise).  All weights >= 0.
 *   loss : device FP32 [4] or NULL; {L_sdf, L_Eik, L_normal, L_features}
 *          (unweighted) are ADDED to it.
 * Sparse grids (n_bricks > 0): s_hat and d_sdf_hat are [n_bricks][16][16][16]
 * as for psdf_sdf_smooth; s is that of the full grid in which every node of
 * an absent brick holds empty_sdf (the table is read from packed_values), and
 * the sums run over the stored nodes: the terms a stored node owns (its
 * L_sdf and L_Eik, and its L_normal pairs with the next node along each axis,
 * whose normal may come from absent nodes' empty_sdf), with gradients added
 * at the stored nodes only (an absent node's s is not a parameter).  The
 * grid's faces are the full grid's. */
psdf_status psdf_grid_regularizers(const psdf_grid_desc* desc, const float* sdf_hat,
                                   const void* packed_values, float lam_sdf, float lam_eik,
                                   float lam_normal, float lam_features, void* grad_grid,
                                   float* d_sdf_hat, float* loss, void* stream);

/* L_probes = sum_i sum_{k in V_i} ||b_i - b_k||^2 over the 6-neighbourhoods V_i
 * of the probe grid (every ordered pair, Eq. 15); lam_probes * its gradient
 * is ADDED to grad (device FP32, the coefficients' layout) and L_probes to
 * loss[0] (device FP32 [1] or NULL).  FP32 coefficients with l*l*n_a a
 * multiple of 4. */
psdf_status psdf_probe_smoothness(const psdf_probe_desc* desc, const float* coeffs, float lam,
                                  float* grad, float* loss, void* stream);

/* ---------------------------------------------------------------------------
 * Learned sample proposal.  The paper has no counterpart: it marches its
 * sparse grid.  A per-ray MLP [(o - box centre) / box extent, d, first
 * occupied position, occupied fraction of each of B equal bins of
 * [t_n, t_f], B step inputs] -> W -> W -> B (ReLU hidden layers, softmax) predicts how the
 * render's weight is spread over the bins; the density p' = (1 - mix) p +
 * mix r, where r puts 1/4 evenly on all bins and 3/4 evenly on the bins that
 * hold an occupied point or neighbour one that does (r = 1/B when no bin
 * does), and p' = 1/B when max p' < theta, is inverted at the quantiles k / n_out, k = 0..n_out, to
 * give t_samples for psdf_render_forward.  The occupancy inputs look up the B n_sub points
 * t = t_n + (k + 1/2) (t_f - t_n) / (B n_sub), k = 0..B n_sub - 1, in the coarse
 * occupancy grid (the cell containing each point): bin b's input is the set
 * share of its n_sub points, the first-position input is (k* + 1/2) / (B n_sub)
 * for the first set point k* (1 when none is), and B step inputs
 * clamp(B first - b, 0, 1) give the share of each bin before that point.
 * Compiled shapes: B = 8 or 16, W = 32.  Parameters are FP32, packed
 * W1[W][7+2B] b1 W2[W][W] b2 W3[B][W] b3[B].
 * ------------------------------------------------------------------------- */

typedef struct psdf_proposal_desc {
    int32_t occ_res[3];  /* occupancy cells along x, y, z over the grid's box; each in [2, 64] */
    int32_t n_bins;      /* B; 8 and 16 are compiled in */
    int32_t width;       /* W; 32 is compiled in */
    int32_t n_sub;       /* occupancy look-ups per bin, in [1, 32] */
    float mix;           /* in [0, 1) */
    float theta;         /* uniform fallback threshold on max p' */
} psdf_proposal_desc;

psdf_status psdf_proposal_param_count(const psdf_proposal_desc* desc, int64_t* count);

/* 32-bit words of an occupancy bitmask with occ_res cells (each in [2, 64]). */
psdf_status psdf_occupancy_words(const int32_t occ_res[3], int64_t* words);

/* Coarse occupancy of the grid's SDF: cell c of occ_res cells along an axis
 * covers the nodes floor(c (R-1)/res) .. ceil((c+1)(R-1)/res); it is set where
 * the smallest |sdf| over them is below `threshold` (world units); in a
 * sparse grid the nodes of bricks that are not stored count with empty_sdf.
 *   occ_bits : device [psdf_occupancy_words] words; cell
 *              i = (z res_y + y) res_x + x is bit (i & 31) of word i >> 5
 *              (bits past the last cell are 0). */
psdf_status psdf_occupancy_build(const psdf_grid* grid, const int32_t occ_res[3],
                                 float threshold, uint32_t* occ_bits, void* stream);

/* Per-bin sums of the weights w_k of a uniform march with params->n_samples
 * samples (SDF only, Eqs. 8-10): hist [n_rays][n_bins] (device FP32);
 * n_samples must be a multiple of n_bins, n_bins <= 32. */
psdf_status psdf_weight_histogram(const psdf_grid* grid, const psdf_render_params* params,
                                  const float* rays_o, const float* rays_d, int64_t n_rays,
                                  int32_t n_bins, float* hist, void* stream);

/* Proposal forward and sample placement:
 *   params    : device FP32 [psdf_proposal_param_count]
 *   occ_bits  : device occupancy bitmask of psdf_occupancy_build for desc->occ_res
 *   t_samples : device FP32 [n_rays][n_out + 1] (rays missing the box get
 *               zeros), or NULL: the densities alone (render them with
 *               psdf_render_params.n_bins = B)
 *   probs     : device FP32 [n_rays][B] mixed density p', or NULL (not both) */
psdf_status psdf_proposal_forward(const psdf_grid* grid, const psdf_proposal_desc* desc,
                                  const float* params, const uint32_t* occ_bits,
                                  const float* rays_o,
                                  const float* rays_d, int64_t n_rays, int32_t n_out,
                                  float* t_samples, float* probs, void* stream);

/* Training signal: for rays whose weight mass sum(hist) >= min_mass, the
 * mass-weighted cross-entropy loss = -sum_b hist_b log p_b against the
 * proposal's softmax p (d loss / d logit_b = mass p_b - hist_b); the gradient
 * of scale * sum_rays loss is ACCUMULATED into grad_params (device FP32);
 * loss (device FP32 [n_rays], 0 for skipped rays) may be NULL. */
psdf_status psdf_proposal_backward(const psdf_grid* grid, const psdf_proposal_desc* desc,
                                   const float* params, const uint32_t* occ_bits,
                                   const float* rays_o,
                                   const float* rays_d, int64_t n_rays, const float* hist,
                                   float min_mass, float scale, float* grad_params, float* loss,
                                   void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PROBESDF_H */
