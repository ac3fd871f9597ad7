// Internal (C++) interface between the C ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>

#include "render_common.cuh"

namespace psdf {

constexpr int kFwdThreads = 128;
constexpr int kBwdThreads = 128;

// Compile-time shape of a render kernel: angular channels, SH coefficients,
// MLP width, Fresnel powers (3 spatial features), and storage: feature
// storage fb (0 FP32 node records, 1 BF16 node features, 2 tile tri-planes,
// 3 sparse bricks of FP32 node records),
// FP16 probes (ph), plain-FP16 MLP (mh).
struct KernelShape {
    int na, l2, width, k, fb, ph, mh;
    bool match(int na_, int l2_, int w_, int k_, int fb_, int ph_, int mh_) const
    {
        return na == na_ && l2 == l2_ && width == w_ && k == k_ && fb == fb_ && ph == ph_ &&
               mh == mh_;
    }
};

// Shapes compiled into the library: the FP32 path (widths 16/32, 4 or 8
// angular channels), the reduced-precision path (BF16 features, FP16 probes,
// FP16 MLP), BF16 features with FP32 probes and MLP, tile tri-plane
// features (widths 16/32), l = 4 SH (16 coefficients, Sec. 4) with node
// or tri-plane features, and sparse 16^3-node bricks (l = 3 and 4).
#define PSDF_FOR_EACH_SHAPE(X) \
    X(4, 9, 16, 3, 0, 0, 0)    \
    X(4, 9, 32, 3, 0, 0, 0)    \
    X(8, 9, 32, 3, 0, 0, 0)    \
    X(4, 9, 32, 3, 1, 1, 1)    \
    X(8, 9, 32, 3, 1, 0, 0)    \
    X(4, 9, 16, 3, 2, 0, 0)    \
    X(4, 9, 32, 3, 2, 0, 0)    \
    X(4, 16, 32, 3, 0, 0, 0)   \
    X(4, 16, 32, 3, 2, 0, 0)   \
    X(4, 9, 32, 3, 3, 0, 0)    \
    X(4, 16, 32, 3, 3, 0, 0)

cudaError_t launch_forward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                           cudaStream_t stream);
cudaError_t launch_backward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                            cudaStream_t stream);
// Resident CTAs per SM of a kernel from its registers and shared memory, the
// device's per-SM limits and the tensor-memory columns each CTA allocates.
int resident_ctas(const cudaFuncAttributes& fa, int threads, size_t dyn_smem, unsigned tmem_cols);
// Sets the kernel's shared-memory carveout hint to the smallest split of the
// SM's unified L1 / shared memory that holds its resident CTAs (resident_ctas),
// so that the rest of the SM's on-chip memory serves its gathers as L1.
cudaError_t set_smem_carveout(const void* func, int threads, size_t dyn_smem, unsigned tmem_cols);

// Resident CTAs per SM (occupancy, capped by tensor-memory columns).
cudaError_t forward_ctas_per_sm(const KernelShape& ks, int* n);
cudaError_t backward_ctas_per_sm(const KernelShape& ks, int* n);

// Two-pass inference (twopass.cu): per-view node shading, colour-field march.
struct ShadeArgs {
    float cam[3];   // camera centre (world)
    float band;     // nodes with |s| < band are shaded, the others get colour 0
    float h[3];     // node spacing (bmax - bmin) / (R - 1), FP32
    uint2* colours; // [R^3] FP16 {r, g, b, 0}
};
cudaError_t launch_shade(const RenderArgs& A, const KernelShape& ks, const ShadeArgs& S,
                         cudaStream_t stream);
cudaError_t launch_colour_render(const RenderArgs& A, const void* colours, cudaStream_t stream);

cudaError_t launch_adam(float* p, float* g, float* m, float* v, int64_t n, float lr, float beta1,
                        float beta2, float eps, int step, int clear_grad, cudaStream_t stream);
// Grid-level training terms (regularize.cu).  SDF arrays are read and written
// with an element stride (4 in FP32 node records, 1 in a plain FP32 array).
cudaError_t launch_smooth(const int R[3], const float* in, int in_stride, float* out,
                          int out_stride, bool transpose, bool accumulate, cudaStream_t stream);
// s = G(s_hat) or G^T on sparse 16^3-node bricks (R a multiple of 16): the
// stored nodes of the full grid whose absent bricks hold `empty` (forward) or
// carry no input (transpose); node `local` of slot b at
// buf[base + (b * 4096 + local) * stride].
cudaError_t launch_smooth_sparse(const int R[3], const int* table, int n_bricks, const float* in,
                                 int64_t in_base, int in_stride, float* out, int64_t out_base,
                                 int out_stride, float empty, bool transpose, bool accumulate,
                                 cudaStream_t stream);
// Dense grids (table null), or sparse 16^3-node bricks behind `table` (R
// multiples of 16; s_hat, s, d_s, d_s_hat then hold the stored bricks' nodes,
// slot-major; absent nodes read `empty`).
cudaError_t launch_sdf_reg(const int R[3], const float h[3], const float* s_hat, const float* s,
                           int s_stride, float lam_sdf, float lam_eik, float lam_normal,
                           float* d_s, int d_stride, float* d_s_hat, float* loss,
                           cudaStream_t stream, const int* table = nullptr, int n_bricks = 0,
                           float empty = 0.0f);
cudaError_t launch_plane_reg(const float4* planes, int64_t n_texels, float lam, float4* grad,
                             float* loss, cudaStream_t stream);
cudaError_t launch_probe_reg(const float4* b, const int P[3], int n4, float lam, float4* grad,
                             float* loss, cudaStream_t stream);
cudaError_t launch_brick_copy(const int dims[3], int n_bricks, const int* table, float4* bricks,
                              float* sdf, float* feat, float fill, bool pack,
                              cudaStream_t stream);
cudaError_t launch_tri_copy(const float* sdf, const float* planes, void* packed, size_t plane_off,
                            int64_t n_nodes, int64_t n_texels, bool pack, cudaStream_t stream);
cudaError_t launch_pack(const float* sdf, const float* feat, float4* packed, int64_t n_nodes,
                        cudaStream_t stream);
cudaError_t launch_unpack(const float4* packed, float* sdf, float* feat, int64_t n_nodes,
                          cudaStream_t stream);
// BF16-feature layout: FP32 SDF array, then {f0, f1, f2, 0} BF16 records at feat_off bytes.
cudaError_t launch_pack_bf16(const float* sdf, const float* feat, void* packed, size_t feat_off,
                             int64_t n_nodes, cudaStream_t stream);
cudaError_t launch_unpack_bf16(const void* packed, size_t feat_off, float* sdf, float* feat,
                               int64_t n_nodes, cudaStream_t stream);

}  // namespace psdf
