// Internal (C++) interface between the C ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>

#include "render_common.cuh"

namespace psdf {

constexpr int kFwdThreads = 128;
constexpr int kBwdThreads = 128;

// Compile-time shape of a render kernel: angular channels, SH coefficients,
// MLP width, Fresnel powers (3 spatial features are fixed by the record).
struct KernelShape {
    int na, l2, width, k;
};

// Shapes compiled into the library.
#define PSDF_FOR_EACH_SHAPE(X) \
    X(4, 9, 16, 3)             \
    X(4, 9, 32, 3)             \
    X(8, 9, 32, 3)

cudaError_t launch_forward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                           cudaStream_t stream);
cudaError_t launch_backward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                            cudaStream_t stream);
// Resident CTAs per SM of a kernel from its registers and shared memory, the
// device's per-SM limits and the tensor-memory columns each CTA allocates.
int resident_ctas(const cudaFuncAttributes& fa, int threads, size_t dyn_smem, unsigned tmem_cols);

// Resident CTAs per SM (occupancy, capped by tensor-memory columns).
cudaError_t forward_ctas_per_sm(const KernelShape& ks, int* n);
cudaError_t backward_ctas_per_sm(const KernelShape& ks, int* n);

cudaError_t launch_pack(const float* sdf, const float* feat, float4* packed, int64_t n_nodes,
                        cudaStream_t stream);
cudaError_t launch_unpack(const float4* packed, float* sdf, float* feat, int64_t n_nodes,
                          cudaStream_t stream);

}  // namespace psdf
