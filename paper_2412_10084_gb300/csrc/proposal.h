// Internal interface of the learned sample proposal kernels.
#pragma once

#include <cuda_runtime.h>

#include "render_common.cuh"

namespace psdf {

struct ProposalLaunch {
    GridView grid;
    int occ_res[3];
    const float* occ;
    const float* params;
    float mix, theta;
    const float* rays_o;
    const float* rays_d;
    int64_t n_rays;
    int n_out;
    float* t_samples;
    float* probs;
    const float* hist;
    float min_mass, scale;
    float* grad;
    float* loss;
};

int proposal_param_count();
int proposal_bins();
int proposal_width();
cudaError_t launch_occupancy(const GridView& g, const int res[3], float threshold, float* occ,
                             cudaStream_t stream);
cudaError_t launch_histogram(const RenderArgs& A, int n_bins, float* hist, cudaStream_t stream);
cudaError_t launch_proposal_forward(const ProposalLaunch& L, cudaStream_t stream);
cudaError_t launch_proposal_backward(const ProposalLaunch& L, cudaStream_t stream);

}  // namespace psdf
