// Internal interface of the learned sample proposal kernels.
#pragma once

#include <cuda_runtime.h>

#include "render_common.cuh"

namespace psdf {

struct ProposalLaunch {
    GridView grid;
    int occ_res[3];
    int n_bins;
    int n_sub;
    const uint32_t* occ_bits;
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

int proposal_param_count(int n_bins);  // 0 for an uncompiled bin count
bool proposal_bins_supported(int n_bins);
int proposal_width();
int occupancy_words(const int res[3]);
cudaError_t launch_occupancy(const GridView& g, const int res[3], float threshold,
                             uint32_t* bits, cudaStream_t stream);
cudaError_t launch_histogram(const RenderArgs& A, int n_bins, float* hist, cudaStream_t stream);
cudaError_t launch_proposal_forward(const ProposalLaunch& L, cudaStream_t stream);
cudaError_t launch_proposal_backward(const ProposalLaunch& L, cudaStream_t stream);

}  // namespace psdf
