// Forward ProbeSDF render (Sec. 3, Eqs. 4-10; Sec. 4), FP32, sm_103a.
//
// Persistent grid; each warp takes rays in a grid-stride loop and walks a ray
// in chunks of 32 samples (lane = sample).  Per chunk: one trilinear gather
// of 8 packed 16-byte node records per sample, the probe blend, the MLP
// (weights broadcast from shared memory), then a warp scan of the clipped
// log-opacities gives the transmittance of every sample of the chunk; the
// chunk total is carried to the next chunk with compensated summation.
#include "internal.h"
#include "sample_eval.cuh"

namespace psdf {

template <class C>
__global__ void __launch_bounds__(kFwdThreads)
render_forward_kernel(RenderArgs A)
{
    __shared__ __align__(16) float sw[C::kMlpSmem];
    load_mlp_smem<C>(A.mlp, sw);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int N = A.n_samples;
    const unsigned FULL = 0xffffffffu;

    for (int64_t ray = warp0; ray < A.n_rays; ray += nwarps) {
        const RayIn R = load_ray(A, ray);
        const RaySpan sp = ray_span(A, R, ray);
        if (!sp.hit) {
            if (lane == 0) {
                A.rgb[3 * ray + 0] = A.bg[0];
                A.rgb[3 * ray + 1] = A.bg[1];
                A.rgb[3 * ray + 2] = A.bg[2];
                A.depth[ray] = 0.0f;
                A.wsum[ray] = 0.0f;
                A.logT[ray] = 0.0f;
            }
            continue;
        }
        float acc_r = 0.f, acc_g = 0.f, acc_b = 0.f, acc_d = 0.f, acc_w = 0.f;
        float carry = 0.f, comp = 0.f;  // Kahan sum of log T over chunks

        for (int base = 0; base < N; base += 32) {
            const int k = base + lane;
            const bool active = k < N;
            const int kc = active ? k : N - 1;  // colour sample evaluated by this lane
            const float t = span_t(sp, kc);

            SampleGeom<C> S;
            eval_geometry<C>(A, R.o, R.d, t, S);
            float col[3];
            mlp_forward<C, false>(sw, S.x, col, nullptr, nullptr, nullptr);

            // s at point k+1: the next lane's point, or an extra gather for the
            // chunk's last lane.
            float s_next = __shfl_down_sync(FULL, S.s, 1);
            if (lane == 31 || k + 1 >= N) {
                if (active) {
                    float xw[3];
                    point_at(R.o, R.d, span_t(sp, k + 1), xw);
                    const Cell c1 = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
                    s_next = sdf_value(A.grid, c1);
                }
            }
            // Eq. 9 in log space: log(1 - alpha_k) = min(log Phi(s_k+1) - log Phi(s_k), 0)
            float lam = 0.0f;
            if (active) {
                const float diff = log_transmittance(A.tau, S.s, s_next);
                lam = diff < 0.0f ? diff : 0.0f;
            }
            // exclusive warp scan of lam -> log T_k within the chunk (Eq. 8)
            float incl = lam;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float v = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += v;
            }
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0.0f;
            const float total = __shfl_sync(FULL, incl, 31);
            if (active) {
                const float T = expf((carry - comp) + excl);
                const float w = T * -expm1f(lam);
                acc_r = fmaf(w, col[0], acc_r);
                acc_g = fmaf(w, col[1], acc_g);
                acc_b = fmaf(w, col[2], acc_b);
                acc_d = fmaf(w, t, acc_d);
                acc_w += w;
            }
            const float y = total - comp;
            const float tt = carry + y;
            comp = (tt - carry) - y;
            carry = tt;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc_r += __shfl_xor_sync(FULL, acc_r, off);
            acc_g += __shfl_xor_sync(FULL, acc_g, off);
            acc_b += __shfl_xor_sync(FULL, acc_b, off);
            acc_d += __shfl_xor_sync(FULL, acc_d, off);
            acc_w += __shfl_xor_sync(FULL, acc_w, off);
        }
        if (lane == 0) {
            const float logT = carry - comp;
            const float TN = expf(logT);
            A.rgb[3 * ray + 0] = fmaf(TN, A.bg[0], acc_r);
            A.rgb[3 * ray + 1] = fmaf(TN, A.bg[1], acc_g);
            A.rgb[3 * ray + 2] = fmaf(TN, A.bg[2], acc_b);
            A.depth[ray] = acc_d;
            A.wsum[ray] = acc_w;
            A.logT[ray] = logT;
        }
    }
}

template <class C>
cudaError_t launch_forward_t(const RenderArgs& A, int grid_ctas, cudaStream_t stream)
{
    render_forward_kernel<C><<<grid_ctas, kFwdThreads, 0, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_forward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                           cudaStream_t stream)
{
#define PSDF_FWD_CASE(NA, L2, W, K)                                                          \
    if (ks.na == NA && ks.l2 == L2 && ks.width == W && ks.k == K)                            \
        return launch_forward_t<Cfg<NA, L2, W, K>>(A, grid_ctas, stream);
    PSDF_FOR_EACH_SHAPE(PSDF_FWD_CASE)
#undef PSDF_FWD_CASE
    return cudaErrorInvalidValue;
}

int forward_ctas_per_sm(const KernelShape& ks)
{
    int n = 0;
#define PSDF_FWD_OCC(NA, L2, W, K)                                                           \
    if (ks.na == NA && ks.l2 == L2 && ks.width == W && ks.k == K)                            \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                       \
            &n, render_forward_kernel<Cfg<NA, L2, W, K>>, kFwdThreads, 0);
    PSDF_FOR_EACH_SHAPE(PSDF_FWD_OCC)
#undef PSDF_FWD_OCC
    return n;
}

}  // namespace psdf
