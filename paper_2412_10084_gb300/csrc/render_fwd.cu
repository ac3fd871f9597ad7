// Forward ProbeSDF render (Sec. 3, Eqs. 4-10; Sec. 4), sm_103a.
//
// Persistent CTAs of 4 warps.  Each warp takes rays in a grid-stride loop
// (misses are written out at once) and walks its ray in chunks of 32 samples,
// lane = sample.  The 4 warps advance chunk by chunk in lockstep so that their
// 128 samples form one M = 128 tile for the tensor-core MLP:
//   P0  trilinear gather of 8 packed 16-byte node records per sample and the
//       sample's opacity; where it is nonzero, normal, SH of the lookup
//       direction, probe blend, Fresnel powers -> MLP input row (split FP16)
//       in shared memory (a sample with alpha = 0 has weight 0, so its
//       appearance is never evaluated);
//   P1  layer 1 on the tensor cores; meanwhile the warp scan of the clipped
//       log-opacities gives every sample's transmittance (Eq. 8);
//   P2  ReLU epilogue -> layer 2 on the tensor cores -> layer 3 and sigmoid on
//       the CUDA cores; the chunk's weights, colours and depths are summed.
// The log-transmittance carry between chunks uses compensated summation.
#include "internal.h"
#include "mlp_tc.cuh"

namespace psdf {

template <class C>
struct FwdLayout {
    using M = MlpTC<C>;
    static constexpr int K1 = M::K1;
    static constexpr int kXT = 128 * K1 * 2;   // one split of the input tile [128][16]
    static constexpr int kHT = 128 * C::W * 2; // one split of the hidden tile [128][W]
    static constexpr int oW = 0;
    static constexpr int oF32 = oW + M::kWeightBytes;
    static constexpr int oX = (oF32 + 4 * M::kF32 + 127) & ~127;
    // the hidden tile reuses the input tile's bytes: layer 1 has read the
    // input (its MMA completed) before the hidden rows are written, and layer
    // 2 has completed before the next chunk writes its input rows
    static constexpr int oH = oX;
    static_assert(kHT >= kXT, "the hidden tile covers the input tile");
    static constexpr int oTab = oH + M::kSplit * kHT;  // per warp: 64-float placement table
    static constexpr int oBar = oTab + 4 * 64 * 4;
    static constexpr int kBytes = oBar + 16;
    static constexpr uint32_t kTmemCols = 64;  // layer 1 at column 0, layer 2 at 32
};

template <class C>
__global__ void __launch_bounds__(kFwdThreads, 4)
render_forward_kernel(RenderArgs A)
{
    using M = MlpTC<C>;
    using L = FwdLayout<C>;
    constexpr int W = C::W;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* wt = smem + L::oW;
    float* f32 = reinterpret_cast<float*>(smem + L::oF32);
    uint8_t* xh = smem + L::oX;
    uint8_t* xl = xh + L::kXT;
    uint8_t* hh = smem + L::oH;
    uint8_t* hl = hh + L::kHT;
    float* stab = reinterpret_cast<float*>(smem + L::oTab);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::oBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::oBar + 8);
    int* sbad = reinterpret_cast<int*>(smem + L::oBar + 12);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    load_mlp_tc<C>(A.mlp, wt, f32);
    if (warp == 0) tc::tmem_alloc(tslot, L::kTmemCols);
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        *sbad = 0;
    }
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * warp) << 16);
    uint32_t phase = 0;
    bool bad = false;

    const unsigned FULL = 0xffffffffu;
    const int N = A.n_samples;
    const int64_t stride = int64_t(gridDim.x) * 4;
    int64_t ray = int64_t(blockIdx.x) * 4 + warp;

    for (;;) {
        // this warp's next ray that hits the box; misses are finished here
        RayIn R;
        RaySpan sp;
        bool have = false;
        while (ray < A.n_rays) {
            R = load_ray(A, ray);
            sp = ray_span(A, R, ray, stab + 64 * warp);
            if (sp.hit) {
                have = true;
                break;
            }
            if (lane == 0) {
                A.rgb[3 * ray + 0] = A.bg[0];
                A.rgb[3 * ray + 1] = A.bg[1];
                A.rgb[3 * ray + 2] = A.bg[2];
                A.depth[ray] = 0.0f;
                A.wsum[ray] = 0.0f;
                A.logT[ray] = 0.0f;
                if (A.n_live) A.n_live[ray] = 0;
            }
            ray += stride;
        }
        if (!__syncthreads_or(have)) break;

        float acc_r = 0.f, acc_g = 0.f, acc_b = 0.f, acc_d = 0.f, acc_w = 0.f;
        float carry = 0.f, comp = 0.f;  // Kahan sum of log T over chunks
        int n_live = 0;                 // 1 + last sample with lam < 0
        // Lane l of a chunk gathers point k + 1 (the opacity of sample k needs
        // both ends of its interval) and takes sample k's SDF value, gradient
        // and spatial features from lane l - 1; lane 0 takes them from the
        // previous chunk's lane 31, and in a ray's first chunk from point 0,
        // gathered here.  So no lane gathers a second point after its own.
        float c_s = 0.f, c_g[3] = {0.f, 0.f, 0.f}, c_f[3] = {0.f, 0.f, 0.f};
        if (have) {
            SampleGeom<C> P;
            eval_sdf<C>(A, R.o, R.d, span_t(sp, 0), P);
            c_s = P.s;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                c_g[a] = P.g[a];
                c_f[a] = P.x[a];
            }
        }
        for (int base = 0; base < N; base += 32) {
            const int k = base + lane;
            const bool active = have && k < N;
            float t = 0.0f, lam = 0.0f;
            // ---- P0: geometry, angular and spatial features -> input row ----
            if (have) {
                t = span_t(sp, k < N ? k : N - 1);
                SampleGeom<C> P;  // point k + 1 (lanes past the ray's end: point N)
                eval_sdf<C>(A, R.o, R.d, span_t(sp, k < N ? k + 1 : N), P);
                SampleGeom<C> S;  // sample k
                S.s = __shfl_up_sync(FULL, P.s, 1);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    S.g[a] = __shfl_up_sync(FULL, P.g[a], 1);
                    S.x[a] = __shfl_up_sync(FULL, P.x[a], 1);
                }
                if (lane == 0) {
                    S.s = c_s;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        S.g[a] = c_g[a];
                        S.x[a] = c_f[a];
                    }
                }
                c_s = __shfl_sync(FULL, P.s, 31);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    c_g[a] = __shfl_sync(FULL, P.g[a], 31);
                    c_f[a] = __shfl_sync(FULL, P.x[a], 31);
                }
                const float s_next = P.s;
                bool opaque = false;
                if (active) {
                    const float diff = log_transmittance(A.tau, S.s, s_next);
                    opaque = diff < 0.0f;
                    lam = opaque ? diff : 0.0f;
                }
                // a clipped opacity (alpha = 0) gives the sample weight 0: its
                // colour, and so its appearance inputs, never reach an output
                if (opaque)
                    eval_appearance<C>(A, R.o, R.d, t, S);
                else
                    zero_appearance<C>(S);
                float xin[M::K1];
#pragma unroll
                for (int i = 0; i < M::K1; ++i) xin[i] = i < C::NIN ? S.x[i] : 0.0f;
                store_row<M::K1, M::kSplit>(xh, xl, tid, 0, M::K1, xin);
            } else {
                zero_row<M::K1, M::kSplit>(xh, xl, tid, 0, M::K1);
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            // One barrier both publishes the input rows and tells whether any
            // sample of the CTA's 128 has a nonzero opacity; a failed wait
            // (rare) is passed on through shared memory
            if (bad) *sbad = 1;
            const bool run_mlp = __syncthreads_or(lam < 0.0f);
            if (*sbad) goto done;
            tc::fence_after();
            // ---- P1: layer 1 on the tensor cores ----
            // Without an opaque sample every weight of the chunk is zero and
            // no colour reaches an output: the MLP is skipped (the outputs are
            // the same bits), only the transmittance carry below is updated.
            if (run_mlp && tid == 0) {
                mma_k<M::kSplit>(tmem + 0, xh, xl, M::w1h(wt), M::w1l(wt), 128,
                                 (M::K1 / 8) * 128, 128, (M::K1 / 8) * 128, M::kIdescL, false);
                tc::commit(mbar);
            }
            {
                const uint32_t opaque = __ballot_sync(FULL, lam < 0.0f);
                if (opaque) n_live = base + 32 - __clz(opaque);
            }
            // transmittance of the chunk (Eq. 8): exclusive warp scan of lam
            float incl = lam;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float v = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += v;
            }
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0.0f;
            const float total = __shfl_sync(FULL, incl, 31);
            const float wgt = active ? expf((carry - comp) + excl) * -expm1f(lam) : 0.0f;
            {
                const float y = total - comp;
                const float tt = carry + y;
                comp = (tt - carry) - y;
                carry = tt;
            }
            if (!run_mlp) continue;
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            {
                float z[W];
                tc::tmem_ld<W>(t_row + 0, z);
#pragma unroll
                for (int o = 0; o < W; ++o) z[o] = fmaxf(z[o] + f32[M::kB1 + o], 0.0f);
                store_row<W, M::kSplit>(hh, hl, tid, 0, W, z);
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            // ---- P2: layer 2 on the tensor cores, layer 3 on the CUDA cores ----
            if (tid == 0) {
#pragma unroll
                for (int s = 0; s < W / 16; ++s)
                    mma_k<M::kSplit>(tmem + 32, hh + s * 256, hl + s * 256,
                                     M::w2h(wt) + s * 256, M::w2l(wt) + s * 256, 128,
                                     (W / 8) * 128, 128, (W / 8) * 128, M::kIdescL, s > 0);
                tc::commit(mbar);
            }
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            {
                float z[W];
                tc::tmem_ld<W>(t_row + 32, z);
#pragma unroll
                for (int o = 0; o < W; ++o) z[o] = fmaxf(z[o] + f32[M::kB2 + o], 0.0f);
                float col[3];
                mlp_layer3<C>(f32, z, col);
                if (active) {
                    acc_r = fmaf(wgt, col[0], acc_r);
                    acc_g = fmaf(wgt, col[1], acc_g);
                    acc_b = fmaf(wgt, col[2], acc_b);
                    acc_d = fmaf(wgt, t, acc_d);
                    acc_w += wgt;
                }
            }
            tc::fence_before();
        }
        if (have) {
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
                if (A.n_live) A.n_live[ray] = n_live;
            }
            ray += stride;
        }
    }
done:
    bad = __syncthreads_or(bad);
    if (bad) {
        // an MMA never signalled completion: give it one more bounded wait
        // before the tensor memory is released, and report the failure
        // the last commit's phase has the parity before the final flip
        tc::mbar_wait(mbar, phase ^ 1u);
        if (tid == 0) atomicOr(A.status, 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, L::kTmemCols);
}

template <class C>
cudaError_t launch_forward_t(const RenderArgs& A, int grid_ctas, cudaStream_t stream)
{
    using L = FwdLayout<C>;
    cudaError_t e = cudaFuncSetAttribute(render_forward_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    render_forward_kernel<C><<<grid_ctas, kFwdThreads, L::kBytes, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_forward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                           cudaStream_t stream)
{
#define PSDF_FWD_CASE(NA, L2, W, K, FB, PH, MH)                                              \
    if (ks.match(NA, L2, W, K, FB, PH, MH))                                                  \
        return launch_forward_t<Cfg<NA, L2, W, K, FB, PH, MH>>(A, grid_ctas, stream);
    PSDF_FOR_EACH_SHAPE(PSDF_FWD_CASE)
#undef PSDF_FWD_CASE
    return cudaErrorInvalidValue;
}

template <class C>
cudaError_t forward_occupancy_t(int* n)
{
    using L = FwdLayout<C>;
    cudaError_t e = cudaFuncSetAttribute(render_forward_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, render_forward_kernel<C>);
    if (e != cudaSuccess) return e;
    *n = resident_ctas(fa, kFwdThreads, L::kBytes, L::kTmemCols);
    return *n > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t forward_ctas_per_sm(const KernelShape& ks, int* n)
{
    *n = 0;
#define PSDF_FWD_OCC(NA, L2, W, K, FB, PH, MH)                                                \
    if (ks.match(NA, L2, W, K, FB, PH, MH))                                                  \
        return forward_occupancy_t<Cfg<NA, L2, W, K, FB, PH, MH>>(n);
    PSDF_FOR_EACH_SHAPE(PSDF_FWD_OCC)
#undef PSDF_FWD_OCC
    return cudaErrorInvalidValue;
}

}  // namespace psdf
