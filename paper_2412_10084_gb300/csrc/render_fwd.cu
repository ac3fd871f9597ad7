// Forward ProbeSDF render (Sec. 3, Eqs. 4-10; Sec. 4), sm_103a.
//
// Persistent CTAs of 4 warps.  Each warp takes rays in a grid-stride loop
// (misses are written out at once) and walks its ray in chunks of 32 samples,
// lane = sample.  The warps run independently (no CTA barrier in the loop):
//   P0  trilinear gather of 8 packed 16-byte node records per sample and the
//       sample's opacity; where it is nonzero, normal, SH of the lookup
//       direction, probe blend, Fresnel powers -> the warp's 32 rows of the
//       MLP input tile (split FP16) in shared memory (a sample with alpha = 0
//       has weight 0, so its appearance is never evaluated);
//   P1  layer 1 on the tensor cores, issued by the warp itself over the whole
//       M = 128 tile into its own 32 tensor-memory columns (it reads back only
//       its own 32 lanes, i.e. its own rows; the other rows of its result are
//       never read); meanwhile the warp scan of the clipped log-opacities
//       gives every sample's transmittance (Eq. 8);
//   P2  ReLU epilogue -> layer 2 into the same columns -> layer 3 and sigmoid
//       on the CUDA cores; the chunk's weights, colours and depths are summed.
// A chunk without an opaque sample skips P1-P2 (its weights are all zero).
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
    // the warps' MLP steps are not in step with each other, so a warp's hidden
    // rows must not cover another warp's input rows: the tiles lie apart
    static constexpr int oH = oX + M::kSplit * kXT;
    static constexpr int oTab = oH + M::kSplit * kHT;  // per warp: 64-float placement table
    static constexpr int oBar = oTab + 4 * 64 * 4;       // one mbarrier per warp
    static constexpr int kBytes = oBar + 4 * 8 + 16;
    // 32 columns per warp: layer 1's accumulator, then layer 2's over it
    static constexpr uint32_t kTmemCols = 128;
    static_assert(C::W <= 32, "a warp's accumulator fits its 32 columns");
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
    uint64_t* mbars = reinterpret_cast<uint64_t*>(smem + L::oBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::oBar + 32);
    int* ray_counter = reinterpret_cast<int*>(smem + L::oBar + 36);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    load_mlp_tc<C>(A.mlp, wt, f32);
    if (warp == 0) tc::tmem_alloc(tslot, L::kTmemCols);
    if (tid < 4) tc::mbar_init(mbars + tid, 1);
    if (tid == 0) *ray_counter = 0;
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    uint64_t* mbar = mbars + warp;
    // the warp's accumulator columns (all 128 lanes written by its MMAs) and
    // its own 32 lanes of them
    const uint32_t t_acc = tmem + 32u * static_cast<uint32_t>(warp);
    const uint32_t t_row = t_acc + (static_cast<uint32_t>(32 * warp) << 16);
    uint32_t phase = 0;
    bool bad = false;

    const unsigned FULL = 0xffffffffu;
    const int N = A.n_samples;
    const int64_t stride = int64_t(gridDim.x) * 4;
    int64_t ray = next_cta_ray(ray_counter, stride);

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
            ray = next_cta_ray(ray_counter, stride);
        }
        if (!have) break;  // warp-uniform: every lane holds the same ray

        float acc_r = 0.f, acc_g = 0.f, acc_b = 0.f, acc_d = 0.f, acc_w = 0.f;
        float carry = 0.f, comp = 0.f;  // Kahan sum of log T over chunks
        int n_live = 0;                 // 1 + last sample with lam < 0
        // Lane l of a chunk gathers point k + 1 (the opacity of sample k needs
        // both ends of its interval) and takes sample k's SDF value, gradient
        // and spatial features from lane l - 1; lane 0 takes them from the
        // previous chunk's lane 31, and in a ray's first chunk from point 0,
        // gathered here.  So no lane gathers a second point after its own.
        float c_s, c_g[3], c_f[3];
        {
            SampleGeom<C> P;
            if constexpr (features_apart<C>())
                eval_sdf_geom<C>(A, R.o, R.d, span_t(sp, 0), P);
            else
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
            const bool active = k < N;
            float lam = 0.0f;
            // ---- P0: geometry, angular and spatial features -> input row ----
            const float t = span_t(sp, k < N ? k : N - 1);
            {
                SampleGeom<C> P;  // point k + 1 (lanes past the ray's end: point N)
                // (the features apart from the SDF are gathered below, for the
                // samples with a nonzero opacity only)
                if constexpr (features_apart<C>())
                    eval_sdf_geom<C>(A, R.o, R.d, span_t(sp, k < N ? k + 1 : N), P);
                else
                    eval_sdf<C>(A, R.o, R.d, span_t(sp, k < N ? k + 1 : N), P);
                SampleGeom<C> S;  // sample k
                S.s = __shfl_up_sync(FULL, P.s, 1);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    S.g[a] = __shfl_up_sync(FULL, P.g[a], 1);
                    S.x[a] = features_apart<C>() ? 0.0f : __shfl_up_sync(FULL, P.x[a], 1);
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
                    c_f[a] = features_apart<C>() ? 0.0f : __shfl_sync(FULL, P.x[a], 31);
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
                if (opaque) {
                    if constexpr (features_apart<C>()) eval_features<C>(A, R.o, R.d, t, S);
                    eval_appearance<C>(A, R.o, R.d, t, S);
                } else {
                    zero_appearance<C>(S);
                }
                // the input rows are needed only if the warp runs its MLP step
                if (__any_sync(FULL, lam < 0.0f)) {
                    float xin[M::K1];
#pragma unroll
                    for (int i = 0; i < M::K1; ++i) xin[i] = i < C::NIN ? S.x[i] : 0.0f;
                    store_row<M::K1, M::kSplit>(xh, xl, tid, 0, M::K1, xin);
                }
            }
            // Without an opaque sample every weight of the chunk is zero and
            // no colour reaches an output: the MLP is skipped (the outputs are
            // the same bits), only the transmittance carry below is updated.
            const uint32_t opaque = __ballot_sync(FULL, lam < 0.0f);
            if (opaque) {
                n_live = base + 32 - __clz(opaque);
                // ---- P1: layer 1 on the tensor cores ----
                tc::fence_smem_to_async();
                tc::fence_before();
                __syncwarp();
                tc::fence_after();
                if (lane == 0) {
                    mma_k<M::kSplit>(t_acc, xh, xl, M::w1h(wt), M::w1l(wt), 128,
                                     (M::K1 / 8) * 128, 128, (M::K1 / 8) * 128, M::kIdescL,
                                     false);
                    tc::commit(mbar);
                }
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
            if (!opaque) continue;
            {
                // one decision per warp: every lane leaves, or none
                const bool ok = __all_sync(FULL, tc::mbar_wait(mbar, phase, A.wait_polls));
                phase ^= 1;
                if (!ok) {
                    bad = true;
                    goto done;
                }
            }
            tc::fence_after();
            {
                float z[W];
                tc::tmem_ld<W>(t_row, z);
                bias_relu<W>(z, f32 + M::kB1);
                store_row<W, M::kSplit>(hh, hl, tid, 0, W, z);
            }
            // the layer-1 reads are complete (tcgen05.wait::ld) before the
            // layer-2 MMA overwrites the columns
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncwarp();
            tc::fence_after();
            // ---- P2: layer 2 on the tensor cores, layer 3 on the CUDA cores ----
            if (lane == 0) {
#pragma unroll
                for (int s = 0; s < W / 16; ++s)
                    mma_k<M::kSplit>(t_acc, hh + s * 256, hl + s * 256,
                                     M::w2h(wt) + s * 256, M::w2l(wt) + s * 256, 128,
                                     (W / 8) * 128, 128, (W / 8) * 128, M::kIdescL, s > 0);
                tc::commit(mbar);
            }
            {
                const bool ok = __all_sync(FULL, tc::mbar_wait(mbar, phase, A.wait_polls));
                phase ^= 1;
                if (!ok) {
                    bad = true;
                    goto done;
                }
            }
            tc::fence_after();
            {
                float z[W];
                tc::tmem_ld<W>(t_row, z);
                bias_relu<W>(z, f32 + M::kB2);
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
            // the layer-2 reads are complete before the next chunk's layer-1
            // MMA (issued after this warp's next __syncwarp) overwrites them
            tc::fence_before();
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
            if (A.n_live) A.n_live[ray] = n_live;
        }
        ray = next_cta_ray(ray_counter, stride);
    }
done:
    bad = __syncthreads_or(bad);
    if (bad) {
        // an MMA never signalled completion: give this warp's last commit one
        // more bounded wait before the tensor memory is released (a warp with
        // nothing pending passes at once), and report the failure
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
    if (e == cudaSuccess)
        e = set_smem_carveout(reinterpret_cast<const void*>(render_forward_kernel<C>),
                              kFwdThreads, L::kBytes, L::kTmemCols);
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
