// Adjoint of the ProbeSDF render (Sec. 3.3-3.4), sm_103a.
//
// Persistent CTAs of 4 warps, one ray per warp (the CTA's rays taken from a
// shared-memory counter), lane = sample.  Unlike the forward, whose warps run
// their own MLP steps, the 4 warps advance in lockstep 32-sample chunks whose
// 128 samples form one M = 128 tile: the adjoint's tensor memory (activations,
// the weight-gradient accumulator and the blended probe coefficients) has no
// room for per-warp accumulators at 3 CTAs per SM.  Chunks are walked back to
// front starting from the saved log T_N, and every per-sample activation is
// recomputed (nothing per sample is stored by the forward).  Per chunk:
//   P0  recompute geometry and features -> input row of the XH tile;
//   P1  layer 1 (tensor cores); warp suffix sum of the clipped log-opacities
//       gives log T_k;
//   P2  layer 2 (tensor cores) and layer 3; the suffix term of
//       dL/dalpha_k = T_k (G_k - S_k) from a warp scan of the affine recurrence
//       S_k = alpha_{k+1} G_{k+1} + (1 - alpha_{k+1}) S_{k+1}; sigmoid and layer-3
//       adjoints on the CUDA cores -> dz2 row of the DZ tile;
//   P3  dh1 = dz2 W2 (tensor cores, W2 read transposed) -> dz1 row;
//   P4  dx = dz1 W1 (tensor cores) and the weight gradient
//       [dz1 | dz2]^T [x, 1 | h1] as an M = 64 MMA over the transposed tiles,
//       accumulated in tensor memory for the whole kernel;
//   P5  angular, Fresnel, normal and spatial-feature adjoints; SDF + feature
//       gradients as one 16-byte vector reduction per corner; probe gradients
//       summed over runs of samples sharing a probe cell.
// MLP-path gradients in the FP16 tiles are carried scaled by per-CTA powers of
// two, from rigorous bounds (largest dL/drgb among the CTA's rays and column
// sums of |W3| and |W2|), so they never overflow and keep their precision.
#include "internal.h"
#include "mlp_tc.cuh"

namespace psdf {

// Gradient-buffer record of corner q (cx + 2 cy + 4 cz) of cell c: the node's
// linear index, or for sparse bricks its record index (-1: brick not stored).
template <class C>
__device__ __forceinline__ int64_t grad_record(const GridView& g, const Cell& c, int q)
{
    if constexpr (C::SP)
        return brick_record(g, c.i[0] + (q & 1), c.i[1] + ((q >> 1) & 1), c.i[2] + (q >> 2));
    else
        return c.base + (q & 1) + ((q >> 1) & 1) * g.R[0] + (q >> 2) * g.R[0] * g.R[1];
}

template <class C>
struct BwdLayout {
    using M = MlpTC<C>;
    static constexpr int W = C::W;
    static constexpr int K1 = M::K1;
    static constexpr int XHC = K1 + W;   // XH tile: [x (n_in), 1, 0.. | h1 (W)]
    static constexpr int DZC = 64;       // DZ tile: [dz1 (W) | dz2 (W) | unused]
    static constexpr int kXH = 128 * XHC * 2;
    static constexpr int kDZ = 128 * DZC * 2;
    static constexpr uint32_t kSboXH = (XHC / 8) * 128;
    static constexpr uint32_t kSboDZ = (DZC / 8) * 128;
    static constexpr int kDZWarp = 4 * kSboDZ;  // bytes of a warp's 32 rows of a DZ tile
    static_assert(32 * C::W * 4 <= kDZWarp, "h2 staging fits the warp's rows of the DZ tile");
    static constexpr int PST = ((8 + C::L2 + C::NA + 1) + 3) & ~3;  // probe staging row (floats)
    static constexpr int kParamsPad = (C::kParams + 3) & ~3;
    static constexpr int oW = 0;
    static constexpr int oF32 = oW + M::kWeightBytes;
    static constexpr int oXH = (oF32 + 4 * M::kF32 + 127) & ~127;
    static constexpr int oDZ = oXH + M::kSplit * kXH;
    // the CTA's MLP-gradient sums are formed after the chunk loop, in the
    // operand tiles (free by then), so they take no shared memory of their own
    static constexpr int oG = oXH;
    static_assert(4 * kParamsPad <= M::kSplit * (kXH + kDZ), "gradient sums fit the tiles");
    static constexpr int oTab = oDZ + M::kSplit * kDZ;  // per warp: 64-float placement table
    static constexpr int oMisc = oTab + 4 * 64 * 4;
    static constexpr int kBytes = oMisc + 64;
    static constexpr uint32_t kTmemCols = 128;  // z1/dh1 at 0, z2/dx at 32, dW at 64..111
    // blended probe coefficients of each sample (Bc, L2 x NA floats), kept from
    // P0 to P5 in columns 112..127 and a second 32-column allocation
    static constexpr int kBc = C::L2 * C::NA;
    static constexpr bool kKeepBc = kBc <= 48 && kBc % 4 == 0;
    static constexpr uint32_t kTmemCols2 = kKeepBc ? 32 : 0;
    static constexpr uint32_t kBcCol = 112;
    static_assert(128 * PST * 4 <= M::kSplit * kDZ, "probe staging aliases the DZ tiles");
    static_assert(XHC <= 64, "dW accumulator fits columns 64..127");
};

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Probe-coefficient gradient (Eqs. 6-7): dL/db_ijc = sum_k w_i(k) Y_j(k) dF_a,c(k).
// Samples of a chunk that share a probe cell are consecutive; lane (corner i,
// channel c) sums each run over the rows in `live` and issues one reduction
// per coefficient at the run's last sample (the bits of `ends`).  The next
// row's operands are loaded while the current row is summed.
template <class C, int PST>
__device__ __forceinline__ void scatter_probe_grad(const RenderArgs& A, const float* pst,
                                                   uint32_t live, uint32_t ends, int lane)
{
    constexpr int L2 = C::L2, NA = C::NA;
    constexpr int CPL = (8 * NA) / 32;
    static_assert((8 * NA) % 32 == 0, "8 corners x channels must fill whole warps");
    static_assert(PST % 4 == 0, "rows of whole 16-byte vectors");
    constexpr int L2V = (L2 + 3) / 4;  // Y_j starts at float 8: 16-byte aligned
    static_assert(8 + 4 * L2V <= PST, "vector reads stay inside the row");
    if (!live) return;
    const int Px = A.probes.P[0], Pxy = A.probes.P[0] * A.probes.P[1];
    int q[CPL], ch[CPL], qoff[CPL];
    float acc[CPL][L2];
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int combo = lane + 32 * m;
        q[m] = combo / NA;
        ch[m] = combo % NA;
        qoff[m] = (q[m] & 1) + ((q[m] >> 1) & 1) * Px + ((q[m] >> 2) & 1) * Pxy;
#pragma unroll
        for (int j = 0; j < L2; ++j) acc[m][j] = 0.f;
    }
    // row s: w_i at [0, 8), Y_j at 8, dF_a at 8 + L2, the probe cell at 8 + L2 + NA
    auto load = [&](int s, float4 (&y)[L2V], float (&coef)[CPL]) {
        const float* row = pst + s * PST;
#pragma unroll
        for (int v = 0; v < L2V; ++v) y[v] = *reinterpret_cast<const float4*>(row + 8 + 4 * v);
#pragma unroll
        for (int m = 0; m < CPL; ++m) coef[m] = row[q[m]] * row[8 + L2 + ch[m]];
    };
    int s = __ffs(live) - 1;
    uint32_t rem = live & (live - 1);
    float4 y[L2V];
    float coef[CPL];
    load(s, y, coef);
    for (;;) {
        const int sn = rem ? __ffs(rem) - 1 : s;
        float4 yn[L2V];
        float coefn[CPL];
        load(sn, yn, coefn);
        const float* Y = reinterpret_cast<const float*>(y);
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const float2 c2 = make_float2(coef[m], coef[m]);
#pragma unroll
            for (int j = 0; j + 1 < L2; j += 2) {
                const float2 r = fma2(c2, make_float2(Y[j], Y[j + 1]),
                                      make_float2(acc[m][j], acc[m][j + 1]));
                acc[m][j] = r.x;
                acc[m][j + 1] = r.y;
            }
            if constexpr (L2 % 2) acc[m][L2 - 1] = fmaf(coef[m], Y[L2 - 1], acc[m][L2 - 1]);
        }
        if ((ends >> s) & 1u) {
            const int cell = __float_as_int(pst[s * PST + 8 + L2 + NA]);
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                float* dst = A.grad_probes + (size_t)(cell + qoff[m]) * (L2 * NA) + ch[m];
#pragma unroll
                for (int j = 0; j < L2; ++j) {
                    red_add(dst + j * NA, acc[m][j]);
                    acc[m][j] = 0.f;
                }
            }
        }
        if (!rem) break;
        rem &= rem - 1;
        s = sn;
#pragma unroll
        for (int v = 0; v < L2V; ++v) y[v] = yn[v];
#pragma unroll
        for (int m = 0; m < CPL; ++m) coef[m] = coefn[m];
    }
}

// The blended probe coefficients of the warp's 32 samples into / out of their
// tensor-memory columns (warp-collective): the first 16 in columns 112..127 of
// the main allocation, the rest from column 0 of the second.
template <class L>
__device__ __forceinline__ void bc_store(uint32_t t_row, uint32_t t_row2, const float* Bc)
{
    tc::tmem_st16(t_row + L::kBcCol, Bc);
#pragma unroll
    for (int i = 16; i < L::kBc; i += 16) {
        if (i + 16 <= L::kBc)
            tc::tmem_st16(t_row2 + (i - 16), Bc + i);
        else
#pragma unroll
            for (int r = i; r < L::kBc; r += 4) tc::tmem_st4(t_row2 + (r - 16), Bc + r);
    }
    tc::tmem_st_wait();
}

template <class L>
__device__ __forceinline__ void bc_load(uint32_t t_row, uint32_t t_row2, float* Bc)
{
    tc::tmem_ld16(t_row + L::kBcCol, Bc);
#pragma unroll
    for (int i = 16; i < L::kBc; i += 16) {
        if (i + 16 <= L::kBc)
            tc::tmem_ld16(t_row2 + (i - 16), Bc + i);
        else
#pragma unroll
            for (int r = i; r < L::kBc; r += 4) tc::tmem_ld4(t_row2 + (r - 16), Bc + r);
    }
}

template <class C>
__global__ void __launch_bounds__(kBwdThreads, 3)
render_backward_kernel(RenderArgs A)
{
    using M = MlpTC<C>;
    using L = BwdLayout<C>;
    constexpr int W = C::W, L2 = C::L2, NA = C::NA, NIN = C::NIN, K1 = M::K1;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* wt = smem + L::oW;
    uint8_t* w1h = M::w1h(wt);
    uint8_t* w1l = M::w1l(wt);
    uint8_t* w2h = M::w2h(wt);
    uint8_t* w2l = M::w2l(wt);
    float* f32 = reinterpret_cast<float*>(smem + L::oF32);
    uint8_t* xhh = smem + L::oXH;
    uint8_t* xhl = xhh + L::kXH;
    uint8_t* dzh = smem + L::oDZ;
    uint8_t* dzl = dzh + L::kDZ;
    float* gacc = reinterpret_cast<float*>(smem + L::oG);
    float* stab = reinterpret_cast<float*>(smem + L::oTab);
    float* red = reinterpret_cast<float*>(smem + L::oMisc);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::oMisc + 32);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::oMisc + 40);
    uint32_t* tslot2 = reinterpret_cast<uint32_t*>(smem + L::oMisc + 44);
    int* ray_counter = reinterpret_cast<int*>(smem + L::oMisc + 48);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned FULL = 0xffffffffu;
    const int N = A.n_samples;
    const float tau = A.tau;
    const int64_t stride = int64_t(gridDim.x) * 4;

    load_mlp_tc<C>(A.mlp, wt, f32);
    if (warp == 0) {
        tc::tmem_alloc(tslot, L::kTmemCols, !L::kKeepBc);
        if constexpr (L::kKeepBc) tc::tmem_alloc(tslot2, L::kTmemCols2, true);
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        *ray_counter = 0;
    }
    {
        // gradient scale: the largest |dL/drgb| over the rays this CTA renders
        // (warp w reads the rays b * 4 + w + i * stride; together all of them)
        float m = 0.0f;
        for (int64_t r = int64_t(blockIdx.x) * 4 + warp + int64_t(lane) * stride; r < A.n_rays;
             r += 32 * stride)
            m = fmaxf(m, fmaxf(fabsf(__ldg(A.d_rgb + 3 * r)),
                               fmaxf(fabsf(__ldg(A.d_rgb + 3 * r + 1)),
                                     fabsf(__ldg(A.d_rgb + 3 * r + 2)))));
        m = warp_max(m);
        if (lane == 0) red[warp] = m;
    }
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * warp) << 16);
    const uint32_t t_row2 = L::kKeepBc ? *tslot2 + (static_cast<uint32_t>(32 * warp) << 16) : 0u;
    // Power-of-two scales of the dz2 and dz1 tiles.  With |w| <= 1 and
    // sigmoid' <= 1/4: |dz3| <= M/4 (M = largest |dL/drgb| of the CTA),
    // |dz2_i| <= B2 = M/4 * sum_c |W3[c][i]|, |dz1_i| <= B1 = max_i sum_o |W2[o][i]| * B2.
    // Scaling each bound to <= 2^12 keeps every value finite in FP16 while
    // values down to ~1e-5 of the bound keep both halves of the split normal.
    float s1 = 1.0f, inv_s1 = 1.0f, s2 = 1.0f, inv_s2 = 1.0f;
    {
        const float m = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
        float c3 = 0.0f, c2 = 0.0f;
        for (int i = 0; i < W; ++i)
            c3 = fmaxf(c3, fabsf(f32[M::kW3 + i]) + fabsf(f32[M::kW3 + W + i]) +
                               fabsf(f32[M::kW3 + 2 * W + i]));
        for (int i = 0; i < W; ++i) {
            float cs = 0.0f;
            for (int o = 0; o < W; ++o) cs += fabsf(__ldg(A.mlp + C::gW2 + o * W + i));
            c2 = fmaxf(c2, cs);
        }
        const float b2 = 0.25f * m * c3, b1 = b2 * c2;
        int e;
        if (b2 > 0.0f && b2 < 1e30f) {
            frexpf(b2, &e);
            s2 = ldexpf(1.0f, 12 - e);
            inv_s2 = ldexpf(1.0f, e - 12);
        }
        if (b1 > 0.0f && b1 < 1e30f) {
            frexpf(b1, &e);
            s1 = ldexpf(1.0f, 12 - e);
            inv_s1 = ldexpf(1.0f, e - 12);
        }
    }
    uint32_t phase = 0;
    bool bad = false, any_chunk = false, dw_started = false;
    float acc3[3] = {0.f, 0.f, 0.f}, accb3 = 0.0f;  // dW3 column (lane % W) and db3 (lane < 3)

    // Per-warp work cursor: the warp's current ray and chunk.  Each CTA step
    // every warp renders one chunk (or an empty tile slice), so the barriers
    // below stay CTA-uniform while rays take different numbers of chunks.
    // A ray starts at the chunk that holds sample n_live: every later sample
    // has alpha = 0 and a zero adjoint, and lam = 0 there leaves log T and the
    // suffix term of Eq. 10 at their end-of-ray values.
    // The point after a chunk's last sample is the first sample of the chunk
    // processed just before it (back to front), whose SDF value lane 0 carries
    // over (s_first, valid while have_first); only a ray's first chunk, and
    // the point after the ray's last sample, gather it.
    int64_t ray = next_cta_ray(ray_counter, stride);
    RayIn R;
    RaySpan sp;
    bool have = false, have_first = false;
    int ch = -1;
    float s_first = 0.0f;
    float drgb[3] = {0.f, 0.f, 0.f}, ddepth = 0.f, dwsum = 0.f, logT_end = 0.f, s_carry = 0.f;
    const int nch = (N + 31) >> 5;
    for (;;) {
        if (ch < 0) {
            if (have) ray = next_cta_ray(ray_counter, stride);
            have = false;
            while (ray < A.n_rays) {
                R = load_ray(A, ray);
                sp = ray_span(A, R, ray, stab + 64 * warp);
                const int live = A.n_live ? __ldg(A.n_live + ray) : N;
                if (sp.hit && live > 0) {
                    // the chunk of the last sample with alpha > 0; sample
                    // n_live (alpha = 0) enters only through that sample's
                    // opacity, as the point after it
                    have = true;
                    ch = min(nch - 1, (live - 1) >> 5);
                    break;
                }
                ray = next_cta_ray(ray_counter, stride);
            }
            drgb[0] = drgb[1] = drgb[2] = 0.f;
            ddepth = dwsum = logT_end = 0.f;
            have_first = false;
            if (have) {
                drgb[0] = __ldg(A.d_rgb + 3 * ray);
                drgb[1] = __ldg(A.d_rgb + 3 * ray + 1);
                drgb[2] = __ldg(A.d_rgb + 3 * ray + 2);
                ddepth = A.d_depth ? __ldg(A.d_depth + ray) : 0.0f;
                dwsum = A.d_wsum ? __ldg(A.d_wsum + ray) : 0.0f;
                logT_end = __ldg(A.logT + ray);
            }
            s_carry = drgb[0] * A.bg[0] + drgb[1] * A.bg[1] + drgb[2] * A.bg[2];
        }
        if (!__syncthreads_or(have)) break;
        any_chunk = true;
        {
            const int base = (have ? ch : 0) * 32;
            const int k = base + lane;
            const bool active = have && k < N;
            const int nact = have ? min(32, N - base) : 0;
            const bool extra = active && (lane == 31 || k + 1 >= N);

            // ---- P0: recompute geometry and features -> XH columns [0, 16) ----
            SampleGeom<C> S;
            float t = 0.0f, lam = 0.0f, s_next = 0.0f;
            bool unclipped = false;
            Cell c1;
            c1.base = 0;
            c1.i[0] = c1.i[1] = c1.i[2] = 0;
            c1.f[0] = c1.f[1] = c1.f[2] = 0.0f;
            if (have) {
                t = span_t(sp, k < N ? k : N - 1);
                // the extra point's SDF: carried from the previous chunk's lane
                // 0 (the same point, the same arithmetic, so the same bits), or
                // gathered in a ray's first chunk and after its last sample
                const bool carried = have_first && k + 1 < N;
                if (extra) {
                    float xw[3];
                    point_at(R.o, R.d, span_t(sp, k + 1), xw);
                    c1 = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
                }
                // (features apart from the SDF: gathered below for the samples
                // with a nonzero opacity only; the others' MLP rows carry zeros)
                if constexpr (features_apart<C>())
                    eval_sdf_geom<C>(A, R.o, R.d, t, S);
                else
                    eval_sdf<C>(A, R.o, R.d, t, S);
                s_next = __shfl_down_sync(FULL, S.s, 1);
                if (extra) {
                    if (carried)
                        s_next = s_first;
                    else
                        s_next = sdf_value(A.grid, c1);
                }
                s_first = __shfl_sync(FULL, S.s, 0);
                if (active) {
                    const float diff = log_transmittance(tau, S.s, s_next);
                    unclipped = diff < 0.0f;
                    lam = unclipped ? diff : 0.0f;
                }
                // alpha = 0 where the opacity is clipped: the sample's weight,
                // colour terms, dz rows and so dF (dx) are exactly zero, and its
                // appearance is not needed (see P5)
                if constexpr (L::kKeepBc) {
                    float Bc[L::kBc];
                    if (unclipped) {
                        if constexpr (features_apart<C>()) eval_features<C>(A, R.o, R.d, t, S);
                        eval_appearance_blend<C>(A, R.o, R.d, t, S, Bc);
                    } else {
                        zero_appearance<C>(S);
#pragma unroll
                        for (int i = 0; i < L::kBc; ++i) Bc[i] = 0.0f;
                    }
                    bc_store<L>(t_row, t_row2, Bc);
                } else if (unclipped) {
                    if constexpr (features_apart<C>()) eval_features<C>(A, R.o, R.d, t, S);
                    eval_appearance<C>(A, R.o, R.d, t, S);
                } else {
                    zero_appearance<C>(S);
                }
                float xin[K1];
#pragma unroll
                for (int i = 0; i < K1; ++i) xin[i] = i < NIN ? S.x[i] : (i == NIN ? 1.0f : 0.0f);
                store_row<K1, M::kSplit>(xhh, xhl, tid, 0, L::XHC, xin);
            } else {
                zero_row<K1, M::kSplit>(xhh, xhl, tid, 0, L::XHC);
                S.s = 0.0f;
                if constexpr (L::kKeepBc) {  // warp-collective store: keep every warp in step
                    float Bc[L::kBc];
#pragma unroll
                    for (int i = 0; i < L::kBc; ++i) Bc[i] = 0.0f;
                    bc_store<L>(t_row, t_row2, Bc);
                }
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            if (__syncthreads_or(bad)) goto done;
            tc::fence_after();

            // ---- P1: layer 1; log T_k from a suffix sum of lam ----
            if (tid == 0) {
                mma_k<M::kSplit>(tmem + 0, xhh, xhl, w1h, w1l, 128, L::kSboXH, 128, (K1 / 8) * 128,
                     M::kIdescL, false);
                tc::commit(mbar);
            }
            float suf = lam;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float v = __shfl_down_sync(FULL, suf, off);
                if (lane + off < 32) suf += v;
            }
            const float logTk = logT_end - suf;
            const float Tk = expf(logTk);
            const float Tk1 = expf(logTk + lam);
            const float alpha = -expm1f(lam);
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            uint32_t mask1 = 0;
            {
                float z[W];
                tc::tmem_ld<W>(t_row + 0, z);
                mask1 = bias_relu_mask<W>(z, f32 + M::kB1);
                if (!have) {
#pragma unroll
                    for (int o = 0; o < W; ++o) z[o] = 0.0f;
                }
                store_row<W, M::kSplit>(xhh, xhl, tid, K1, L::XHC, z);
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();

            // ---- P2: layer 2 + 3; compositing adjoint; dz3 -> dz2 ----
            if (tid == 0) {
#pragma unroll
                for (int s = 0; s < W / 16; ++s)
                    mma_k<M::kSplit>(tmem + 32, xhh + 256 + s * 256, xhl + 256 + s * 256, w2h + s * 256,
                         w2l + s * 256, 128, L::kSboXH, 128, (W / 8) * 128, M::kIdescL, s > 0);
                tc::commit(mbar);
            }
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            float h2[W];
            uint32_t mask2 = 0;
            float col[3];
            {
                tc::tmem_ld<W>(t_row + 32, h2);
                mask2 = bias_relu_mask<W>(h2, f32 + M::kB2);
                mlp_layer3<C>(f32, h2, col);
            }
            const float w = active ? Tk * alpha : 0.0f;
            const float G = active ? drgb[0] * col[0] + drgb[1] * col[1] + drgb[2] * col[2] +
                                         ddepth * t + dwsum
                                   : 0.0f;
            const float a_own = active ? expf(lam) : 1.0f;
            const float b_own = active ? alpha * G : 0.0f;
            float Am = __shfl_down_sync(FULL, a_own, 1);
            float Bm = __shfl_down_sync(FULL, b_own, 1);
            if (lane == 31) {
                Am = 1.0f;
                Bm = 0.0f;
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float a2 = __shfl_down_sync(FULL, Am, off);
                const float b2 = __shfl_down_sync(FULL, Bm, off);
                if (lane + off < 32) {
                    Bm = fmaf(Am, b2, Bm);
                    Am = Am * a2;
                }
            }
            const float Shat = fmaf(Am, s_carry, Bm);
            const float next_carry = __shfl_sync(FULL, fmaf(a_own, Shat, b_own), 0);
            const float dlam = unclipped ? -Tk1 * (G - Shat) : 0.0f;
            float dlam_prev = __shfl_up_sync(FULL, dlam, 1);
            if (lane == 0) dlam_prev = 0.0f;
            const float ds_own = active ? (dlam_prev - dlam) * dlog_phi(tau, S.s) : 0.0f;

            float dz3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) dz3[c] = w * drgb[c] * col[c] * (1.0f - col[c]);
            // dW3 and db3 on the CUDA cores.  The warp's rows of the DZ tiles
            // are free until its dz2 row is stored below: h2 goes there
            // transposed (16-byte groups XOR-swizzled by row, so that both the
            // row writes and the column reads are free of bank conflicts) and
            // lane l sums column l of dz3 (x) h2 over the warp's 32 samples.
            {
                float* h2s = reinterpret_cast<float*>(dzh + warp * L::kDZWarp);
#pragma unroll
                for (int v = 0; v < W / 4; ++v)
                    *reinterpret_cast<float4*>(h2s + lane * W + 4 * (v ^ (lane & (W / 4 - 1)))) =
                        make_float4(h2[4 * v], h2[4 * v + 1], h2[4 * v + 2], h2[4 * v + 3]);
                float* d3s = nullptr;
                if constexpr (M::kSplit == 2) {
                    d3s = reinterpret_cast<float*>(dzl + warp * L::kDZWarp);
                    *reinterpret_cast<float4*>(d3s + 4 * lane) =
                        make_float4(dz3[0], dz3[1], dz3[2], 0.0f);
                }
                __syncwarp();
                const int col_l = lane & (W - 1);
#pragma unroll 8
                for (int r = 0; r < 32; ++r) {
                    const float h = h2s[r * W + 4 * ((col_l >> 2) ^ (r & (W / 4 - 1))) + (col_l & 3)];
                    float e0, e1, e2;
                    if constexpr (M::kSplit == 2) {
                        const float4 e = *reinterpret_cast<const float4*>(d3s + 4 * r);
                        e0 = e.x;
                        e1 = e.y;
                        e2 = e.z;
                    } else {
                        e0 = __shfl_sync(FULL, dz3[0], r);
                        e1 = __shfl_sync(FULL, dz3[1], r);
                        e2 = __shfl_sync(FULL, dz3[2], r);
                    }
                    acc3[0] = fmaf(e0, h, acc3[0]);
                    acc3[1] = fmaf(e1, h, acc3[1]);
                    acc3[2] = fmaf(e2, h, acc3[2]);
                }
                __syncwarp();
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float sb = dz3[c];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sb += __shfl_xor_sync(FULL, sb, off);
                if (lane == c) accb3 += sb;
            }
            {
                // dh2 = W3^T dz3 over pairs of hidden units (W3 row-major)
                float dz2[W];
                const float2 e0 = make_float2(dz3[0], dz3[0]), e1 = make_float2(dz3[1], dz3[1]);
                const float2 e2 = make_float2(dz3[2], dz3[2]), sc2 = make_float2(s2, s2);
#pragma unroll
                for (int i = 0; i < W; i += 2) {
                    float2 dh2 = mul2(*reinterpret_cast<const float2*>(f32 + M::kW3 + i), e0);
                    dh2 = fma2(*reinterpret_cast<const float2*>(f32 + M::kW3 + W + i), e1, dh2);
                    dh2 = fma2(*reinterpret_cast<const float2*>(f32 + M::kW3 + 2 * W + i), e2, dh2);
                    dh2 = mul2(dh2, sc2);
                    dz2[i] = ((mask2 >> i) & 1u) ? dh2.x : 0.0f;
                    dz2[i + 1] = ((mask2 >> (i + 1)) & 1u) ? dh2.y : 0.0f;
                }
                store_row<W, M::kSplit>(dzh, dzl, tid, W, L::DZC, dz2);
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();

            // ---- P3: dh1 = dz2 W2 (W2 read as its transpose) -> dz1 ----
            if (tid == 0) {
                const uint32_t idesc = tc::idesc_f16(128, W, 0, 1);
#pragma unroll
                for (int s = 0; s < W / 16; ++s)
                    mma_k<M::kSplit>(tmem + 0, dzh + (W / 8) * 128 + s * 256, dzl + (W / 8) * 128 + s * 256,
                         w2h + s * 2 * (W / 8) * 128, w2l + s * 2 * (W / 8) * 128, 128,
                         L::kSboDZ, (W / 8) * 128, 128, idesc, s > 0);
                tc::commit(mbar);
            }
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            {
                float dh1[W];
                tc::tmem_ld<W>(t_row + 0, dh1);
                const float r12 = s1 * inv_s2;  // dh1 arrives scaled by s2; dz1 is stored scaled by s1
                const float2 r2 = make_float2(r12, r12);
#pragma unroll
                for (int i = 0; i < W; i += 2) {
                    const float2 v = mul2(make_float2(dh1[i], dh1[i + 1]), r2);
                    dh1[i] = ((mask1 >> i) & 1u) ? v.x : 0.0f;
                    dh1[i + 1] = ((mask1 >> (i + 1)) & 1u) ? v.y : 0.0f;
                }
                store_row<W, M::kSplit>(dzh, dzl, tid, 0, L::DZC, dh1);
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();

            // ---- P4: dx = dz1 W1 (transposed W1) and the weight gradient ----
            if (tid == 0) {
                const uint32_t idx = tc::idesc_f16(128, 16, 0, 1);
#pragma unroll
                for (int s = 0; s < W / 16; ++s)
                    mma_k<M::kSplit>(tmem + 32, dzh + s * 256, dzl + s * 256, w1h + s * 512, w1l + s * 512,
                         128, L::kSboDZ, 256, 128, idx, s > 0);
                const uint32_t idw = tc::idesc_f16(64, L::XHC, 1, 1);
#pragma unroll
                for (int s = 0; s < 8; ++s)
                    mma_k<M::kSplit>(tmem + 64, dzh + s * 2 * L::kSboDZ, dzl + s * 2 * L::kSboDZ,
                         xhh + s * 2 * L::kSboXH, xhl + s * 2 * L::kSboXH, L::kSboDZ, 128,
                         L::kSboXH, 128, idw, dw_started || s > 0);
                dw_started = true;
                tc::commit(mbar);
            }
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            float dx[16];
            tc::tmem_ld<16>(t_row + 32, dx);
            {
                const float2 is1 = make_float2(inv_s1, inv_s1);
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const float2 v = mul2(make_float2(dx[i], dx[i + 1]), is1);
                    dx[i] = v.x;
                    dx[i + 1] = v.y;
                }
            }
            tc::fence_before();
            __syncthreads();  // tiles are free from here on

            // ---- P5: angular / Fresnel / normal adjoints and grid reductions ----
            // Samples with a clipped opacity have dx = 0 exactly: no angular,
            // Fresnel or normal adjoint, and only the SDF-value gradient of the
            // transmittance term (ds_own), skipped when that is zero too.
            float* pst = reinterpret_cast<float*>(dzh) + warp * 32 * L::PST;
            if (have) {
                float gxs = 0.0f, gys = 0.0f, gzs = 0.0f;
                float Bc[L::kKeepBc ? L::kBc : 1];
                if constexpr (L::kKeepBc) bc_load<L>(t_row, t_row2, Bc);  // warp-collective
                if (unclipped) {
                    float wq[8];
                    corner_weights(S.pcell.f, wq);
                    float dY[L2];
#pragma unroll
                    for (int j = 0; j < L2; ++j) dY[j] = 0.0f;
                    if constexpr (L::kKeepBc) {
                        // dF_a,c / dY_j = Bc_jc (Eq. 7)
#pragma unroll
                        for (int j = 0; j < L2; ++j)
#pragma unroll
                            for (int c = 0; c < NA; ++c)
                                dY[j] = fmaf(Bc[j * NA + c], dx[3 + c], dY[j]);
                    } else {
                    int pidx[8];
                    probe_corner_index(A.probes, S.pcell, pidx);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
#pragma unroll
                        for (int j = 0; j < L2; ++j) {
                            float acc = 0.0f;
#pragma unroll
                            for (int cg = 0; cg < C::NA4; ++cg) {
                                const float4 bb = probe_coeffs<C>(A.probes, pidx[q], j, cg);
                                acc = fmaf(bb.x, dx[3 + 4 * cg + 0], acc);
                                acc = fmaf(bb.y, dx[3 + 4 * cg + 1], acc);
                                acc = fmaf(bb.z, dx[3 + 4 * cg + 2], acc);
                                acc = fmaf(bb.w, dx[3 + 4 * cg + 3], acc);
                            }
                            dY[j] = fmaf(wq[q], acc, dY[j]);
                        }
                    }
                    }
                    {
                        float Y[L2];
                        sh_basis<L2>(S.r, Y);
                        float* row = pst + lane * L::PST;
#pragma unroll
                        for (int q = 0; q < 8; ++q) row[q] = wq[q];
#pragma unroll
                        for (int j = 0; j < L2; ++j) row[8 + j] = Y[j];
#pragma unroll
                        for (int c = 0; c < NA; ++c) row[8 + L2 + c] = dx[3 + c];
                        row[8 + L2 + NA] = __int_as_float(S.pcell.base);
                    }
                    float dr[3];
                    sh_basis_vjp<L2>(S.r, dY, dr);
                    const float v[3] = {-R.d[0], -R.d[1], -R.d[2]};
                    float dn[3] = {0.f, 0.f, 0.f};
                    if (A.dir_mode != 1) {
                        const float drn = dr[0] * S.n[0] + dr[1] * S.n[1] + dr[2] * S.n[2];
#pragma unroll
                        for (int a = 0; a < 3; ++a) dn[a] = 2.0f * drn * v[a] + 2.0f * S.ndv * dr[a];
                    }
                    {
                        const float om = 1.0f - S.ndv;
                        float dndv = 0.0f, pw = 1.0f;
#pragma unroll
                        for (int kk = 1; kk <= C::K; ++kk) {
                            dndv -= dx[3 + NA + kk - 1] * static_cast<float>(kk) * pw;
                            pw *= om;
                        }
#pragma unroll
                        for (int a = 0; a < 3; ++a) dn[a] = fmaf(dndv, v[a], dn[a]);
                    }
                    const float ndn = S.n[0] * dn[0] + S.n[1] * dn[1] + S.n[2] * dn[2];
                    const float irho = 1.0f / S.rho;
                    gxs = (dn[0] - S.n[0] * ndn) * irho * A.grid.sc[0];
                    gys = (dn[1] - S.n[1] * ndn) * irho * A.grid.sc[1];
                    gzs = (dn[2] - S.n[2] * ndn) * irho * A.grid.sc[2];
                }
                if (unclipped) {
                    const float fx = S.cell.f[0], fy = S.cell.f[1], fz = S.cell.f[2];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int cx = q & 1, cy = (q >> 1) & 1, cz = (q >> 2) & 1;
                        const float wx = cx ? fx : 1.0f - fx, sgx = cx ? 1.0f : -1.0f;
                        const float wy = cy ? fy : 1.0f - fy, sgy = cy ? 1.0f : -1.0f;
                        const float wz = cz ? fz : 1.0f - fz, sgz = cz ? 1.0f : -1.0f;
                        const float wc = wx * wy * wz;
                        const float dsdf = ds_own * wc + gxs * sgx * wy * wz +
                                           gys * wx * sgy * wz + gzs * wx * wy * sgz;
                        const int64_t node = grad_record<C>(A.grid, S.cell, q);
                        if (C::SP && node < 0) continue;  // a brick that is not stored
                        if constexpr (C::TP)
                            red_add(A.grad_grid + node, dsdf);
                        else
                            red_add_v4(A.grad_grid + A.grid.rec_off + 4 * node, dsdf, wc * dx[0],
                                       wc * dx[1], wc * dx[2]);
                    }
                    if constexpr (C::TP) {
                        // F_s = b0 b1 b2 per channel: plane p's lookup gets dF_s times
                        // the other two, spread over its 4 texels bilinearly
                        float xw[3];
                        point_at(R.o, R.d, t, xw);
                        TriAt T;
                        triplane_locate(A.grid, xw, T);
                        float4 bp[3];
                        float fs_unused[3];
                        triplane_lookup(A.grid, T, fs_unused, bp);
                        float4* gpl = reinterpret_cast<float4*>(A.grad_grid + A.grid.plane_off);
#pragma unroll
                        for (int p = 0; p < 3; ++p) {
                            const float4 o1 = bp[(p + 1) % 3], o2 = bp[(p + 2) % 3];
                            const float gx0 = dx[0] * o1.x * o2.x, gx1 = dx[1] * o1.y * o2.y;
                            const float gx2 = dx[2] * o1.z * o2.z;
                            const int ra = tri_row(p), ca = tri_col(p);
                            const float fr = T.f[ra], fc = T.f[ca];
                            float4* P = gpl + T.plane0 + p * kTile * kTile + T.i[ra] * kTile +
                                        T.i[ca];
                            const float w4[4] = {(1.0f - fr) * (1.0f - fc), (1.0f - fr) * fc,
                                                 fr * (1.0f - fc), fr * fc};
                            const int o4[4] = {0, 1, kTile, kTile + 1};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                red_add_v4(reinterpret_cast<float*>(P + o4[e]), w4[e] * gx0,
                                           w4[e] * gx1, w4[e] * gx2, 0.0f);
                        }
                    }
                } else if (active && ds_own != 0.0f) {
                    float w8[8];
                    corner_weights(S.cell.f, w8);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int64_t node = grad_record<C>(A.grid, S.cell, q);
                        if (C::SP && node < 0) continue;
                        red_add(A.grad_grid + (C::TP ? node : A.grid.rec_off + 4 * node),
                                ds_own * w8[q]);
                    }
                }
                if (extra) {
                    const float ds1 = dlam * dlog_phi(tau, s_next);
                    if (ds1 != 0.0f) {
                        float w1[8];
                        corner_weights(c1.f, w1);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int64_t node = grad_record<C>(A.grid, c1, q);
                            if (C::SP && node < 0) continue;
                            red_add(A.grad_grid + (C::TP ? node : A.grid.rec_off + 4 * node),
                                    ds1 * w1[q]);
                        }
                    }
                }
                // runs of live samples in one probe cell end where the next live
                // sample's cell differs (or no live sample follows)
                const uint32_t live = __ballot_sync(FULL, unclipped);
                const int my_cell = unclipped ? S.pcell.base : -1;
                const uint32_t later = lane == 31 ? 0u : live & (0xffffffffu << (lane + 1));
                const int nl = __ffs(later) - 1;
                const int next_cell = __shfl_sync(FULL, my_cell, nl >= 0 ? nl : lane);
                const uint32_t ends =
                    __ballot_sync(FULL, unclipped && (nl < 0 || next_cell != my_cell));
                __syncwarp();
                scatter_probe_grad<C, L::PST>(A, pst, live, ends, lane);
                logT_end = __shfl_sync(FULL, logTk, 0);
                s_carry = next_carry;
                have_first = true;
            }
        }
        if (have) --ch;
    }
done:
    // every thread reaches this point together (the loop exits and the jump
    // above are CTA-uniform), so the flag can be made uniform here
    bad = __syncthreads_or(bad);
    if (bad) {
        // the last commit's phase has the parity before the final flip
        tc::mbar_wait(mbar, phase ^ 1u);
        if (tid == 0) atomicOr(A.status, 1);
    }
    // the tiles are free: every MMA that read them has completed (the loop
    // waited for each one), and so has every warp's use of the probe staging
    const bool fold = any_chunk && !bad;
    if (fold)
        for (int i = tid; i < L::kParamsPad; i += blockDim.x) gacc[i] = 0.0f;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (fold) {
        // dW1, db1, dW2, db2 from the tensor-memory accumulator (M = 64 layout:
        // row r lives in lane 32 (r / 16) + r % 16)
        float v[L::XHC];
        tc::tmem_ld<L::XHC>(t_row + 64, v);
        const int r = 16 * warp + lane;
        if (lane < 16) {
            if (r < W) {  // dz1 rows, scaled by s1
#pragma unroll
                for (int j = 0; j < NIN; ++j) gacc[C::gW1 + r * NIN + j] += v[j] * inv_s1;
                gacc[C::gB1 + r] += v[NIN] * inv_s1;
            } else if (r < 2 * W) {  // dz2 rows, scaled by s2
#pragma unroll
                for (int i = 0; i < W; ++i) gacc[C::gW2 + (r - W) * W + i] += v[K1 + i] * inv_s2;
                gacc[C::gB2 + (r - W)] += v[NIN] * inv_s2;
            }
        }
        if (lane < W) {  // lane l holds column l (see P2)
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(gacc + C::gW3 + c * W + lane, acc3[c]);
        }
        if (lane < 3) atomicAdd(gacc + C::gB3 + lane, accb3);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tmem_dealloc(tmem, L::kTmemCols);
        if constexpr (L::kKeepBc) tc::tmem_dealloc(*tslot2, L::kTmemCols2);
    }
    if (fold)
        for (int i = tid; i < C::kParams; i += blockDim.x) red_add(A.grad_mlp + i, gacc[i]);
}

template <class C>
cudaError_t launch_backward_t(const RenderArgs& A, int grid_ctas, cudaStream_t stream)
{
    using L = BwdLayout<C>;
    cudaError_t e = cudaFuncSetAttribute(render_backward_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e == cudaSuccess)
        e = set_smem_carveout(reinterpret_cast<const void*>(render_backward_kernel<C>),
                              kBwdThreads, L::kBytes, L::kTmemCols + L::kTmemCols2);
    if (e != cudaSuccess) return e;
    render_backward_kernel<C><<<grid_ctas, kBwdThreads, L::kBytes, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_backward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                            cudaStream_t stream)
{
#define PSDF_BWD_CASE(NA, L2, W, K, FB, PH, MH)                                              \
    if (ks.match(NA, L2, W, K, FB, PH, MH))                                                  \
        return launch_backward_t<Cfg<NA, L2, W, K, FB, PH, MH>>(A, grid_ctas, stream);
    PSDF_FOR_EACH_SHAPE(PSDF_BWD_CASE)
#undef PSDF_BWD_CASE
    return cudaErrorInvalidValue;
}

template <class C>
cudaError_t backward_occupancy_t(int* n)
{
    using L = BwdLayout<C>;
    cudaError_t e = cudaFuncSetAttribute(render_backward_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, render_backward_kernel<C>);
    if (e != cudaSuccess) return e;
    *n = resident_ctas(fa, kBwdThreads, L::kBytes, L::kTmemCols + L::kTmemCols2);
    return *n > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t backward_ctas_per_sm(const KernelShape& ks, int* n)
{
    *n = 0;
#define PSDF_BWD_OCC(NA, L2, W, K, FB, PH, MH)                                               \
    if (ks.match(NA, L2, W, K, FB, PH, MH))                                                  \
        return backward_occupancy_t<Cfg<NA, L2, W, K, FB, PH, MH>>(n);
    PSDF_FOR_EACH_SHAPE(PSDF_BWD_OCC)
#undef PSDF_BWD_OCC
    return cudaErrorInvalidValue;
}

}  // namespace psdf
