// Adjoint of the ProbeSDF render (Sec. 3.3-3.4), FP32, sm_103a.
//
// Each warp walks its ray's 32-sample chunks back to front starting from the
// saved log T_N, recomputing every per-sample activation (nothing per sample
// is stored by the forward).  Per chunk:
//   - transmittance from a warp suffix-sum of the clipped log-opacities;
//   - the suffix term of dL/dalpha_k = T_k (G_k - S_k) from a warp scan of
//     the affine recurrence S_k = alpha_{k+1} G_{k+1} + (1 - alpha_{k+1}) S_{k+1};
//   - MLP backward per lane, the weight gradient as a lane-transposed pass
//     over the chunk's activation rows in shared memory (one CTA-level
//     shared-memory accumulator, flushed to global memory once per CTA);
//   - SDF / feature gradients as one 16-byte vector reduction per corner;
//   - probe gradients reduced over runs of samples that share a probe cell
//     (consecutive along a ray) before the global reductions.
#include "internal.h"
#include "sample_eval.cuh"

namespace psdf {

template <class C>
struct BwdLayout {
    static constexpr int HS = C::W + 4;                  // row stride of h1/h2/dz rows
    static constexpr int PST = ((8 + C::L2 + C::NA + 1) + 3) & ~3;  // probe staging row
    static constexpr int kParamsPad = (C::kParams + 3) & ~3;
    static constexpr int kMlpPad = (C::kMlpSmem + 3) & ~3;
    // per-warp region
    static constexpr int kXs = 0;
    static constexpr int kH1 = kXs + 32 * C::NINP;
    static constexpr int kH2 = kH1 + 32 * HS;
    static constexpr int kDz1 = kH2 + 32 * HS;
    static constexpr int kDz2 = kDz1 + 32 * HS;
    static constexpr int kDz3 = kDz2 + 32 * HS;
    static constexpr int kPst = kDz3 + 32 * 4;
    static constexpr int kWarpFloats = kPst + 32 * PST;
    static constexpr int kWarps = kBwdThreads / 32;
    static constexpr int kSmemFloats = kMlpPad + kParamsPad + kWarps * kWarpFloats;
    static constexpr size_t kSmemBytes = sizeof(float) * kSmemFloats;
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// Lane-transposed accumulation of the MLP weight gradient over the chunk's
// nact activation rows; results are added to the CTA accumulator gacc
// (packed global layout).
template <class C, class Lay>
__device__ __forceinline__ void accumulate_dw(const float* xs, const float* h1s, const float* h2s,
                                              const float* dz1s, const float* dz2s,
                                              const float* dz3s, int nact, int lane, float* gacc)
{
    constexpr int W = C::W, NINP = C::NINP, NIN = C::NIN, HS = Lay::HS;
    if constexpr (W == 32) {
        const int o = lane;
        float a1[NINP], a2[W], a3[3] = {0.f, 0.f, 0.f};
        float db1 = 0.f, db2 = 0.f, db3 = 0.f;
#pragma unroll
        for (int i = 0; i < NINP; ++i) a1[i] = 0.f;
#pragma unroll
        for (int i = 0; i < W; ++i) a2[i] = 0.f;
        for (int s = 0; s < nact; ++s) {
            const float d1 = dz1s[s * HS + o];
            const float d2 = dz2s[s * HS + o];
            const float h2o = h2s[s * HS + o];
            const float4 d3 = ld4(dz3s + 4 * s);
#pragma unroll
            for (int q = 0; q < NINP / 4; ++q) {
                const float4 xv = ld4(xs + s * NINP + 4 * q);
                a1[4 * q + 0] = fmaf(d1, xv.x, a1[4 * q + 0]);
                a1[4 * q + 1] = fmaf(d1, xv.y, a1[4 * q + 1]);
                a1[4 * q + 2] = fmaf(d1, xv.z, a1[4 * q + 2]);
                a1[4 * q + 3] = fmaf(d1, xv.w, a1[4 * q + 3]);
            }
#pragma unroll
            for (int q = 0; q < W / 4; ++q) {
                const float4 hv = ld4(h1s + s * HS + 4 * q);
                a2[4 * q + 0] = fmaf(d2, hv.x, a2[4 * q + 0]);
                a2[4 * q + 1] = fmaf(d2, hv.y, a2[4 * q + 1]);
                a2[4 * q + 2] = fmaf(d2, hv.z, a2[4 * q + 2]);
                a2[4 * q + 3] = fmaf(d2, hv.w, a2[4 * q + 3]);
            }
            a3[0] = fmaf(d3.x, h2o, a3[0]);
            a3[1] = fmaf(d3.y, h2o, a3[1]);
            a3[2] = fmaf(d3.z, h2o, a3[2]);
            db1 += d1;
            db2 += d2;
            db3 += lane == 0 ? d3.x : (lane == 1 ? d3.y : d3.z);
        }
#pragma unroll
        for (int i = 0; i < NIN; ++i) atomicAdd(gacc + C::gW1 + o * NIN + i, a1[i]);
        atomicAdd(gacc + C::gB1 + o, db1);
#pragma unroll
        for (int i = 0; i < W; ++i) atomicAdd(gacc + C::gW2 + o * W + i, a2[i]);
        atomicAdd(gacc + C::gB2 + o, db2);
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(gacc + C::gW3 + c * W + o, a3[c]);
        if (lane < 3) atomicAdd(gacc + C::gB3 + lane, db3);
    } else {
        static_assert(W == 16, "hidden width 16 or 32");
        const int o = lane & 15;
        if (lane < 16) {
            // W1 row o, b1[o], W3 column o, b3
            float a1[NINP], a3[3] = {0.f, 0.f, 0.f};
            float db1 = 0.f, db3 = 0.f;
#pragma unroll
            for (int i = 0; i < NINP; ++i) a1[i] = 0.f;
            for (int s = 0; s < nact; ++s) {
                const float d1 = dz1s[s * HS + o];
                const float h2o = h2s[s * HS + o];
                const float4 d3 = ld4(dz3s + 4 * s);
#pragma unroll
                for (int q = 0; q < NINP / 4; ++q) {
                    const float4 xv = ld4(xs + s * NINP + 4 * q);
                    a1[4 * q + 0] = fmaf(d1, xv.x, a1[4 * q + 0]);
                    a1[4 * q + 1] = fmaf(d1, xv.y, a1[4 * q + 1]);
                    a1[4 * q + 2] = fmaf(d1, xv.z, a1[4 * q + 2]);
                    a1[4 * q + 3] = fmaf(d1, xv.w, a1[4 * q + 3]);
                }
                a3[0] = fmaf(d3.x, h2o, a3[0]);
                a3[1] = fmaf(d3.y, h2o, a3[1]);
                a3[2] = fmaf(d3.z, h2o, a3[2]);
                db1 += d1;
                db3 += lane == 0 ? d3.x : (lane == 1 ? d3.y : d3.z);
            }
#pragma unroll
            for (int i = 0; i < NIN; ++i) atomicAdd(gacc + C::gW1 + o * NIN + i, a1[i]);
            atomicAdd(gacc + C::gB1 + o, db1);
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(gacc + C::gW3 + c * W + o, a3[c]);
            if (lane < 3) atomicAdd(gacc + C::gB3 + lane, db3);
        } else {
            // W2 row o, b2[o]
            float a2[W];
            float db2 = 0.f;
#pragma unroll
            for (int i = 0; i < W; ++i) a2[i] = 0.f;
            for (int s = 0; s < nact; ++s) {
                const float d2 = dz2s[s * HS + o];
#pragma unroll
                for (int q = 0; q < W / 4; ++q) {
                    const float4 hv = ld4(h1s + s * HS + 4 * q);
                    a2[4 * q + 0] = fmaf(d2, hv.x, a2[4 * q + 0]);
                    a2[4 * q + 1] = fmaf(d2, hv.y, a2[4 * q + 1]);
                    a2[4 * q + 2] = fmaf(d2, hv.z, a2[4 * q + 2]);
                    a2[4 * q + 3] = fmaf(d2, hv.w, a2[4 * q + 3]);
                }
                db2 += d2;
            }
#pragma unroll
            for (int i = 0; i < W; ++i) atomicAdd(gacc + C::gW2 + o * W + i, a2[i]);
            atomicAdd(gacc + C::gB2 + o, db2);
        }
    }
}

// Probe-coefficient gradient (Eqs. 6-7): dL/db_ijc = sum_k w_i(k) Y_j(k) dF_a,c(k).
// Samples of a chunk that share a probe cell are consecutive; lane (corner i,
// channel c) sums each run and issues one reduction per coefficient.
template <class C, class Lay>
__device__ __forceinline__ void scatter_probe_grad(const RenderArgs& A, const float* pst, int nact,
                                                   int lane)
{
    constexpr int L2 = C::L2, NA = C::NA, PST = Lay::PST;
    constexpr int CPL = (8 * NA) / 32;
    static_assert((8 * NA) % 32 == 0, "8 corners x channels must fill whole warps");
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
    for (int s = 0; s < nact; ++s) {
        const float* row = pst + s * PST;
        const int cell = __float_as_int(row[8 + L2 + NA]);
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const float coef = row[q[m]] * row[8 + L2 + ch[m]];
#pragma unroll
            for (int j = 0; j < L2; ++j) acc[m][j] = fmaf(coef, row[8 + j], acc[m][j]);
        }
        const int next = s + 1 < nact ? __float_as_int(pst[(s + 1) * PST + 8 + L2 + NA]) : -1;
        if (next != cell) {
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
    }
}

template <class C>
__global__ void __launch_bounds__(kBwdThreads)
render_backward_kernel(RenderArgs A)
{
    using Lay = BwdLayout<C>;
    constexpr int W = C::W, NINP = C::NINP, HS = Lay::HS, NA = C::NA, L2 = C::L2;
    extern __shared__ __align__(16) float smem[];
    float* sw = smem;
    float* gacc = smem + Lay::kMlpPad;
    const int warp_in_cta = threadIdx.x >> 5;
    float* wreg = gacc + Lay::kParamsPad + warp_in_cta * Lay::kWarpFloats;
    float* xs = wreg + Lay::kXs;
    float* h1s = wreg + Lay::kH1;
    float* h2s = wreg + Lay::kH2;
    float* dz1s = wreg + Lay::kDz1;
    float* dz2s = wreg + Lay::kDz2;
    float* dz3s = wreg + Lay::kDz3;
    float* pst = wreg + Lay::kPst;

    load_mlp_smem<C>(A.mlp, sw);
    for (int i = threadIdx.x; i < Lay::kParamsPad; i += blockDim.x) gacc[i] = 0.0f;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int N = A.n_samples;
    const float tau = A.tau;
    const unsigned FULL = 0xffffffffu;

    for (int64_t ray = warp0; ray < A.n_rays; ray += nwarps) {
        const RayIn R = load_ray(A, ray);
        const RaySpan sp = ray_span(A, R, ray);
        if (!sp.hit) continue;
        const float drgb[3] = {__ldg(A.d_rgb + 3 * ray), __ldg(A.d_rgb + 3 * ray + 1),
                               __ldg(A.d_rgb + 3 * ray + 2)};
        const float ddepth = A.d_depth ? __ldg(A.d_depth + ray) : 0.0f;
        const float dwsum = A.d_wsum ? __ldg(A.d_wsum + ray) : 0.0f;
        float logT_end = __ldg(A.logT + ray);  // log T at the point after the chunk
        float s_carry = drgb[0] * A.bg[0] + drgb[1] * A.bg[1] + drgb[2] * A.bg[2];
        const int nch = (N + 31) >> 5;

        for (int ch = nch - 1; ch >= 0; --ch) {
            const int base = ch * 32;
            const int k = base + lane;
            const bool active = k < N;
            const int nact = min(32, N - base);
            const float t = span_t(sp, active ? k : N - 1);

            SampleGeom<C> S;
            eval_geometry<C>(A, R.o, R.d, t, S);
            float col[3];
            mlp_forward<C, true>(sw, S.x, col, xs + lane * NINP, h1s + lane * HS,
                                 h2s + lane * HS);

            // s at point k+1 (extra gather for the chunk's last sample)
            float s_next = __shfl_down_sync(FULL, S.s, 1);
            const bool extra = active && (lane == 31 || k + 1 >= N);
            Cell c1;
            c1.base = 0;
            c1.f[0] = c1.f[1] = c1.f[2] = 0.f;
            if (extra) {
                float xw[3];
                point_at(R.o, R.d, span_t(sp, k + 1), xw);
                c1 = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
                s_next = sdf_value(A.grid, c1);
            }
            float lam = 0.0f;
            bool unclipped = false;
            if (active) {
                const float diff = log_transmittance(tau, S.s, s_next);
                unclipped = diff < 0.0f;
                lam = unclipped ? diff : 0.0f;
            }
            // inclusive suffix sum of lam over the chunk: log T_k = log T_end - suf
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
            const float w = active ? Tk * alpha : 0.0f;
            const float G = active ? drgb[0] * col[0] + drgb[1] * col[1] + drgb[2] * col[2] +
                                         ddepth * t + dwsum
                                   : 0.0f;
            // suffix recurrence S_k = a_{k+1} S_{k+1} + b_{k+1}, a = 1 - alpha, b = alpha G
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

            // ---- colour path: sigmoid, MLP backward ----
            float dz3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) dz3[c] = w * drgb[c] * col[c] * (1.0f - col[c]);
            st4(dz3s + 4 * lane, dz3[0], dz3[1], dz3[2], 0.0f);
            float dh1[W];
#pragma unroll
            for (int i = 0; i < W; ++i) dh1[i] = 0.0f;
            const float* h2row = h2s + lane * HS;
            float* dz2row = dz2s + lane * HS;
#pragma unroll
            for (int o4 = 0; o4 < W / 4; ++o4) {
                const float4 hv = ld4(h2row + 4 * o4);
                const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
                float dz2v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int o = 4 * o4 + u;
                    const float4 w3 = ld4(sw + C::kW3T + 4 * o);
                    const float dh2 = w3.x * dz3[0] + w3.y * dz3[1] + w3.z * dz3[2];
                    const float dz2 = hh[u] > 0.0f ? dh2 : 0.0f;
                    dz2v[u] = dz2;
                    const float4* wr = reinterpret_cast<const float4*>(sw + C::kW2 + o * W);
#pragma unroll
                    for (int q = 0; q < W / 4; ++q) {
                        const float4 w4 = wr[q];
                        dh1[4 * q + 0] = fmaf(w4.x, dz2, dh1[4 * q + 0]);
                        dh1[4 * q + 1] = fmaf(w4.y, dz2, dh1[4 * q + 1]);
                        dh1[4 * q + 2] = fmaf(w4.z, dz2, dh1[4 * q + 2]);
                        dh1[4 * q + 3] = fmaf(w4.w, dz2, dh1[4 * q + 3]);
                    }
                }
                st4(dz2row + 4 * o4, dz2v[0], dz2v[1], dz2v[2], dz2v[3]);
            }
            float dx[NINP];
#pragma unroll
            for (int i = 0; i < NINP; ++i) dx[i] = 0.0f;
            const float* h1row = h1s + lane * HS;
            float* dz1row = dz1s + lane * HS;
#pragma unroll
            for (int i4 = 0; i4 < W / 4; ++i4) {
                const float4 hv = ld4(h1row + 4 * i4);
                const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
                float dz1v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = 4 * i4 + u;
                    const float dz1 = hh[u] > 0.0f ? dh1[i] : 0.0f;
                    dz1v[u] = dz1;
                    const float4* wr = reinterpret_cast<const float4*>(sw + C::kW1 + i * NINP);
#pragma unroll
                    for (int q = 0; q < NINP / 4; ++q) {
                        const float4 w4 = wr[q];
                        dx[4 * q + 0] = fmaf(w4.x, dz1, dx[4 * q + 0]);
                        dx[4 * q + 1] = fmaf(w4.y, dz1, dx[4 * q + 1]);
                        dx[4 * q + 2] = fmaf(w4.z, dz1, dx[4 * q + 2]);
                        dx[4 * q + 3] = fmaf(w4.w, dz1, dx[4 * q + 3]);
                    }
                }
                st4(dz1row + 4 * i4, dz1v[0], dz1v[1], dz1v[2], dz1v[3]);
            }

            // ---- angular features: dY, probe-gradient staging ----
            float wq[8];
            corner_weights(S.pcell.f, wq);
            int pidx[8];
            probe_corner_index(A.probes, S.pcell, pidx);
            float dY[L2];
#pragma unroll
            for (int j = 0; j < L2; ++j) dY[j] = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4* b = A.probes.coeffs + (size_t)pidx[q] * (L2 * C::NA4);
#pragma unroll
                for (int j = 0; j < L2; ++j) {
                    float acc = 0.0f;
#pragma unroll
                    for (int cg = 0; cg < C::NA4; ++cg) {
                        const float4 bb = __ldg(b + j * C::NA4 + cg);
                        acc = fmaf(bb.x, dx[3 + 4 * cg + 0], acc);
                        acc = fmaf(bb.y, dx[3 + 4 * cg + 1], acc);
                        acc = fmaf(bb.z, dx[3 + 4 * cg + 2], acc);
                        acc = fmaf(bb.w, dx[3 + 4 * cg + 3], acc);
                    }
                    dY[j] = fmaf(wq[q], acc, dY[j]);
                }
            }
            {
                float* row = pst + lane * Lay::PST;
#pragma unroll
                for (int q = 0; q < 8; ++q) row[q] = wq[q];
#pragma unroll
                for (int j = 0; j < L2; ++j) row[8 + j] = S.Y[j];
#pragma unroll
                for (int c = 0; c < NA; ++c) row[8 + L2 + c] = active ? dx[3 + c] : 0.0f;
                row[8 + L2 + NA] = __int_as_float(S.pcell.base);
            }

            // ---- normal path: r(n), Fresnel(n), n(g) ----
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
            const float gxs = (dn[0] - S.n[0] * ndn) * irho * A.grid.sc[0];
            const float gys = (dn[1] - S.n[1] * ndn) * irho * A.grid.sc[1];
            const float gzs = (dn[2] - S.n[2] * ndn) * irho * A.grid.sc[2];

            // ---- SDF + feature node gradients: one vector reduction per corner ----
            if (active) {
                const float fx = S.cell.f[0], fy = S.cell.f[1], fz = S.cell.f[2];
                const int sy = A.grid.R[0], sz = A.grid.R[0] * A.grid.R[1];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int cx = q & 1, cy = (q >> 1) & 1, cz = (q >> 2) & 1;
                    const float wx = cx ? fx : 1.0f - fx, sgx = cx ? 1.0f : -1.0f;
                    const float wy = cy ? fy : 1.0f - fy, sgy = cy ? 1.0f : -1.0f;
                    const float wz = cz ? fz : 1.0f - fz, sgz = cz ? 1.0f : -1.0f;
                    const float wc = wx * wy * wz;
                    const float dsdf = ds_own * wc + gxs * sgx * wy * wz + gys * wx * sgy * wz +
                                       gzs * wx * wy * sgz;
                    float* dst = A.grad_grid + 4 * (size_t)(S.cell.base + cx + cy * sy + cz * sz);
                    red_add_v4(dst, dsdf, wc * dx[0], wc * dx[1], wc * dx[2]);
                }
            }
            if (extra) {
                const float ds1 = dlam * dlog_phi(tau, s_next);
                float w1[8];
                corner_weights(c1.f, w1);
                const int sy = A.grid.R[0], sz = A.grid.R[0] * A.grid.R[1];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int cx = q & 1, cy = (q >> 1) & 1, cz = (q >> 2) & 1;
                    red_add(A.grad_grid + 4 * (size_t)(c1.base + cx + cy * sy + cz * sz),
                            ds1 * w1[q]);
                }
            }

            __syncwarp();
            accumulate_dw<C, Lay>(xs, h1s, h2s, dz1s, dz2s, dz3s, nact, lane, gacc);
            scatter_probe_grad<C, Lay>(A, pst, nact, lane);
            __syncwarp();

            logT_end = __shfl_sync(FULL, logTk, 0);
            s_carry = next_carry;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C::kParams; i += blockDim.x) red_add(A.grad_mlp + i, gacc[i]);
}

template <class C>
cudaError_t launch_backward_t(const RenderArgs& A, int grid_ctas, cudaStream_t stream)
{
    using Lay = BwdLayout<C>;
    cudaError_t e = cudaFuncSetAttribute(render_backward_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Lay::kSmemBytes);
    if (e != cudaSuccess) return e;
    render_backward_kernel<C><<<grid_ctas, kBwdThreads, Lay::kSmemBytes, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_backward(const RenderArgs& A, const KernelShape& ks, int grid_ctas,
                            cudaStream_t stream)
{
#define PSDF_BWD_CASE(NA, L2, W, K)                                                          \
    if (ks.na == NA && ks.l2 == L2 && ks.width == W && ks.k == K)                            \
        return launch_backward_t<Cfg<NA, L2, W, K>>(A, grid_ctas, stream);
    PSDF_FOR_EACH_SHAPE(PSDF_BWD_CASE)
#undef PSDF_BWD_CASE
    return cudaErrorInvalidValue;
}

int backward_ctas_per_sm(const KernelShape& ks)
{
    int n = 0;
#define PSDF_BWD_OCC(NA, L2, W, K)                                                           \
    if (ks.na == NA && ks.l2 == L2 && ks.width == W && ks.k == K) {                          \
        using C_ = Cfg<NA, L2, W, K>;                                                        \
        cudaFuncSetAttribute(render_backward_kernel<C_>,                                     \
                             cudaFuncAttributeMaxDynamicSharedMemorySize,                    \
                             (int)BwdLayout<C_>::kSmemBytes);                                \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_backward_kernel<C_>,        \
                                                      kBwdThreads,                           \
                                                      BwdLayout<C_>::kSmemBytes);            \
    }
    PSDF_FOR_EACH_SHAPE(PSDF_BWD_OCC)
#undef PSDF_BWD_OCC
    return n;
}

}  // namespace psdf
