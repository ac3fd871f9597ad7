// Per-sample evaluation shared by the forward and backward kernels: geometry
// (Sec. 3, Eq. 13), probe-blended SH angular features (Eqs. 5-7) and Fresnel
// inputs (Eq. 4), FP32 on the CUDA cores; the MLP input row is their concatenation.
#pragma once

#include <cuda_fp16.h>

#include "render_common.cuh"

namespace psdf {

// Compile-time shape and storage precision of a render kernel.
//   FS: spatial-feature storage: 0 FP32 node records, 1 BF16 node features
//       (SDF stays FP32), 2 tile tri-planes (Sec. 3.1), 3 sparse bricks of
//       FP32 node records
//   PH: probe coefficients stored as FP16
//   MH: MLP on the tensor cores in plain FP16 (else the FP32-equivalent
//       hi/lo split)
template <int NA_, int L2_, int W_, int K_, int FS_ = 0, int PH_ = 0, int MH_ = 0>
struct Cfg {
    static constexpr int FB = FS_ == 1;
    static constexpr int TP = FS_ == 2;
    static constexpr int SP = FS_ == 3;
    static constexpr int PH = PH_;
    static constexpr int MH = MH_;
    static constexpr int NS = 3;
    static constexpr int NA = NA_;
    static constexpr int L2 = L2_;
    static constexpr int W = W_;
    static constexpr int K = K_;
    static constexpr int NIN = NS + NA + K;
    static constexpr int NINP = (NIN + 3) & ~3;  // MLP input row, padded to float4
    static constexpr int NA4 = NA / 4;           // float4 groups per SH coefficient
    // packed (global) parameter offsets: W1[W][NIN] b1 W2[W][W] b2 W3[3][W] b3[3]
    static constexpr int gW1 = 0;
    static constexpr int gB1 = W * NIN;
    static constexpr int gW2 = gB1 + W;
    static constexpr int gB2 = gW2 + W * W;
    static constexpr int gW3 = gB2 + W;
    static constexpr int gB3 = gW3 + 3 * W;
    static constexpr int kParams = gB3 + 3;
    static_assert(NA % 4 == 0, "angular channels are read as float4 groups");
    static_assert(W % 4 == 0, "hidden width must be a multiple of 4");
};

template <class C>
__device__ __forceinline__ void gather_corners_t(const GridView& g, const Cell& c, Corners& k)
{
    if constexpr (C::SP)
        gather_corners_sparse(g, c, k);
    else if constexpr (C::TP)
        gather_corners_sdf(g, c, k);
    else if constexpr (C::FB)
        gather_corners_bf16(g, c, k);
    else
        gather_corners(g, c, k);
}

// Channels [4 cg, 4 cg + 4) of SH coefficient j of probe `probe`.
template <class C>
__device__ __forceinline__ float4 probe_coeffs(const ProbeView& p, int probe, int j, int cg)
{
    const size_t i = (static_cast<size_t>(probe) * C::L2 + j) * C::NA4 + cg;
    if constexpr (C::PH) {
        const uint2 u = __ldg(p.coeffs16 + i);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    } else {
        return ldg_keep(p.coeffs + i);
    }
}

// Geometry and appearance inputs of one colour sample.
template <class C>
struct SampleGeom {
    Cell cell;       // SDF cell of the point
    float s;         // SDF value
    float g[3];      // trilinear gradient (world units)
    float rho;       // sqrt(|g|^2 + eps^2)
    float n[3];      // normal
    float ndv;       // n . v
    float r[3];      // SH lookup direction
    float Y[C::L2];  // SH basis at r
    Cell pcell;      // probe cell of the point
    float x[C::NINP];  // MLP input [F_s, F_a, fresnel, 0-pad]
};

// Probe corner offsets (in probes) of a probe cell.
__device__ __forceinline__ void probe_corner_index(const ProbeView& p, const Cell& pc, int idx[8])
{
    const int sx = 1, sy = p.P[0], sz = p.P[0] * p.P[1];
    idx[0] = pc.base;
    idx[1] = pc.base + sx;
    idx[2] = pc.base + sy;
    idx[3] = pc.base + sy + sx;
    idx[4] = pc.base + sz;
    idx[5] = pc.base + sz + sx;
    idx[6] = pc.base + sz + sy;
    idx[7] = pc.base + sz + sy + sx;
}

// SDF part of a sample: cell, trilinear SDF value and gradient, spatial
// features (MLP input columns 0..2).
template <class C>
__device__ __forceinline__ void eval_sdf(const RenderArgs& A, const float o[3], const float d[3],
                                         float t, SampleGeom<C>& S)
{
    float xw[3];
    point_at(o, d, t, xw);
    S.cell = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
    Corners k;
    float fs[3];
    if constexpr (C::SP) {
        if (gather_corners_sparse(A.grid, S.cell, k) == 0) {
            // every corner is empty space: s is the empty value exactly
            S.s = A.grid.empty_sdf;
            S.g[0] = S.g[1] = S.g[2] = 0.0f;
            S.x[0] = S.x[1] = S.x[2] = 0.0f;
            return;
        }
    } else {
        gather_corners_t<C>(A.grid, S.cell, k);
    }
    sdf_full(A.grid, S.cell, k, S.s, S.g, fs);
    if constexpr (C::TP) {
        TriAt T;
        triplane_locate(A.grid, xw, T);
        triplane_lookup(A.grid, T, fs);
    }
    S.x[0] = fs[0];
    S.x[1] = fs[1];
    S.x[2] = fs[2];
}

// Layouts that keep the spatial features apart from the SDF (the BF16 feature
// array, the tile tri-planes) gather the features only for the samples that
// need them: those with a nonzero opacity, known once the SDF is.
template <class C>
__device__ __forceinline__ constexpr bool features_apart()
{
    return C::FB || C::TP;
}

// eval_sdf without the spatial features (S.x[0..2] = 0): the cell, SDF value
// and gradient, from the 8 SDF values alone (the same bits as eval_sdf).
template <class C>
__device__ __forceinline__ void eval_sdf_geom(const RenderArgs& A, const float o[3],
                                              const float d[3], float t, SampleGeom<C>& S)
{
    static_assert(features_apart<C>(), "features stored apart from the SDF");
    float xw[3];
    point_at(o, d, t, xw);
    S.cell = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
    Corners k;
    gather_corners_sdf(A.grid, S.cell, k);
    float fs[3];
    sdf_full(A.grid, S.cell, k, S.s, S.g, fs);
    S.x[0] = S.x[1] = S.x[2] = 0.0f;
}

// The spatial features (MLP input columns 0..2) of the point at distance t,
// with the arithmetic of eval_sdf (so the same bits).
template <class C>
__device__ __forceinline__ void eval_features(const RenderArgs& A, const float o[3],
                                              const float d[3], float t, SampleGeom<C>& S)
{
    static_assert(features_apart<C>(), "features stored apart from the SDF");
    float xw[3];
    point_at(o, d, t, xw);
    float fs[3];
    if constexpr (C::TP) {
        TriAt T;
        triplane_locate(A.grid, xw, T);
        triplane_lookup(A.grid, T, fs);
    } else {
        const Cell c = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
        const int sx = 1, sy = A.grid.R[0], sz = A.grid.R[0] * A.grid.R[1];
        const int off[8] = {0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sy + sx};
        float w[8];
        corner_weights(c.f, w);
        fs[0] = fs[1] = fs[2] = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint2 f = __ldg(A.grid.feat16 + c.base + off[q]);
            fs[0] = fmaf(w[q], bf16_lo(f.x), fs[0]);
            fs[1] = fmaf(w[q], bf16_hi(f.x), fs[1]);
            fs[2] = fmaf(w[q], bf16_lo(f.y), fs[2]);
        }
    }
    S.x[0] = fs[0];
    S.x[1] = fs[1];
    S.x[2] = fs[2];
}

// Appearance part at world point xw seen along v (towards the viewer): normal
// (Eq. 13) from S.g, SH lookup direction and basis, probe-blended angular
// features (Eqs. 6-7) and Fresnel inputs (Eq. 4), the MLP input columns 3.. .
template <class C>
__device__ __forceinline__ void eval_appearance_at(const RenderArgs& A, const float xw[3],
                                                   const float v[3], SampleGeom<C>& S)
{
    const float gg = S.g[0] * S.g[0] + S.g[1] * S.g[1] + S.g[2] * S.g[2];
    S.rho = sqrtf(gg + kNormalEps * kNormalEps);
    const float inv = 1.0f / S.rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) S.n[a] = S.g[a] * inv;
    S.ndv = S.n[0] * v[0] + S.n[1] * v[1] + S.n[2] * v[2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        S.r[a] = A.dir_mode == 1 ? v[a] : 2.0f * S.ndv * S.n[a] - v[a];
    sh_basis<C::L2>(S.r, S.Y);

    // Angular features (Eqs. 6-7): F_a = sum_i w_i sum_j b_ij Y_j(r).
    S.pcell = locate(xw, A.grid.bmin, A.probes.sc, A.probes.P);
    float wq[8];
    corner_weights(S.pcell.f, wq);
    int pidx[8];
    probe_corner_index(A.probes, S.pcell, pidx);
    float2 fa[C::NA / 2];
#pragma unroll
    for (int c = 0; c < C::NA / 2; ++c) fa[c] = make_float2(0.0f, 0.0f);
    if constexpr (C::L2 * C::NA <= 36) {
        // blended coefficients b^_j = sum_i w_i b_ij first (one weight per
        // probe serves all of its coefficients), then F_a = sum_j Y_j b^_j
        float2 B2[C::L2 * C::NA / 2];
#pragma unroll
        for (int i = 0; i < C::L2 * C::NA / 2; ++i) B2[i] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float2 w2 = make_float2(wq[q], wq[q]);
#pragma unroll
            for (int j = 0; j < C::L2; ++j) {
#pragma unroll
                for (int cg = 0; cg < C::NA4; ++cg) {
                    const float4 bb = probe_coeffs<C>(A.probes, pidx[q], j, cg);
                    float2* b2 = B2 + (j * C::NA + 4 * cg) / 2;
                    b2[0] = fma2(w2, make_float2(bb.x, bb.y), b2[0]);
                    b2[1] = fma2(w2, make_float2(bb.z, bb.w), b2[1]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < C::L2; ++j) {
            const float2 y = make_float2(S.Y[j], S.Y[j]);
#pragma unroll
            for (int c = 0; c < C::NA / 2; ++c) fa[c] = fma2(y, B2[j * C::NA / 2 + c], fa[c]);
        }
    } else {
        // wide rows (more SH coefficients or channels): one probe at a time,
        // F_a += w_i sum_j b_ij Y_j, so only NA partial sums are live
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float2 part[C::NA / 2];
#pragma unroll
            for (int c = 0; c < C::NA / 2; ++c) part[c] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < C::L2; ++j) {
                const float2 y = make_float2(S.Y[j], S.Y[j]);
#pragma unroll
                for (int cg = 0; cg < C::NA4; ++cg) {
                    const float4 bb = probe_coeffs<C>(A.probes, pidx[q], j, cg);
                    part[2 * cg] = fma2(make_float2(bb.x, bb.y), y, part[2 * cg]);
                    part[2 * cg + 1] = fma2(make_float2(bb.z, bb.w), y, part[2 * cg + 1]);
                }
            }
            const float2 w2 = make_float2(wq[q], wq[q]);
#pragma unroll
            for (int c = 0; c < C::NA / 2; ++c) fa[c] = fma2(w2, part[c], fa[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < C::NA / 2; ++c) {
        S.x[3 + 2 * c] = fa[c].x;
        S.x[4 + 2 * c] = fa[c].y;
    }
    // Fresnel inputs (Eq. 4): (1 - n.v)^k, k = 1..K
    const float om = 1.0f - S.ndv;
    float pw = 1.0f;
#pragma unroll
    for (int kk = 0; kk < C::K; ++kk) {
        pw *= om;
        S.x[3 + C::NA + kk] = pw;
    }
#pragma unroll
    for (int i = C::NIN; i < C::NINP; ++i) S.x[i] = 0.0f;
}

// Appearance part of a ray sample (v = -d at o + t d).  Needed only where the
// sample's opacity is nonzero.
template <class C>
__device__ __forceinline__ void eval_appearance(const RenderArgs& A, const float o[3],
                                                const float d[3], float t, SampleGeom<C>& S)
{
    float xw[3], v[3];
    point_at(o, d, t, xw);
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = -d[a];
    eval_appearance_at<C>(A, xw, v, S);
}

// eval_appearance that also returns the blended probe coefficients
// Bc[j NA + c] = sum_i w_i b_ijc (Eq. 7 before the SH contraction), which the
// adjoint reuses for dF_a / dY_j = Bc_j . dF_a.
template <class C>
__device__ __forceinline__ void eval_appearance_blend(const RenderArgs& A, const float o[3],
                                                      const float d[3], float t,
                                                      SampleGeom<C>& S, float* Bc)
{
    const float gg = S.g[0] * S.g[0] + S.g[1] * S.g[1] + S.g[2] * S.g[2];
    S.rho = sqrtf(gg + kNormalEps * kNormalEps);
    const float inv = 1.0f / S.rho;
    float v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S.n[a] = S.g[a] * inv;
        v[a] = -d[a];
    }
    S.ndv = S.n[0] * v[0] + S.n[1] * v[1] + S.n[2] * v[2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        S.r[a] = A.dir_mode == 1 ? v[a] : 2.0f * S.ndv * S.n[a] - v[a];
    sh_basis<C::L2>(S.r, S.Y);

    float xw[3];
    point_at(o, d, t, xw);
    S.pcell = locate(xw, A.grid.bmin, A.probes.sc, A.probes.P);
    float wq[8];
    corner_weights(S.pcell.f, wq);
    int pidx[8];
    probe_corner_index(A.probes, S.pcell, pidx);
    // channel pairs of every coefficient accumulated as float2 (paired FMAs)
    float2 B2[C::L2 * C::NA / 2];
#pragma unroll
    for (int i = 0; i < C::L2 * C::NA / 2; ++i) B2[i] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float2 w2 = make_float2(wq[q], wq[q]);
#pragma unroll
        for (int j = 0; j < C::L2; ++j) {
#pragma unroll
            for (int cg = 0; cg < C::NA4; ++cg) {
                const float4 bb = probe_coeffs<C>(A.probes, pidx[q], j, cg);
                float2* b2 = B2 + (j * C::NA + 4 * cg) / 2;
                b2[0] = fma2(w2, make_float2(bb.x, bb.y), b2[0]);
                b2[1] = fma2(w2, make_float2(bb.z, bb.w), b2[1]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < C::L2 * C::NA / 2; ++i) {
        Bc[2 * i] = B2[i].x;
        Bc[2 * i + 1] = B2[i].y;
    }
#pragma unroll
    for (int c = 0; c < C::NA; ++c) {
        float fa = 0.0f;
#pragma unroll
        for (int j = 0; j < C::L2; ++j) fa = fmaf(S.Y[j], Bc[j * C::NA + c], fa);
        S.x[3 + c] = fa;
    }
    const float om = 1.0f - S.ndv;
    float pw = 1.0f;
#pragma unroll
    for (int kk = 0; kk < C::K; ++kk) {
        pw *= om;
        S.x[3 + C::NA + kk] = pw;
    }
#pragma unroll
    for (int i = C::NIN; i < C::NINP; ++i) S.x[i] = 0.0f;
}

// MLP input of a sample whose opacity is zero: its colour is never used
// (every term it enters is multiplied by alpha = 0), so the appearance
// columns are left at zero.
template <class C>
__device__ __forceinline__ void zero_appearance(SampleGeom<C>& S)
{
#pragma unroll
    for (int i = 3; i < C::NINP; ++i) S.x[i] = 0.0f;
}

template <class C>
__device__ __forceinline__ void eval_geometry(const RenderArgs& A, const float o[3],
                                              const float d[3], float t, SampleGeom<C>& S)
{
    eval_sdf<C>(A, o, d, t, S);
    eval_appearance<C>(A, o, d, t, S);
}

// Ray record (broadcast by every lane of the warp).
struct RayIn {
    float o[3], d[3];
};

__device__ __forceinline__ RayIn load_ray(const RenderArgs& A, int64_t ray)
{
    RayIn R;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.o[a] = __ldg(A.rays_o + 3 * ray + a);
        R.d[a] = __ldg(A.rays_d + 3 * ray + a);
    }
    return R;
}

// Sample distances of a ray: uniform over the box segment, or given.
struct RaySpan {
    bool hit;
    float tn, dt;
    const float* tk;  // given distances or nullptr
    // placement at the quantiles k / N of per-bin densities (n_bins > 0): the
    // warp's shared-memory table holds the running sums c_b = q_0 + .. + q_{b-1}
    // at [0, 32) and 1 / q_b at [32, 64); dt is then the bin width
    int n_bins, n;
    float tf, inv_n;
    const float* tab;
};

// tab: this warp's 64-float shared-memory table (used in the bin-density
// mode).  Warp-uniform: every lane of the warp calls it for the warp's ray.
__device__ __forceinline__ RaySpan ray_span(const RenderArgs& A, const RayIn& R, int64_t ray,
                                            float* tab)
{
    RaySpan sp;
    sp.tk = nullptr;
    sp.tn = 0.0f;
    sp.tf = 0.0f;
    sp.dt = 0.0f;
    sp.n_bins = 0;
    sp.n = A.n_samples;
    sp.inv_n = 0.0f;
    sp.tab = tab;
    if (A.t_samples && A.n_bins > 0) {
        const int lane = threadIdx.x & 31;
        float tf;
        sp.hit = ray_box(R.o, R.d, A.grid, sp.tn, tf);
        sp.tf = tf;
        sp.n_bins = A.n_bins;
        const float q = lane < A.n_bins ? __ldg(A.t_samples + ray * (int64_t)A.n_bins + lane) : 0.0f;
        float c = 0.0f;
        for (int i = 0; i < A.n_bins; ++i) {  // running sums in bin order
            const float qi = __shfl_sync(0xffffffffu, q, i);
            if (i < lane) c += qi;
        }
        __syncwarp();  // the previous ray's readers are done with the table
        tab[lane] = c;
        tab[32 + lane] = lane < A.n_bins ? 1.0f / q : 0.0f;
        __syncwarp();
        sp.dt = (tf - sp.tn) / A.n_bins;
        sp.inv_n = 1.0f / A.n_samples;
        return sp;
    }
    if (A.t_samples) {
        sp.tk = A.t_samples + ray * (int64_t)(A.n_samples + 1);
        sp.hit = __ldg(sp.tk + A.n_samples) > __ldg(sp.tk);
        return sp;
    }
    float tf;
    sp.hit = ray_box(R.o, R.d, A.grid, sp.tn, tf);
    if (sp.hit) sp.dt = __fdiv_rn(__fsub_rn(tf, sp.tn), static_cast<float>(A.n_samples));
    return sp;
}

// Distance of sample k (0..N).
__device__ __forceinline__ float span_t(const RaySpan& sp, int k)
{
    if (sp.n_bins > 0) {
        // the sample's bin is the last with c_b <= u (binary search over the
        // running sums), then t = t_n + (b + (u - c_b) / q_b) width, with the
        // reciprocals rounded once per ray (the proposal kernel uses the same
        // expressions, so both place samples at the same FP32 distances)
        const float u = static_cast<float>(k) * sp.inv_n;
        int b = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int j = b + step;
            if (j < sp.n_bins && sp.tab[j] <= u) b = j;
        }
        const float frac = fminf((u - sp.tab[b]) * sp.tab[32 + b], 1.0f);
        return k == 0 ? sp.tn : (k == sp.n ? sp.tf : fmaf(b + frac, sp.dt, sp.tn));
    }
    return sp.tk ? __ldg(sp.tk + k) : sample_t(k, sp.dt, sp.tn);
}

}  // namespace psdf
