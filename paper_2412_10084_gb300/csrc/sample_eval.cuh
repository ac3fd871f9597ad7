// Per-sample colour evaluation shared by the forward and backward kernels:
// geometry (Sec. 3, Eq. 13), probe-blended SH angular features (Eqs. 5-7),
// Fresnel inputs (Eq. 4) and the colour MLP (Sec. 4), FP32 SIMT.
#pragma once

#include "render_common.cuh"

namespace psdf {

template <int NA_, int L2_, int W_, int K_>
struct Cfg {
    static constexpr int NS = 3;
    static constexpr int NA = NA_;
    static constexpr int L2 = L2_;
    static constexpr int W = W_;
    static constexpr int K = K_;
    static constexpr int NIN = NS + NA + K;
    static constexpr int NINP = (NIN + 3) & ~3;  // MLP input row, padded to float4
    static constexpr int NA4 = NA / 4;           // float4 groups per SH coefficient
    // MLP parameters in shared memory, rows padded to float4:
    //   W1 [W][NINP], b1 [W], W2 [W][W], b2 [W], W3T [W][4] (W3 transposed), b3 [4]
    static constexpr int kW1 = 0;
    static constexpr int kB1 = kW1 + W * NINP;
    static constexpr int kW2 = kB1 + W;
    static constexpr int kB2 = kW2 + W * W;
    static constexpr int kW3T = kB2 + W;
    static constexpr int kB3 = kW3T + 4 * W;
    static constexpr int kMlpSmem = kB3 + 4;  // floats
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

// Cooperative copy of the packed parameters into the padded smem layout.
template <class C>
__device__ __forceinline__ void load_mlp_smem(const float* __restrict__ g, float* s)
{
    for (int i = threadIdx.x; i < C::kMlpSmem; i += blockDim.x) {
        float v = 0.0f;
        if (i < C::kB1) {
            const int o = i / C::NINP, c = i % C::NINP;
            v = c < C::NIN ? g[C::gW1 + o * C::NIN + c] : 0.0f;
        } else if (i < C::kW2) {
            v = g[C::gB1 + (i - C::kB1)];
        } else if (i < C::kB2) {
            v = g[C::gW2 + (i - C::kW2)];
        } else if (i < C::kW3T) {
            v = g[C::gB2 + (i - C::kB2)];
        } else if (i < C::kB3) {
            const int o = (i - C::kW3T) / 4, c = (i - C::kW3T) % 4;
            v = c < 3 ? g[C::gW3 + c * C::W + o] : 0.0f;
        } else {
            const int c = i - C::kB3;
            v = c < 3 ? g[C::gB3 + c] : 0.0f;
        }
        s[i] = v;
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

template <class C>
__device__ __forceinline__ void eval_geometry(const RenderArgs& A, const float o[3],
                                              const float d[3], float t, SampleGeom<C>& S)
{
    float xw[3];
    point_at(o, d, t, xw);
    S.cell = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
    Corners k;
    gather_corners(A.grid, S.cell, k);
    float fs[3];
    sdf_full(A.grid, S.cell, k, S.s, S.g, fs);

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

    // Angular features (Eqs. 6-7): F_a = sum_i w_i sum_j b_ij Y_j(r).
    S.pcell = locate(xw, A.grid.bmin, A.probes.sc, A.probes.P);
    float wq[8];
    corner_weights(S.pcell.f, wq);
    int pidx[8];
    probe_corner_index(A.probes, S.pcell, pidx);
    float fa[C::NA];
#pragma unroll
    for (int c = 0; c < C::NA; ++c) fa[c] = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4* b = A.probes.coeffs + (size_t)pidx[q] * (C::L2 * C::NA4);
        float part[C::NA];
#pragma unroll
        for (int c = 0; c < C::NA; ++c) part[c] = 0.0f;
#pragma unroll
        for (int j = 0; j < C::L2; ++j) {
#pragma unroll
            for (int cg = 0; cg < C::NA4; ++cg) {
                const float4 bb = __ldg(b + j * C::NA4 + cg);
                part[4 * cg + 0] = fmaf(bb.x, S.Y[j], part[4 * cg + 0]);
                part[4 * cg + 1] = fmaf(bb.y, S.Y[j], part[4 * cg + 1]);
                part[4 * cg + 2] = fmaf(bb.z, S.Y[j], part[4 * cg + 2]);
                part[4 * cg + 3] = fmaf(bb.w, S.Y[j], part[4 * cg + 3]);
            }
        }
#pragma unroll
        for (int c = 0; c < C::NA; ++c) fa[c] = fmaf(wq[q], part[c], fa[c]);
    }

    S.x[0] = fs[0];
    S.x[1] = fs[1];
    S.x[2] = fs[2];
#pragma unroll
    for (int c = 0; c < C::NA; ++c) S.x[3 + c] = fa[c];
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

// Colour MLP (Sec. 4): n_in -> W -> W -> 3, ReLU, ReLU, sigmoid.  Weights are
// read from shared memory as warp-uniform float4 broadcasts.  If STORE, the
// input, h1 and h2 rows of this lane are written to shared memory for the
// weight-gradient pass.
template <class C, bool STORE>
__device__ __forceinline__ void mlp_forward(const float* __restrict__ sw, const float x[C::NINP],
                                            float col[3], float* xrow, float* h1row,
                                            float* h2row)
{
    float h1[C::W];
#pragma unroll
    for (int o = 0; o < C::W; ++o) {
        const float4* wr = reinterpret_cast<const float4*>(sw + C::kW1 + o * C::NINP);
        float z = sw[C::kB1 + o];
#pragma unroll
        for (int q = 0; q < C::NINP / 4; ++q) {
            const float4 w4 = wr[q];
            z = fmaf(w4.x, x[4 * q + 0], z);
            z = fmaf(w4.y, x[4 * q + 1], z);
            z = fmaf(w4.z, x[4 * q + 2], z);
            z = fmaf(w4.w, x[4 * q + 3], z);
        }
        h1[o] = fmaxf(z, 0.0f);
    }
    const float4 b3 = *reinterpret_cast<const float4*>(sw + C::kB3);
    float z3[3] = {b3.x, b3.y, b3.z};
#pragma unroll
    for (int o = 0; o < C::W; ++o) {
        const float4* wr = reinterpret_cast<const float4*>(sw + C::kW2 + o * C::W);
        float z = sw[C::kB2 + o];
#pragma unroll
        for (int q = 0; q < C::W / 4; ++q) {
            const float4 w4 = wr[q];
            z = fmaf(w4.x, h1[4 * q + 0], z);
            z = fmaf(w4.y, h1[4 * q + 1], z);
            z = fmaf(w4.z, h1[4 * q + 2], z);
            z = fmaf(w4.w, h1[4 * q + 3], z);
        }
        const float h2 = fmaxf(z, 0.0f);
        const float4 w3 = *reinterpret_cast<const float4*>(sw + C::kW3T + 4 * o);
        z3[0] = fmaf(w3.x, h2, z3[0]);
        z3[1] = fmaf(w3.y, h2, z3[1]);
        z3[2] = fmaf(w3.z, h2, z3[2]);
        if constexpr (STORE) h2row[o] = h2;
    }
    col[0] = sigmoidf(z3[0]);
    col[1] = sigmoidf(z3[1]);
    col[2] = sigmoidf(z3[2]);
    if constexpr (STORE) {
#pragma unroll
        for (int q = 0; q < C::NINP / 4; ++q)
            reinterpret_cast<float4*>(xrow)[q] =
                make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
#pragma unroll
        for (int q = 0; q < C::W / 4; ++q)
            reinterpret_cast<float4*>(h1row)[q] =
                make_float4(h1[4 * q], h1[4 * q + 1], h1[4 * q + 2], h1[4 * q + 3]);
    }
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
};

__device__ __forceinline__ RaySpan ray_span(const RenderArgs& A, const RayIn& R, int64_t ray)
{
    RaySpan sp;
    sp.tk = nullptr;
    sp.tn = 0.0f;
    sp.dt = 0.0f;
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

__device__ __forceinline__ float span_t(const RaySpan& sp, int k)
{
    return sp.tk ? __ldg(sp.tk + k) : sample_t(k, sp.dt, sp.tn);
}

}  // namespace psdf
