// Grid-level training terms of ProbeSDF (Sec. 3.3, Eqs. 11-15).
//
//   smooth_kernel<false>  s = G(s_hat): 5^3 Gaussian (sigma = 1 node, separable,
//                         replicated edge nodes); one shared-memory tile pass
//                         (32 x 8 x 8 outputs, 2-node halo) per CTA
//   smooth_kernel<true>   G^T: the same tiles with the transposed 1D operators,
//                         applied z, y, x (edge outputs gather the replicated taps)
//   sparse_smooth_kernel  both on sparse 16^3-node bricks: one CTA per stored
//                         brick, its 16^3 nodes plus a 2-node halo gathered
//                         through the brick table into a 20^3 tile
//   sdf_reg_kernel        L_sdf, L_Eik and L_normal on the smoothed SDF, their
//                         gradients scaled by (1 + 5 |s|)^-1: a z-streaming
//                         stencil whose central-difference adjoint is a gather
//   plane_reg_kernel      L_features: forward differences inside each tile plane
//   probe_reg_kernel      L_probes: ordered pairs of 6-neighbour probes
//
// Streaming stencils over HBM-resident grids; loss values are summed per CTA
// and added to device accumulators.
#include <cmath>

#include "internal.h"

namespace psdf {

namespace {

constexpr int TX = 32, TY = 8, TZ = 8, HALO = 2;
constexpr int AX = TX + 2 * HALO, AY = TY + 2 * HALO, AZ = TZ + 2 * HALO;
constexpr int kBufA = AZ * AY * AX;  // 5184 floats
constexpr int kBufB = AZ * AY * TX;  // 4608 floats (>= TZ * AY * AX = 3456)
constexpr int kSmoothThreads = 256;

struct Taps {
    float w[5];
};

__device__ __forceinline__ int clampi(int v, int lo, int hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// Transposed 1D pass at output node k of an axis of n nodes; p[j * st] holds
// input node k - 2 + j (0 outside the grid).  Inside the axis, output k takes
// input i with the weight w[k - i + 2] that the forward gave input k in output
// i; the replicated edge taps add (w0 + w1) x in[0] + w0 x in[1] at k = 0 and
// (w3 + w4) x in[n-1] + w4 x in[n-2] at k = n - 1.
__device__ __forceinline__ float tconv(const float* p, int st, int k, int n, const Taps& T)
{
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < 5; ++j) acc = fmaf(T.w[4 - j], p[j * st], acc);
    if (k == 0) acc = fmaf(T.w[0] + T.w[1], p[2 * st], fmaf(T.w[0], p[3 * st], acc));
    if (k == n - 1) acc = fmaf(T.w[3] + T.w[4], p[2 * st], fmaf(T.w[4], p[st], acc));
    return acc;
}

// Work is laid out in rows along x: warp w takes rows w, w + 8, ..., lane =
// x (a 36-wide halo row takes a second slot on lanes 0..3), so no element
// index is ever divided or reduced modulo a tile size.
constexpr int kSmoothWarps = kSmoothThreads / 32;

template <bool TRANSPOSE>
__global__ void __launch_bounds__(kSmoothThreads) smooth_kernel(const float* __restrict__ in,
                                                                 int in_stride,
                                                                 float* __restrict__ out,
                                                                 int out_stride, int Rx, int Ry,
                                                                 int Rz, Taps T, int accumulate)
{
    __shared__ float A[kBufA];
    __shared__ float B[kBufB];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- tile + halo, rows (az, ay) of AX nodes: forward reads replicate the
    // edge nodes; the transposed operator has no input outside the grid ----
    {
        const int gx0 = x0 - HALO + lane, gx1 = x0 - HALO + 32 + lane;
        const bool in0 = gx0 >= 0 && gx0 < Rx, in1 = lane < AX - 32 && gx1 >= 0 && gx1 < Rx;
        const int cx0 = clampi(gx0, 0, Rx - 1), cx1 = clampi(gx1, 0, Rx - 1);
        constexpr int kRows = AZ * AY / kSmoothWarps;  // 18
        constexpr int kBatch = 6;
#pragma unroll 1
        for (int i0 = 0; i0 < kRows; i0 += kBatch) {
            float v0[kBatch], v1[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                const int r = warp + kSmoothWarps * (i0 + i);
                const int ay = r % AY, az = r / AY;
                const int gy = y0 + ay - HALO, gz = z0 + az - HALO;
                v0[i] = v1[i] = 0.0f;
                if (!TRANSPOSE) {
                    const size_t row =
                        ((size_t)clampi(gz, 0, Rz - 1) * Ry + clampi(gy, 0, Ry - 1)) * Rx;
                    v0[i] = __ldg(in + (row + cx0) * in_stride);
                    if (lane < AX - 32) v1[i] = __ldg(in + (row + cx1) * in_stride);
                } else if (gy >= 0 && gy < Ry && gz >= 0 && gz < Rz) {
                    const size_t row = ((size_t)gz * Ry + gy) * Rx;
                    if (in0) v0[i] = __ldg(in + (row + gx0) * in_stride);
                    if (in1) v1[i] = __ldg(in + (row + gx1) * in_stride);
                }
            }
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                const int r = warp + kSmoothWarps * (i0 + i);
                A[r * AX + lane] = v0[i];
                if (lane < AX - 32) A[r * AX + 32 + lane] = v1[i];
            }
        }
    }
    __syncthreads();
    if (!TRANSPOSE) {
        // x: A[AZ][AY][AX] -> B[AZ][AY][TX]
        for (int r = warp; r < AZ * AY; r += kSmoothWarps) {
            const float* a = A + r * AX + lane;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], a[j], acc);
            B[r * TX + lane] = acc;
        }
        __syncthreads();
        // y: B[AZ][AY][TX] -> A[AZ][TY][TX]
        for (int r = warp; r < AZ * TY; r += kSmoothWarps) {
            const int y = r % TY, az = r / TY;
            const float* b = B + (az * AY + y) * TX + lane;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], b[j * TX], acc);
            A[r * TX + lane] = acc;
        }
        __syncthreads();
        // z: A[AZ][TY][TX] -> output
        const int gx = x0 + lane;
        for (int r = warp; r < TZ * TY; r += kSmoothWarps) {
            const int y = r % TY, z = r / TY;
            const int gy = y0 + y, gz = z0 + z;
            if (gx >= Rx || gy >= Ry || gz >= Rz) continue;
            const float* a = A + r * TX + lane;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], a[j * TY * TX], acc);
            float* o = out + (((size_t)gz * Ry + gy) * Rx + gx) * out_stride;
            *o = accumulate ? *o + acc : acc;
        }
    } else {
        // G^T = Gx^T Gy^T Gz^T, applied z, y, x with tconv (zeros outside the
        // grid, as loaded)
        // z: A[AZ][AY][AX] -> B[TZ][AY][AX]
        for (int r = warp; r < TZ * AY; r += kSmoothWarps) {
            const int z = r / AY;
            const float* a = A + r * AX + lane;  // rows (z, ay) of A start the tap column
            B[r * AX + lane] = tconv(a, AY * AX, z0 + z, Rz, T);
            if (lane < AX - 32) B[r * AX + 32 + lane] = tconv(a + 32, AY * AX, z0 + z, Rz, T);
        }
        __syncthreads();
        // y: B[TZ][AY][AX] -> A[TZ][TY][AX]
        for (int r = warp; r < TZ * TY; r += kSmoothWarps) {
            const int y = r % TY, z = r / TY;
            const float* b = B + (z * AY + y) * AX + lane;
            A[r * AX + lane] = tconv(b, AX, y0 + y, Ry, T);
            if (lane < AX - 32) A[r * AX + 32 + lane] = tconv(b + 32, AX, y0 + y, Ry, T);
        }
        __syncthreads();
        // x: A[TZ][TY][AX] -> output
        const int gx = x0 + lane;
        for (int r = warp; r < TZ * TY; r += kSmoothWarps) {
            const int y = r % TY, z = r / TY;
            const int gy = y0 + y, gz = z0 + z;
            if (gx >= Rx || gy >= Ry || gz >= Rz) continue;
            const float acc = tconv(A + r * AX + lane, 1, gx, Rx, T);
            float* o = out + (((size_t)gz * Ry + gy) * Rx + gx) * out_stride;
            *o = accumulate ? *o + acc : acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Sparse bricks.  The grid is the full R^3 grid in which every node of a
// brick that is not stored holds `empty` (forward: s_hat = s = empty_sdf
// there); G and G^T are those of the full grid, evaluated at the stored nodes
// only.  The transposed pass has no input at absent nodes (their s is fixed,
// so they carry no gradient) nor outside the grid.  One CTA per table entry;
// absent entries return at once.
// ---------------------------------------------------------------------------

constexpr int SB = 16, SA = SB + 2 * HALO;  // brick edge, tile edge (20)
constexpr int kSpTile = SA * SA * SA;       // 8000 floats
constexpr int kSpPass = SA * SA * SB;       // 6400 floats
constexpr int kSpThreads = 256;
constexpr int kSpBytes = static_cast<int>(sizeof(float)) * (kSpTile + kSpPass);

struct SparseSmooth {
    const int* table;  // [B2][B1][B0]: slot, or -1 (outside [0, n_bricks) counts as absent)
    int B[3], R[3], n_bricks;
    const float* in;   // node `local` of slot b at in[in_base + (b * 4096 + local) * in_stride]
    int64_t in_base;
    int in_stride;
    float* out;        // likewise
    int64_t out_base;
    int out_stride;
    float empty;       // forward: the value of a node of an absent brick
    int accumulate;
};

__device__ __forceinline__ int sparse_slot(const SparseSmooth& P, int bx, int by, int bz)
{
    const int s = __ldg(P.table + (int64_t(bz) * P.B[1] + by) * P.B[0] + bx);
    return s >= 0 && s < P.n_bricks ? s : -1;
}

template <bool TRANSPOSE>
__global__ void __launch_bounds__(kSpThreads) sparse_smooth_kernel(SparseSmooth P, Taps T)
{
    extern __shared__ float sp_smem[];
    float* A = sp_smem;            // tile [SA][SA][SA] (z, y, x), later the y pass
    float* Bp = sp_smem + kSpTile; // x pass [SA][SA][SB]
    __shared__ int nb[27];         // slots of the brick and its 26 neighbours
    const int e = blockIdx.x;
    const int bx = e % P.B[0], by = (e / P.B[0]) % P.B[1], bz = e / (P.B[0] * P.B[1]);
    const int slot = sparse_slot(P, bx, by, bz);
    if (slot < 0) return;  // CTA-uniform
    const int tid = threadIdx.x;
    if (tid < 27) {
        const int nx = bx + tid % 3 - 1, ny = by + (tid / 3) % 3 - 1, nz = bz + tid / 9 - 1;
        const bool in_grid = nx >= 0 && nx < P.B[0] && ny >= 0 && ny < P.B[1] && nz >= 0 &&
                             nz < P.B[2];
        nb[tid] = in_grid ? sparse_slot(P, nx, ny, nz) : -1;
    }
    __syncthreads();
    // ---- tile: node g = 16 b - 2 + l.  Forward: the replicated edge node
    // outside the grid, `empty` in an absent brick.  Transposed: 0 for both ----
    const int g0[3] = {bx * SB - HALO, by * SB - HALO, bz * SB - HALO};
    const int b0[3] = {bx, by, bz};
    for (int i = tid; i < kSpTile; i += kSpThreads) {
        const int l[3] = {i % SA, (i / SA) % SA, i / (SA * SA)};
        int g[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g[a] = g0[a] + l[a];
            inside = inside && g[a] >= 0 && g[a] < P.R[a];
            g[a] = clampi(g[a], 0, P.R[a] - 1);
        }
        float v = TRANSPOSE ? 0.0f : P.empty;
        if (!TRANSPOSE || inside) {
            // the clamped node lies in this brick or a face / edge / corner neighbour
            const int q = ((g[2] >> 4) - b0[2] + 1) * 9 + ((g[1] >> 4) - b0[1] + 1) * 3 +
                          ((g[0] >> 4) - b0[0] + 1);
            const int s = nb[q];
            if (s >= 0) {
                const int local = ((g[2] & 15) << 8) | ((g[1] & 15) << 4) | (g[0] & 15);
                v = __ldg(P.in + P.in_base + (int64_t(s) * 4096 + local) * P.in_stride);
            }
        }
        A[i] = v;
    }
    __syncthreads();
    // ---- x: A[SA][SA][SA] -> Bp[SA][SA][SB] ----
    for (int i = tid; i < kSpPass; i += kSpThreads) {
        const int x = i % SB, r = i / SB;
        const float* a = A + r * SA + x;
        float acc = 0.0f;
        if (TRANSPOSE) {
            acc = tconv(a, 1, bx * SB + x, P.R[0], T);
        } else {
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], a[j], acc);
        }
        Bp[i] = acc;
    }
    __syncthreads();
    // ---- y: Bp[SA][SA][SB] -> A[SA][SB][SB] ----
    for (int i = tid; i < SA * SB * SB; i += kSpThreads) {
        const int x = i % SB, y = (i / SB) % SB, z = i / (SB * SB);
        const float* b = Bp + (z * SA + y) * SB + x;
        float acc = 0.0f;
        if (TRANSPOSE) {
            acc = tconv(b, SB, by * SB + y, P.R[1], T);
        } else {
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], b[j * SB], acc);
        }
        A[i] = acc;
    }
    __syncthreads();
    // ---- z: A[SA][SB][SB] -> the brick's 16^3 outputs ----
    for (int i = tid; i < SB * SB * SB; i += kSpThreads) {
        const float* a = A + i;
        float acc = 0.0f;
        if (TRANSPOSE) {
            acc = tconv(a, SB * SB, bz * SB + (i >> 8), P.R[2], T);
        } else {
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], a[j * SB * SB], acc);
        }
        float* o = P.out + P.out_base + (int64_t(slot) * 4096 + i) * P.out_stride;
        *o = P.accumulate ? *o + acc : acc;
    }
}

// Block sum of up to three loss partials, added to acc[0..n-1] (skipped when acc is null).
__device__ __forceinline__ void block_loss(float a, float b, float c, float* acc, int n)
{
    __shared__ float part[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    if (lane == 0) {
        part[0][warp] = a;
        part[1][warp] = b;
        part[2][warp] = c;
    }
    __syncthreads();
    if (acc && threadIdx.x < n) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[threadIdx.x][w];
        atomicAdd(acc + threadIdx.x, s);
    }
    __syncthreads();
}

struct SdfReg {
    const float* s_hat;  // dense [R^3], or sparse [n_bricks][16^3] in slot order
    const float* s;      // smoothed, element stride s_stride (sparse: the brick records)
    int s_stride;
    float* d_s;          // gradient w.r.t. s (accumulated), stride d_stride
    int d_stride;
    float* d_s_hat;      // gradient w.r.t. s_hat (accumulated), laid out as s_hat
    float* loss;         // [3]: L_sdf, L_Eik, L_normal (accumulated)
    int R[3];
    float inv2h[3];      // 1 / (2 h_a)
    float lam_sdf, lam_eik, lam_normal;
    // sparse 16^3-node bricks: brick table [B2][B1][B0] (slot, or -1; a slot
    // outside [0, n_bricks) counts as absent); node `local` of slot b is
    // element b * 4096 + local of every array above; absent nodes read `empty`
    const int* table;
    int B[3], n_bricks;
    float empty;
};

// z-streaming stencil.  A CTA owns an RX x RY column tile and ZC output planes
// and walks z with three shared-memory rings of 3 planes each:
//   s  (halo 3)  the smoothed SDF,
//   N  (halo 2)  normal n, voxel weight w, rho = sqrt(|g|^2 + eps^2) (0 marks a
//                node that is not interior), |g|,
//   G  (halo 1)  dg = dObjective/d(grad s) of the node's Eikonal and normal
//                terms.
// Step t loads s plane zs, computes N at zs - 1, G at zs - 2 and the outputs
// at zs - 3: ds_i = own L_sdf term + sum_a (dg_a(i - e_a) - dg_a(i + e_a)) / 2h_a
// (the central-difference adjoint as a gather), so every output has one
// writer and no atomics are needed.
//
// Dense grids: 32 x 8 columns, 32 planes per CTA.  Sparse bricks: one CTA per
// brick-table entry (absent entries return at once), 16 x 16 columns and the
// brick's 16 planes; s is that of the full grid with every node of an absent
// brick at `empty` (as the render and the smoothing read it), and the terms
// are those of the stored nodes: an absent node gets voxel weight 0, so its
// own Eikonal term and the normal pairs it owns add nothing, while its
// normal still enters the pairs its stored neighbours own.  Gradients are
// written for the stored nodes only (an absent node's s is not a parameter).
template <int RX_, int RY_, int ZC_>
struct RegTile {
    static constexpr int RX = RX_, RY = RY_, ZC = ZC_;
    static constexpr int SX = RX + 6, SY = RY + 6;
    static constexpr int NX = RX + 4, NY = RY + 4;
    static constexpr int GX = RX + 2, GY = RY + 2;
    static constexpr int kThreads = RX * RY;
    struct Smem {
        float s[3][SY * SX];
        float n[3][6][NY * NX];  // n.x n.y n.z w rho |g|
        float g[3][3][GY * GX];  // dg
    };
};
using DenseReg = RegTile<32, 8, 32>;
using SparseReg = RegTile<16, 16, 16>;
constexpr int kRegThreads = 256;
static_assert(DenseReg::kThreads == kRegThreads && SparseReg::kThreads == kRegThreads, "");

template <class T, bool SPARSE>
__global__ void __launch_bounds__(kRegThreads) sdf_reg_kernel(SdfReg P)
{
    constexpr int RX = T::RX, RY = T::RY, ZC = T::ZC;
    constexpr int SX = T::SX, SY = T::SY, NX = T::NX, NY = T::NY, GX = T::GX, GY = T::GY;
    extern __shared__ __align__(16) float reg_smem[];
    typename T::Smem& S = *reinterpret_cast<typename T::Smem*>(reg_smem);
    __shared__ int nb[27];  // sparse: slots of the brick and its 26 neighbours
    const int tid = threadIdx.x;
    const int Rx = P.R[0], Ry = P.R[1], Rz = P.R[2];
    int x0, y0, z0, slot = 0;
    if constexpr (SPARSE) {
        const int e = blockIdx.x;
        const int bx = e % P.B[0], by = (e / P.B[0]) % P.B[1], bz = e / (P.B[0] * P.B[1]);
        const int sv = __ldg(P.table + e);
        if (sv < 0 || sv >= P.n_bricks) return;  // CTA-uniform
        slot = sv;
        if (tid < 27) {
            const int nx = bx + tid % 3 - 1, ny = by + (tid / 3) % 3 - 1, nz = bz + tid / 9 - 1;
            int q = -1;
            if (nx >= 0 && nx < P.B[0] && ny >= 0 && ny < P.B[1] && nz >= 0 && nz < P.B[2]) {
                q = __ldg(P.table + (int64_t(nz) * P.B[1] + ny) * P.B[0] + nx);
                if (q >= P.n_bricks) q = -1;
            }
            nb[tid] = q < 0 ? -1 : q;
        }
        __syncthreads();
        x0 = bx * RX;
        y0 = by * RY;
        z0 = bz * ZC;
    } else {
        x0 = blockIdx.x * RX;
        y0 = blockIdx.y * RY;
        z0 = blockIdx.z * ZC;
    }
    const int z1 = min(z0 + ZC, Rz);
    const float cn = 2.0f * P.lam_normal;
    const size_t plane = (size_t)Ry * Rx;
    float l_sdf = 0.0f, l_eik = 0.0f, l_nrm = 0.0f;
    // sparse: element of in-grid node (x, y, z) in the arrays, or -1 if its
    // brick is not stored (the node then lies in this brick or a neighbour)
    auto sparse_elem = [&](int x, int y, int z) -> int64_t {
        const int q = ((z >> 4) - (z0 >> 4) + 1) * 9 + ((y >> 4) - (y0 >> 4) + 1) * 3 +
                      ((x >> 4) - (x0 >> 4) + 1);
        const int b = nb[q];
        return b < 0 ? -1 : int64_t(b) * 4096 + (((z & 15) << 8) | ((y & 15) << 4) | (x & 15));
    };

    // A thread's elements of each plane are the same at every step: their
    // (x, y) offsets and in-grid tests are computed once.
    constexpr int kPerS = (SY * SX + kRegThreads - 1) / kRegThreads;
    constexpr int kPerN = (NY * NX + kRegThreads - 1) / kRegThreads;
    constexpr int kPerG = (GY * GX + kRegThreads - 1) / kRegThreads;
    size_t s_xy[kPerS];
    bool s_in[kPerS];
    int s_x[kPerS], s_y[kPerS];
#pragma unroll
    for (int k = 0; k < kPerS; ++k) {
        const int e = tid + k * kRegThreads;
        const int x = x0 - 3 + e % SX, y = y0 - 3 + e / SX;
        s_in[k] = e < SY * SX && x >= 0 && x < Rx && y >= 0 && y < Ry;
        s_xy[k] = s_in[k] ? (size_t)y * Rx + x : 0;
        s_x[k] = x;
        s_y[k] = y;
    }
    int n_c[kPerN], n_x[kPerN], n_y[kPerN];
    bool n_ok[kPerN], n_xy[kPerN];
#pragma unroll
    for (int k = 0; k < kPerN; ++k) {
        const int e = tid + k * kRegThreads;
        const int nx = e % NX, ny = e / NX, x = x0 - 2 + nx, y = y0 - 2 + ny;
        n_ok[k] = e < NY * NX;
        n_c[k] = (ny + 1) * SX + nx + 1;  // the node in the s planes
        n_xy[k] = x > 0 && y > 0 && x < Rx - 1 && y < Ry - 1;
        n_x[k] = x;
        n_y[k] = y;
    }
    int g_c[kPerG];
    bool g_ok[kPerG], g_xy[kPerG];
#pragma unroll
    for (int k = 0; k < kPerG; ++k) {
        const int e = tid + k * kRegThreads;
        const int gx = e % GX, gy = e / GX, x = x0 - 1 + gx, y = y0 - 1 + gy;
        g_ok[k] = e < GY * GX;
        g_c[k] = (gy + 1) * NX + gx + 1;  // the node in the N planes
        g_xy[k] = x >= x0 && x < x0 + RX && y >= y0 && y < y0 + RY;  // owned in x, y
    }

    // s plane loads are software-pipelined: the values of plane zs + 1 are in
    // flight while plane zs is processed
    float pre[kPerS];
    auto load_plane = [&](int z) {
        const bool zin = z >= 0 && z < Rz;
#pragma unroll
        for (int k = 0; k < kPerS; ++k) {
            if constexpr (SPARSE) {
                float v = 0.0f;
                if (zin && s_in[k]) {
                    const int64_t el = sparse_elem(s_x[k], s_y[k], z);
                    v = el < 0 ? P.empty : __ldg(P.s + el * P.s_stride);
                }
                pre[k] = v;
            } else {
                pre[k] = (zin && s_in[k])
                             ? __ldg(P.s + ((size_t)z * plane + s_xy[k]) * P.s_stride)
                             : 0.0f;
            }
        }
    };
    load_plane(z0 - 3);
    const int ox = tid % RX, oy = tid / RX;
    const int x_o = x0 + ox, y_o = y0 + oy;
    const int c_o = (oy + 1) * GX + ox + 1;  // the output node in the G planes
    // ring slots of the planes of two steps back (ra), one step back (rb) and
    // this step (rc): s holds zs, zs - 1, zs - 2; N holds zs - 1 .. zs - 3; G
    // holds zs - 2 .. zs - 4
    int ra = 0, rb = 1, rc = 2;
    for (int zs = z0 - 3; zs <= z1 + 2; ++zs) {
        // ---- s plane zs (zeros outside the grid), then the next plane's loads ----
#pragma unroll
        for (int k = 0; k < kPerS; ++k) {
            const int e = tid + k * kRegThreads;
            if (e < SY * SX) S.s[rc][e] = pre[k];
        }
        if (zs + 1 <= z1 + 2) load_plane(zs + 1);
        // the output node's own values, consumed after the G stage
        const int zo = zs - 3;
        const bool out = zo >= z0 && zo < z1 && x_o < Rx && y_o < Ry;
        size_t io = 0;
        float s_o = 0.f, sh_o = 0.f, ds_o = 0.f, dsh_o = 0.f;
        if (out) {
            if constexpr (SPARSE)
                io = size_t(slot) * 4096 + (((zo & 15) << 8) | ((y_o & 15) << 4) | (x_o & 15));
            else
                io = (size_t)zo * plane + (size_t)y_o * Rx + x_o;
            s_o = __ldg(P.s + io * P.s_stride);
            sh_o = __ldg(P.s_hat + io);
            ds_o = P.d_s[io * P.d_stride];
            dsh_o = P.d_s_hat[io];
        }
        __syncthreads();
        // ---- N plane zn = zs - 1: gradient, normal, weight at interior nodes ----
        // (the outputs need N at z0 - 2 .. z1 + 1 and G at z0 - 1 .. z1)
        if (zs - 1 >= z0 - 2) {
            const int zn = zs - 1;
            const float* sm = S.s[ra];
            const float* sc = S.s[rb];
            const float* sp = S.s[rc];
            const bool zin = zn > 0 && zn < Rz - 1;
#pragma unroll
            for (int k = 0; k < kPerN; ++k) {
                if (!n_ok[k]) continue;
                const int e = tid + k * kRegThreads;
                const int c = n_c[k];
                float n0 = 0.f, n1 = 0.f, n2 = 0.f, w = 0.f, rho = 0.f, gn = 0.f;
                if (zin && n_xy[k]) {
                    const float g0 = (sc[c + 1] - sc[c - 1]) * P.inv2h[0];
                    const float g1 = (sc[c + SX] - sc[c - SX]) * P.inv2h[1];
                    const float g2 = (sp[c] - sm[c]) * P.inv2h[2];
                    const float gg = g0 * g0 + g1 * g1 + g2 * g2;
                    rho = sqrtf(gg + 1e-24f);
                    const float ir = 1.0f / rho;
                    n0 = g0 * ir;
                    n1 = g1 * ir;
                    n2 = g2 * ir;
                    gn = sqrtf(gg);
                    w = 1.0f / (1.0f + 5.0f * fabsf(sc[c]));
                    if constexpr (SPARSE)
                        if (sparse_elem(n_x[k], n_y[k], zn) < 0) w = 0.0f;  // no terms of its own
                }
                S.n[rc][0][e] = n0;
                S.n[rc][1][e] = n1;
                S.n[rc][2][e] = n2;
                S.n[rc][3][e] = w;
                S.n[rc][4][e] = rho;
                S.n[rc][5][e] = gn;
            }
        }
        __syncthreads();
        // ---- G plane zg = zs - 2: Eikonal and normal adjoints w.r.t. grad s ----
        if (zs - 2 >= z0 - 1) {
            const int zg = zs - 2;
            const bool zown = zg >= z0 && zg < z1;
#pragma unroll
            for (int k = 0; k < kPerG; ++k) {
                if (!g_ok[k]) continue;
                const int e = tid + k * kRegThreads;
                const int c = g_c[k];
                const float rho = S.n[rb][4][c];
                float d0 = 0.f, d1 = 0.f, d2 = 0.f;
                if (rho > 0.0f) {
                    const bool own = zown && g_xy[k];
                    const float n0 = S.n[rb][0][c], n1 = S.n[rb][1][c], n2 = S.n[rb][2][c];
                    const float w = S.n[rb][3][c], gn = S.n[rb][5][c];
                    // Eq. 12
                    const float ee = gn - 1.0f;
                    if (own) l_eik += ee * ee;
                    const float ce = gn > 0.0f ? P.lam_eik * w * 2.0f * ee / gn : 0.0f;
                    // Eq. 13: pairs (j, j + e_a) owned by j, (j - e_a, j) owned by the neighbour
                    float dn0 = 0.f, dn1 = 0.f, dn2 = 0.f;
                    const int pr[3] = {rb, rb, rc}, po[3] = {c + 1, c + NX, c};
                    const int mr[3] = {rb, rb, ra}, mo[3] = {c - 1, c - NX, c};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (S.n[pr[a]][4][po[a]] > 0.0f) {
                            const float q0 = S.n[pr[a]][0][po[a]] - n0;
                            const float q1 = S.n[pr[a]][1][po[a]] - n1;
                            const float q2 = S.n[pr[a]][2][po[a]] - n2;
                            if (own) l_nrm += q0 * q0 + q1 * q1 + q2 * q2;
                            const float kk = cn * w;
                            dn0 -= kk * q0;
                            dn1 -= kk * q1;
                            dn2 -= kk * q2;
                        }
                        if (S.n[mr[a]][4][mo[a]] > 0.0f) {
                            const float kk = cn * S.n[mr[a]][3][mo[a]];
                            dn0 += kk * (n0 - S.n[mr[a]][0][mo[a]]);
                            dn1 += kk * (n1 - S.n[mr[a]][1][mo[a]]);
                            dn2 += kk * (n2 - S.n[mr[a]][2][mo[a]]);
                        }
                    }
                    const float ndn = n0 * dn0 + n1 * dn1 + n2 * dn2;
                    const float ir = 1.0f / rho;
                    // dg = ce g + (dn - n (n . dn)) / rho, with g = n rho
                    d0 = ce * n0 * rho + (dn0 - n0 * ndn) * ir;
                    d1 = ce * n1 * rho + (dn1 - n1 * ndn) * ir;
                    d2 = ce * n2 * rho + (dn2 - n2 * ndn) * ir;
                }
                S.g[rc][0][e] = d0;
                S.g[rc][1][e] = d1;
                S.g[rc][2][e] = d2;
            }
        }
        __syncthreads();
        // ---- outputs at zo = zs - 3 (G planes zo - 1, zo, zo + 1 in ra, rb, rc) ----
        if (out) {
            const float w = 1.0f / (1.0f + 5.0f * fabsf(s_o));
            // Eq. 11
            const float r = s_o - sh_o;
            l_sdf += r * r;
            const float own = P.lam_sdf * w * 2.0f * r;
            P.d_s_hat[io] = dsh_o - own;
            const int c = c_o;
            const float adj = (S.g[rb][0][c - 1] - S.g[rb][0][c + 1]) * P.inv2h[0] +
                              (S.g[rb][1][c - GX] - S.g[rb][1][c + GX]) * P.inv2h[1] +
                              (S.g[ra][2][c] - S.g[rc][2][c]) * P.inv2h[2];
            P.d_s[io * P.d_stride] = ds_o + (own + adj);
        }
        const int t = ra;  // rotate: this step's slots become one step back
        ra = rb;
        rb = rc;
        rc = t;
    }
    block_loss(l_sdf, l_eik, l_nrm, P.loss, 3);
}

// L_features: planes as 16-byte texels {f0, f1, f2, 0}; gradient gathered per
// texel from its (up to 4) in-plane neighbours.
__global__ void __launch_bounds__(256) plane_reg_kernel(const float4* __restrict__ planes,
                                                        int64_t n_texels, float lam,
                                                        float4* __restrict__ grad, float* loss)
{
    float l = 0.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_texels;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i % 16), r = static_cast<int>((i / 16) % 16);
        const float4 v = __ldg(planes + i);
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        auto pair = [&](const float4& u, float sgn) {  // sgn * (v - u) enters the gradient
            g.x += sgn * 2.0f * lam * (v.x - u.x);
            g.y += sgn * 2.0f * lam * (v.y - u.y);
            g.z += sgn * 2.0f * lam * (v.z - u.z);
        };
        if (c > 0) pair(__ldg(planes + i - 1), 1.0f);
        if (r > 0) pair(__ldg(planes + i - 16), 1.0f);
        if (c < 15) {
            const float4 u = __ldg(planes + i + 1);
            pair(u, 1.0f);
            const float dx = u.x - v.x, dy = u.y - v.y, dz = u.z - v.z;
            l += dx * dx + dy * dy + dz * dz;
        }
        if (r < 15) {
            const float4 u = __ldg(planes + i + 16);
            pair(u, 1.0f);
            const float dx = u.x - v.x, dy = u.y - v.y, dz = u.z - v.z;
            l += dx * dx + dy * dy + dz * dz;
        }
        float4 o = grad[i];
        o.x += g.x;
        o.y += g.y;
        o.z += g.z;
        grad[i] = o;
    }
    block_loss(l, 0.0f, 0.0f, loss, 1);
}

// L_probes over [Pz][Py][Px][l*l * n_a] coefficient vectors, read as float4.
__global__ void __launch_bounds__(256) probe_reg_kernel(const float4* __restrict__ b, int Px,
                                                        int Py, int Pz, int n4, float lam,
                                                        float4* __restrict__ grad, float* loss)
{
    const int64_t n = int64_t(Px) * Py * Pz * n4;
    float l = 0.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t node = i / n4;
        const int x = static_cast<int>(node % Px), y = static_cast<int>((node / Px) % Py);
        const int z = static_cast<int>(node / (int64_t(Px) * Py));
        const float4 v = __ldg(b + i);
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t step[3] = {int64_t(n4), int64_t(Px) * n4, int64_t(Px) * Py * n4};
        const int pos[3] = {x, y, z}, lim[3] = {Px, Py, Pz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const int q = pos[a] + sgn;
                if (q < 0 || q >= lim[a]) continue;
                const float4 u = __ldg(b + i + sgn * step[a]);
                const float dx = v.x - u.x, dy = v.y - u.y, dz = v.z - u.z, dw = v.w - u.w;
                g.x += 4.0f * lam * dx;
                g.y += 4.0f * lam * dy;
                g.z += 4.0f * lam * dz;
                g.w += 4.0f * lam * dw;
                l += dx * dx + dy * dy + dz * dz + dw * dw;  // each ordered pair once
            }
        }
        float4 o = grad[i];
        o.x += g.x;
        o.y += g.y;
        o.z += g.z;
        o.w += g.w;
        grad[i] = o;
    }
    block_loss(l, 0.0f, 0.0f, loss, 1);
}

Taps gauss_taps()
{
    Taps T;
    double w[5], sum = 0.0;
    for (int j = 0; j < 5; ++j) {
        const double k = j - HALO;
        w[j] = std::exp(-0.5 * k * k);
        sum += w[j];
    }
    for (int j = 0; j < 5; ++j) T.w[j] = static_cast<float>(w[j] / sum);
    return T;
}

int sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int blocks(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    const int64_t cap = int64_t(sms()) * 16;
    return static_cast<int>(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

cudaError_t launch_smooth(const int R[3], const float* in, int in_stride, float* out,
                          int out_stride, bool transpose, bool accumulate, cudaStream_t stream)
{
    const dim3 grid((R[0] + TX - 1) / TX, (R[1] + TY - 1) / TY, (R[2] + TZ - 1) / TZ);
    const Taps T = gauss_taps();
    if (transpose)
        smooth_kernel<true><<<grid, kSmoothThreads, 0, stream>>>(in, in_stride, out, out_stride, R[0], R[1],
                                                       R[2], T, accumulate ? 1 : 0);
    else
        smooth_kernel<false><<<grid, kSmoothThreads, 0, stream>>>(in, in_stride, out, out_stride, R[0], R[1],
                                                        R[2], T, accumulate ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_smooth_sparse(const int R[3], const int* table, int n_bricks, const float* in,
                                 int64_t in_base, int in_stride, float* out, int64_t out_base,
                                 int out_stride, float empty, bool transpose, bool accumulate,
                                 cudaStream_t stream)
{
    SparseSmooth P;
    P.table = table;
    int64_t entries = 1;
    for (int a = 0; a < 3; ++a) {
        P.R[a] = R[a];
        P.B[a] = R[a] / SB;
        entries *= P.B[a];
    }
    P.n_bricks = n_bricks;
    P.in = in;
    P.in_base = in_base;
    P.in_stride = in_stride;
    P.out = out;
    P.out_base = out_base;
    P.out_stride = out_stride;
    P.empty = empty;
    P.accumulate = accumulate ? 1 : 0;
    if (entries < 1 || entries > 0x7fffffff) return cudaErrorInvalidValue;
    const Taps T = gauss_taps();
    auto kernel = transpose ? sparse_smooth_kernel<true> : sparse_smooth_kernel<false>;
    const cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpBytes);
    if (e != cudaSuccess) return e;
    kernel<<<static_cast<unsigned>(entries), kSpThreads, kSpBytes, stream>>>(P, T);
    return cudaGetLastError();
}

cudaError_t launch_sdf_reg(const int R[3], const float h[3], const float* s_hat, const float* s,
                           int s_stride, float lam_sdf, float lam_eik, float lam_normal,
                           float* d_s, int d_stride, float* d_s_hat, float* loss,
                           cudaStream_t stream, const int* table, int n_bricks, float empty)
{
    SdfReg P;
    P.s_hat = s_hat;
    P.s = s;
    P.s_stride = s_stride;
    P.d_s = d_s;
    P.d_stride = d_stride;
    P.d_s_hat = d_s_hat;
    P.loss = loss;
    int64_t entries = 1;
    for (int a = 0; a < 3; ++a) {
        P.R[a] = R[a];
        P.inv2h[a] = 0.5f / h[a];
        P.B[a] = R[a] / SB;
        entries *= P.B[a];
    }
    P.lam_sdf = lam_sdf;
    P.lam_eik = lam_eik;
    P.lam_normal = lam_normal;
    P.table = table;
    P.n_bricks = n_bricks;
    P.empty = empty;
    if (table) {
        if (entries < 1 || entries > 0x7fffffff) return cudaErrorInvalidValue;
        constexpr int kBytes = static_cast<int>(sizeof(SparseReg::Smem));
        auto kernel = sdf_reg_kernel<SparseReg, true>;
        cudaError_t e =
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBytes);
        if (e != cudaSuccess) return e;
        kernel<<<static_cast<unsigned>(entries), kRegThreads, kBytes, stream>>>(P);
        return cudaGetLastError();
    }
    constexpr int kBytes = static_cast<int>(sizeof(DenseReg::Smem));
    auto kernel = sdf_reg_kernel<DenseReg, false>;
    cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBytes);
    if (e != cudaSuccess) return e;
    const dim3 grid((R[0] + DenseReg::RX - 1) / DenseReg::RX,
                    (R[1] + DenseReg::RY - 1) / DenseReg::RY,
                    (R[2] + DenseReg::ZC - 1) / DenseReg::ZC);
    kernel<<<grid, kRegThreads, kBytes, stream>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_plane_reg(const float4* planes, int64_t n_texels, float lam, float4* grad,
                             float* loss, cudaStream_t stream)
{
    plane_reg_kernel<<<blocks(n_texels), 256, 0, stream>>>(planes, n_texels, lam, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_probe_reg(const float4* b, const int P[3], int n4, float lam, float4* grad,
                             float* loss, cudaStream_t stream)
{
    probe_reg_kernel<<<blocks(int64_t(P[0]) * P[1] * P[2] * n4), 256, 0, stream>>>(
        b, P[0], P[1], P[2], n4, lam, grad, loss);
    return cudaGetLastError();
}

}  // namespace psdf
