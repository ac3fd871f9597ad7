// Device-side building blocks of the ProbeSDF per-ray render (sm_103a).
//
// One warp renders one ray; lane l holds sample k = 32 c + l of chunk c.
// Everything here is per lane; the warp-level scans live in the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace psdf {

constexpr int kWarp = 32;
constexpr float kNormalEps = 1e-12f;  // n = g / sqrt(|g|^2 + eps^2)

// Kernel view of the packed SDF + feature grid: one float4 {sdf, f0, f1, f2}
// per node, x fastest.
struct GridView {
    const float4* __restrict__ nodes;   // FP32 records {sdf, f0, f1, f2}
    const float* __restrict__ sdf;      // BF16-feature / tri-plane layouts: FP32 SDF per node ...
    const uint2* __restrict__ feat16;   // ... and {f0, f1, f2, 0} as BF16 per node
    const float4* __restrict__ planes;  // ... or tile tri-planes: [tile][3][16][16] {f0, f1, f2, 0}
    int tiles[3];                       // tiles of 16 cells along x, y, z
    int64_t plane_off;                  // tri-planes: float offset of the planes in the values
                                        // and gradient buffers (the SDF array comes first)
    const int* __restrict__ table;      // sparse: brick table [Bz][By][Bx] (slot or -1); the
                                        // records of `nodes` are then the stored bricks'
    int B[3];                           // sparse: bricks of 16^3 nodes along x, y, z
    int n_bricks;                       // sparse: stored bricks (a slot beyond is not stored)
    float empty_sdf;                    // sparse: SDF of the nodes of bricks not stored
    int64_t rec_off;                    // sparse: float offset of the brick records in the
                                        // values and gradient buffers (the table comes first)
    int R[3];
    float bmin[3];
    float bmax[3];
    float sc[3];  // (R - 1) / (bmax - bmin), FP32-rounded on the host
};

// Probe coefficients, [Pz][Py][Px][L2][NA] FP32, viewed as float4 groups of
// four channels.
struct ProbeView {
    const float4* __restrict__ coeffs;    // FP32 coefficients, 4 channels per float4
    const uint2* __restrict__ coeffs16;   // FP16 coefficients, 4 channels per uint2
    int P[3];
    float sc[3];
};

struct RenderArgs {
    GridView grid;
    ProbeView probes;
    const float* __restrict__ mlp;  // W1 b1 W2 b2 W3 b3
    float tau;
    int n_samples;
    int dir_mode;  // 0 reflect, 1 view
    float bg[3];
    const float* __restrict__ rays_o;
    const float* __restrict__ rays_d;
    const float* __restrict__ t_samples;  // nullable [n_rays][N+1], or [n_rays][n_bins]
    int n_bins;                           // > 0: t_samples holds bin densities
    int64_t n_rays;
    // forward outputs / backward inputs
    float* rgb;
    float* depth;
    float* wsum;
    float* logT;
    // forward output / backward input (nullable): 1 + index of the ray's last
    // sample with a nonzero opacity (0 when none is)
    int* n_live;
    // backward
    const float* __restrict__ d_rgb;
    const float* __restrict__ d_depth;
    const float* __restrict__ d_wsum;
    float* grad_grid;
    float* grad_probes;
    float* grad_mlp;
    int* status;  // device status word: bit 0 = a tensor-core wait ran out
    uint32_t wait_polls;  // polls of each tensor-core completion wait before it gives up
};

// ---------------------------------------------------------------------------
// Sample positions.  These decide integer cell indices, so they use explicit
// round-to-nearest intrinsics (never contracted into FMAs) in a fixed order;
// any IEEE-754 FP32 implementation of the same sequence gives the same bits.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool ray_box(const float o[3], const float d[3], const GridView& g,
                                        float& tn, float& tf)
{
    float t_enter = -INFINITY, t_exit = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < g.bmin[a] || o[a] > g.bmax[a]) return false;
            continue;
        }
        const float t0 = __fdiv_rn(__fsub_rn(g.bmin[a], o[a]), d[a]);
        const float t1 = __fdiv_rn(__fsub_rn(g.bmax[a], o[a]), d[a]);
        const float lo = t0 < t1 ? t0 : t1;
        const float hi = t0 < t1 ? t1 : t0;
        if (lo > t_enter) t_enter = lo;
        if (hi < t_exit) t_exit = hi;
    }
    tn = t_enter > 0.0f ? t_enter : 0.0f;
    tf = t_exit;
    return tf > tn;
}

__device__ __forceinline__ float sample_t(int k, float dt, float tn)
{
    return __fmaf_rn(static_cast<float>(k), dt, tn);
}

// Cell of a point along one axis: floor(u) clamped to [0, R-2]; the fraction
// u - i is exact.
__device__ __forceinline__ void locate_axis(float x, float bmin, float sc, int R, int& i,
                                            float& f)
{
    const float u = __fmul_rn(__fsub_rn(x, bmin), sc);
    float fl = floorf(u);
    const float hi = static_cast<float>(R - 2);
    fl = fl >= 0.0f ? fl : 0.0f;  // also maps NaN to cell 0: every index stays in bounds
    fl = fl > hi ? hi : fl;
    i = static_cast<int>(fl);
    f = __fsub_rn(u, fl);
}

struct Cell {
    int base;  // linear index of corner (0,0,0)
    int i[3];  // its node coordinates
    float f[3];
};

__device__ __forceinline__ Cell locate(const float x[3], const float bmin[3], const float sc[3],
                                       const int R[3])
{
    Cell c;
    int i[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) locate_axis(x[a], bmin[a], sc[a], R[a], i[a], c.f[a]);
    c.base = (i[2] * R[1] + i[1]) * R[0] + i[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) c.i[a] = i[a];
    return c;
}

// ---------------------------------------------------------------------------
// Sparse bricks: the nodes form bricks of 16^3; only the bricks the table
// names are stored.  Record index of node (x, y, z), or -1 when its brick is
// not stored (a table entry outside [0, n_bricks) counts as not stored).
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t brick_record(const GridView& g, int x, int y, int z)
{
    const int slot = __ldg(g.table + ((z >> 4) * g.B[1] + (y >> 4)) * g.B[0] + (x >> 4));
    if (slot < 0 || slot >= g.n_bricks) return -1;
    return int64_t(slot) * 4096 + (((z & 15) << 8) | ((y & 15) << 4) | (x & 15));
}

// Record indices of a cell's 8 corners (corner q = cx + 2 cy + 4 cz); returns
// how many are stored.
__device__ __forceinline__ int brick_corners(const GridView& g, const int i[3], int64_t rec[8])
{
    int stored = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        rec[q] = brick_record(g, i[0] + (q & 1), i[1] + ((q >> 1) & 1), i[2] + (q >> 2));
        stored += rec[q] >= 0;
    }
    return stored;
}

__device__ __forceinline__ void point_at(const float o[3], const float d[3], float t, float x[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = __fmaf_rn(t, d[a], o[a]);
}

// Two FP32 fused multiply-adds in one instruction (fma.rn.f32x2, sm_100
// family): each half is rounded exactly as fmaf rounds it, so a pair gives the
// bits of the two scalar calls in half the issue slots.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Paired FP32 add and multiply (add.rn.f32x2, mul.rn.f32x2): each half rounds
// as the scalar operation does.
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// ---------------------------------------------------------------------------
// Trilinear gathers (Sec. 3.1): 8 corner records of 16 bytes each.
// ---------------------------------------------------------------------------

// Read-only 16-byte loads with eviction priorities: the probe coefficients (a
// few MB, reused by every ray) are kept in L1 and L2 over the grid's node
// records (reused only by neighbouring samples), which go first in L1.
// The L2 evict-last policy, in an asm of its own without side effects, so
// that one instance serves every load of a kernel (hoisted, not re-created).
__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ float4 ldg_keep(const float4* p)
{
    float4 v;
    asm("ld.global.nc.L1::evict_last.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(l2_evict_last()));
    return v;
}

__device__ __forceinline__ float4 ldg_stream(const float4* p)
{
    float4 v;
    asm("ld.global.nc.L1::evict_first.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

struct Corners {
    float4 v[8];  // corner c = cx + 2 cy + 4 cz
};

__device__ __forceinline__ void gather_corners(const GridView& g, const Cell& c, Corners& k)
{
    const int sx = 1, sy = g.R[0], sz = g.R[0] * g.R[1];
    const float4* p = g.nodes + c.base;
    k.v[0] = ldg_stream(p);
    k.v[1] = ldg_stream(p + sx);
    k.v[2] = ldg_stream(p + sy);
    k.v[3] = ldg_stream(p + sx + sy);
    k.v[4] = ldg_stream(p + sz);
    k.v[5] = ldg_stream(p + sz + sx);
    k.v[6] = ldg_stream(p + sz + sy);
    k.v[7] = ldg_stream(p + sz + sy + sx);
}

__device__ __forceinline__ void corner_weights(const float f[3], float w[8])
{
    const float x0 = 1.0f - f[0], x1 = f[0];
    const float y0 = 1.0f - f[1], y1 = f[1];
    const float z0 = 1.0f - f[2], z1 = f[2];
    w[0] = x0 * y0 * z0;
    w[1] = x1 * y0 * z0;
    w[2] = x0 * y1 * z0;
    w[3] = x1 * y1 * z0;
    w[4] = x0 * y0 * z1;
    w[5] = x1 * y0 * z1;
    w[6] = x0 * y1 * z1;
    w[7] = x1 * y1 * z1;
}

__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

// Corner records of the BF16-feature layout, widened to the FP32 record form.
__device__ __forceinline__ void gather_corners_bf16(const GridView& g, const Cell& c, Corners& k)
{
    const int sx = 1, sy = g.R[0], sz = g.R[0] * g.R[1];
    const int off[8] = {0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sy + sx};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float s = __ldg(g.sdf + c.base + off[q]);
        const uint2 f = __ldg(g.feat16 + c.base + off[q]);
        k.v[q] = make_float4(s, bf16_lo(f.x), bf16_hi(f.x), bf16_lo(f.y));
    }
}

// SDF only (tri-plane layout): the features come from the tile planes.
__device__ __forceinline__ void gather_corners_sdf(const GridView& g, const Cell& c, Corners& k)
{
    const int sx = 1, sy = g.R[0], sz = g.R[0] * g.R[1];
    const int off[8] = {0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sy + sx};
#pragma unroll
    for (int q = 0; q < 8; ++q) k.v[q] = make_float4(__ldg(g.sdf + c.base + off[q]), 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// Tile tri-plane spatial features (Sec. 3.1, Sec. 4).  The cells form tiles of
// 16^3; a tile holds three 16 x 16 planes of texels {f0, f1, f2}, orthogonal
// to x ([z][y]), y ([z][x]) and z ([y][x]); F_s = F_x * F_y * F_z channel by
// channel, each factor a bilinear lookup at the point's two in-plane
// coordinates.  Texels sit at the centres of the tile's cells, the texel
// coordinate is clamped to the tile.  The tile and texel follow exactly from
// the FP32 grid coordinate u (u / 16 and u - 16 t are exact).
// ---------------------------------------------------------------------------

constexpr int kTile = 16;

struct TriAt {
    int plane0;  // texel index of the tile's first plane
    int i[3];    // texel index along x, y, z (0..14)
    float f[3];  // fraction to the next texel
};

// Tile and texel of FP32 grid coordinates u (node units).
__device__ __forceinline__ void triplane_locate_u(const GridView& g, const float uu[3], TriAt& T)
{
    int t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = uu[a];
        float ta = floorf(u * (1.0f / kTile));
        ta = ta >= 0.0f ? ta : 0.0f;  // also maps NaN to tile 0
        ta = fminf(ta, static_cast<float>(g.tiles[a] - 1));
        float tau = __fsub_rn(__fsub_rn(u, ta * kTile), 0.5f);
        tau = fminf(fmaxf(tau, 0.0f), static_cast<float>(kTile - 1));
        const float fi = fminf(floorf(tau), static_cast<float>(kTile - 2));
        t[a] = static_cast<int>(ta);
        T.i[a] = static_cast<int>(fi);
        T.f[a] = __fsub_rn(tau, fi);
    }
    T.plane0 = ((t[2] * g.tiles[1] + t[1]) * g.tiles[0] + t[0]) * 3 * kTile * kTile;
}

__device__ __forceinline__ void triplane_locate(const GridView& g, const float x[3], TriAt& T)
{
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = __fmul_rn(__fsub_rn(x[a], g.bmin[a]), g.sc[a]);  // as locate_axis
    triplane_locate_u(g, u, T);
}

// plane p: 0 is [z][y], 1 is [z][x], 2 is [y][x]
__device__ __forceinline__ constexpr int tri_row(int p) { return p == 2 ? 1 : 2; }
__device__ __forceinline__ constexpr int tri_col(int p) { return p == 0 ? 1 : 0; }

// The three bilinear lookups b[p] ({f0, f1, f2} of plane p) and F_s.
__device__ __forceinline__ void triplane_lookup(const GridView& g, const TriAt& T, float fs[3],
                                                float4* b = nullptr)
{
    float4 v[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int ra = tri_row(p), ca = tri_col(p);
        const float fr = T.f[ra], fc = T.f[ca];
        const float4* P = g.planes + T.plane0 + p * kTile * kTile + T.i[ra] * kTile + T.i[ca];
        const float4 a00 = __ldg(P), a01 = __ldg(P + 1);
        const float4 a10 = __ldg(P + kTile), a11 = __ldg(P + kTile + 1);
        const float w00 = (1.0f - fr) * (1.0f - fc), w01 = (1.0f - fr) * fc;
        const float w10 = fr * (1.0f - fc), w11 = fr * fc;
        v[p].x = w00 * a00.x + w01 * a01.x + w10 * a10.x + w11 * a11.x;
        v[p].y = w00 * a00.y + w01 * a01.y + w10 * a10.y + w11 * a11.y;
        v[p].z = w00 * a00.z + w01 * a01.z + w10 * a10.z + w11 * a11.z;
        v[p].w = 0.0f;
        if (b) b[p] = v[p];
    }
    fs[0] = v[0].x * v[1].x * v[2].x;
    fs[1] = v[0].y * v[1].y * v[2].y;
    fs[2] = v[0].z * v[1].z * v[2].z;
}

// Corner records of a sparse grid; returns the stored count (0: every corner
// is empty and the caller takes s = empty_sdf exactly).
__device__ __forceinline__ int gather_corners_sparse(const GridView& g, const Cell& c, Corners& k)
{
    int64_t rec[8];
    const int stored = brick_corners(g, c.i, rec);
#pragma unroll
    for (int q = 0; q < 8; ++q)
        k.v[q] = rec[q] >= 0 ? __ldg(g.nodes + rec[q]) : make_float4(g.empty_sdf, 0.f, 0.f, 0.f);
    return stored;
}

// The 8 corner SDF values of a cell of a dense grid (FP32 node records, or
// the SDF array of the BF16-feature and tri-plane layouts), loaded but not yet
// combined, so that a caller can have them in flight with other loads.
__device__ __forceinline__ void sdf_corners_load(const GridView& g, const Cell& c, float v[8])
{
    const int sx = 1, sy = g.R[0], sz = g.R[0] * g.R[1];
    const bool split = g.sdf != nullptr;  // BF16-feature layout: SDF in its own array
    const float* p = split ? g.sdf + c.base : reinterpret_cast<const float*>(g.nodes + c.base);
    const int st = split ? 1 : 4;
    const int off[8] = {0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sy + sx};
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldg(p + st * off[q]);
}

// Trilinear SDF value from the corner values: the same weights and summation
// order as sdf_full, so both give the same bits for the same point.
__device__ __forceinline__ float sdf_corners_combine(const Cell& c, const float v[8])
{
    float w[8];
    corner_weights(c.f, w);
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s = fmaf(w[q], v[q], s);
    return s;
}

// SDF value only (the point after a chunk's last sample).
__device__ __forceinline__ float sdf_value(const GridView& g, const Cell& c)
{
    if (g.table) {
        int64_t rec[8];
        if (brick_corners(g, c.i, rec) == 0) return g.empty_sdf;
        float w[8];
        corner_weights(c.f, w);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            s = fmaf(w[q], rec[q] >= 0 ? __ldg(reinterpret_cast<const float*>(g.nodes + rec[q]))
                                       : g.empty_sdf,
                     s);
        return s;
    }
    float v[8];
    sdf_corners_load(g, c, v);
    return sdf_corners_combine(c, v);
}

// Value, analytic gradient (world units) and 3 features at a point.
__device__ __forceinline__ void sdf_full(const GridView& g, const Cell& c, const Corners& k,
                                         float& s, float grad[3], float feat[3])
{
    float w[8];
    corner_weights(c.f, w);
    s = 0.0f;
    feat[0] = feat[1] = feat[2] = 0.0f;
    float2 sf0 = make_float2(0.0f, 0.0f), f12 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float2 wq = make_float2(w[q], w[q]);
        sf0 = fma2(wq, make_float2(k.v[q].x, k.v[q].y), sf0);  // s, feature 0
        f12 = fma2(wq, make_float2(k.v[q].z, k.v[q].w), f12);  // features 1, 2
    }
    s = sf0.x;
    feat[0] = sf0.y;
    feat[1] = f12.x;
    feat[2] = f12.y;
    const float fx = c.f[0], fy = c.f[1], fz = c.f[2];
    const float x0 = 1.0f - fx, y0 = 1.0f - fy, z0 = 1.0f - fz;
    // d/du_x: differences along x weighted by the (y, z) bilinear weights
    const float gx = (y0 * z0) * (k.v[1].x - k.v[0].x) + (fy * z0) * (k.v[3].x - k.v[2].x) +
                     (y0 * fz) * (k.v[5].x - k.v[4].x) + (fy * fz) * (k.v[7].x - k.v[6].x);
    const float gy = (x0 * z0) * (k.v[2].x - k.v[0].x) + (fx * z0) * (k.v[3].x - k.v[1].x) +
                     (x0 * fz) * (k.v[6].x - k.v[4].x) + (fx * fz) * (k.v[7].x - k.v[5].x);
    const float gz = (x0 * y0) * (k.v[4].x - k.v[0].x) + (fx * y0) * (k.v[5].x - k.v[1].x) +
                     (x0 * fy) * (k.v[6].x - k.v[2].x) + (fx * fy) * (k.v[7].x - k.v[3].x);
    grad[0] = gx * g.sc[0];
    grad[1] = gy * g.sc[1];
    grad[2] = gz * g.sc[2];
}

// ---------------------------------------------------------------------------
// Real spherical harmonics, orthonormal, no Condon-Shortley phase (Eq. 5),
// ordered by degree then m = -deg..deg.  L2 = l*l with l 1-indexed.
// ---------------------------------------------------------------------------

template <int L2>
__device__ __forceinline__ void sh_basis(const float r[3], float Y[L2])
{
    const float x = r[0], y = r[1], z = r[2];
    Y[0] = 0.28209479177387814f;
    if constexpr (L2 > 1) {
        Y[1] = 0.48860251190291992f * y;
        Y[2] = 0.48860251190291992f * z;
        Y[3] = 0.48860251190291992f * x;
    }
    if constexpr (L2 > 4) {
        Y[4] = 1.0925484305920792f * (x * y);
        Y[5] = 1.0925484305920792f * (y * z);
        Y[6] = 0.31539156525252005f * (3.0f * z * z - 1.0f);
        Y[7] = 1.0925484305920792f * (x * z);
        Y[8] = 0.54627421529603959f * (x * x - y * y);
    }
    if constexpr (L2 > 9) {
        Y[9] = 0.59004358992664352f * y * (3.0f * x * x - y * y);
        Y[10] = 2.8906114426405538f * (x * y * z);
        Y[11] = 0.45704579946446572f * y * (5.0f * z * z - 1.0f);
        Y[12] = 0.37317633259011540f * z * (5.0f * z * z - 3.0f);
        Y[13] = 0.45704579946446572f * x * (5.0f * z * z - 1.0f);
        Y[14] = 1.4453057213202769f * z * (x * x - y * y);
        Y[15] = 0.59004358992664352f * x * (x * x - 3.0f * y * y);
    }
}

// dr = sum_j dY_j * grad Y_j(r)
template <int L2>
__device__ __forceinline__ void sh_basis_vjp(const float r[3], const float dY[L2], float dr[3])
{
    const float x = r[0], y = r[1], z = r[2];
    dr[0] = dr[1] = dr[2] = 0.0f;
    if constexpr (L2 > 1) {
        const float c = 0.48860251190291992f;
        dr[1] += c * dY[1];
        dr[2] += c * dY[2];
        dr[0] += c * dY[3];
    }
    if constexpr (L2 > 4) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f,
                    e = 0.54627421529603959f;
        dr[0] += a * (y * dY[4] + z * dY[7]) + 2.0f * e * x * dY[8];
        dr[1] += a * (x * dY[4] + z * dY[5]) - 2.0f * e * y * dY[8];
        dr[2] += a * (y * dY[5] + x * dY[7]) + 6.0f * b * z * dY[6];
    }
    if constexpr (L2 > 9) {
        const float c33 = 0.59004358992664352f, c32 = 2.8906114426405538f,
                    c31 = 0.45704579946446572f, c30 = 0.37317633259011540f,
                    c32b = 1.4453057213202769f;
        dr[0] += c33 * 6.0f * x * y * dY[9] + c32 * y * z * dY[10] +
                 c31 * (5.0f * z * z - 1.0f) * dY[13] + c32b * 2.0f * x * z * dY[14] +
                 c33 * (3.0f * x * x - 3.0f * y * y) * dY[15];
        dr[1] += c33 * (3.0f * x * x - 3.0f * y * y) * dY[9] + c32 * x * z * dY[10] +
                 c31 * (5.0f * z * z - 1.0f) * dY[11] - c32b * 2.0f * y * z * dY[14] -
                 c33 * 6.0f * x * y * dY[15];
        dr[2] += c32 * x * y * dY[10] + c31 * 10.0f * y * z * dY[11] +
                 c30 * (15.0f * z * z - 3.0f) * dY[12] + c31 * 10.0f * x * z * dY[13] +
                 c32b * (x * x - y * y) * dY[14];
    }
}

// ---------------------------------------------------------------------------
// NeuS helpers (Eqs. 9-10).
// ---------------------------------------------------------------------------

// log Phi_tau(s) = -softplus(-tau s)
__device__ __forceinline__ float log_phi(float tau, float s)
{
    const float z = -tau * s;
    return -(fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))));
}

// log(1 - alpha) before the clip of Eq. 9: log Phi(s1) - log Phi(s0).  With
// z = -tau s this is softplus(z0) - softplus(z1) = log1p(sigmoid(z1) expm1(z0 - z1)),
// which keeps full relative accuracy when s1 is close to s0 (a grazing ray),
// where the difference of the two logarithms cancels in FP32.  When the
// argument nears -1 (a large drop deep inside the surface) the plain
// difference is already accurate and avoids log1p(-1).
__device__ __forceinline__ float log_transmittance(float tau, float s0, float s1)
{
    const float p = expm1f(tau * (s1 - s0)) / (1.0f + expf(tau * s1));
    if (p > -0.5f) return log1pf(p);
    return log_phi(tau, s1) - log_phi(tau, s0);
}

// d log Phi / ds = tau * (1 - Phi(s)) = tau * sigmoid(-tau s)
__device__ __forceinline__ float dlog_phi(float tau, float s)
{
    return tau / (1.0f + expf(tau * s));
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// The rays of a persistent CTA of 4 warps are b * 4 + (j & 3) + (j >> 2) * stride,
// j = 0, 1, ... (increasing in j).  Its warps take the next j from a counter in
// shared memory (zeroed before the CTA's first barrier), so a warp whose rays
// end early takes more of them.  Warp-collective; every lane gets the ray.
__device__ __forceinline__ int64_t next_cta_ray(int* counter, int64_t stride)
{
    int j = 0;
    if ((threadIdx.x & 31) == 0) j = atomicAdd(counter, 1);
    j = __shfl_sync(0xffffffffu, j, 0);
    return int64_t(blockIdx.x) * 4 + (j & 3) + int64_t(j >> 2) * stride;
}

// Vector reduction into global memory (no return value).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void red_add(float* addr, float a)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

}  // namespace psdf
