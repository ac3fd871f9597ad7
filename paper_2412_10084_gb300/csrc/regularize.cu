// Grid-level training terms of ProbeSDF (Sec. 3.3, Eqs. 11-15).
//
//   smooth_kernel<false>  s = G(s_hat): 5^3 Gaussian (sigma = 1 node, separable,
//                         replicated edge nodes); one shared-memory tile pass
//                         (32 x 8 x 8 outputs, 2-node halo) per CTA
//   smooth_kernel<true>   G^T: the same tiles with the transposed 1D operators,
//                         applied z, y, x (edge outputs gather the replicated taps)
//   sdf_reg_kernel        L_sdf, L_Eik and L_normal on the smoothed SDF, their
//                         gradients scaled by (1 + 5 |s|)^-1; the central-
//                         difference adjoint is reduced into the 6 neighbours
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

// Weight with which input node `in` enters output node `out` of the 1D
// convolution along an axis of n nodes (tap j reads clamp(out + j - 2)).
__device__ __forceinline__ float conv_weight(const Taps& T, int in, int out, int n)
{
    float w = 0.0f;
#pragma unroll
    for (int j = 0; j < 5; ++j)
        if (clampi(out + j - HALO, 0, n - 1) == in) w += T.w[j];
    return w;
}

template <bool TRANSPOSE>
__global__ void __launch_bounds__(kSmoothThreads) smooth_kernel(const float* __restrict__ in, int in_stride,
                                                     float* __restrict__ out, int out_stride,
                                                     int Rx, int Ry, int Rz, Taps T, int accumulate)
{
    __shared__ float A[kBufA];
    __shared__ float B[kBufB];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int tid = threadIdx.x;
    // tile + halo: forward reads replicate the edge nodes; the transposed
    // operator has no input outside the grid (zeros).  All of a thread's loads
    // are issued before the first store to shared memory.
    constexpr int kLoads = (kBufA + kSmoothThreads - 1) / kSmoothThreads;
    float v[kLoads];
#pragma unroll
    for (int it = 0; it < kLoads; ++it) {
        const int e = tid + it * kSmoothThreads;
        const int ax = e % AX, ay = (e / AX) % AY, az = e / (AX * AY);
        const int gx = x0 + ax - HALO, gy = y0 + ay - HALO, gz = z0 + az - HALO;
        v[it] = 0.0f;
        if (e >= kBufA) continue;
        if (!TRANSPOSE) {
            const size_t g = ((size_t)clampi(gz, 0, Rz - 1) * Ry + clampi(gy, 0, Ry - 1)) * Rx +
                             clampi(gx, 0, Rx - 1);
            v[it] = __ldg(in + g * in_stride);
        } else if (gx >= 0 && gx < Rx && gy >= 0 && gy < Ry && gz >= 0 && gz < Rz) {
            v[it] = __ldg(in + (((size_t)gz * Ry + gy) * Rx + gx) * in_stride);
        }
    }
#pragma unroll
    for (int it = 0; it < kLoads; ++it) {
        const int e = tid + it * kSmoothThreads;
        if (e < kBufA) A[e] = v[it];
    }
    __syncthreads();
    if (!TRANSPOSE) {
        // x: A[AZ][AY][AX] -> B[AZ][AY][TX]
        for (int e = tid; e < AZ * AY * TX; e += kSmoothThreads) {
            const int x = e % TX, ay = (e / TX) % AY, az = e / (TX * AY);
            const float* a = A + (az * AY + ay) * AX + x;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], a[j], acc);
            B[e] = acc;
        }
        __syncthreads();
        // y: B[AZ][AY][TX] -> A[AZ][TY][TX]
        for (int e = tid; e < AZ * TY * TX; e += kSmoothThreads) {
            const int x = e % TX, y = (e / TX) % TY, az = e / (TX * TY);
            const float* b = B + (az * AY + y) * TX + x;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], b[j * TX], acc);
            A[e] = acc;
        }
        __syncthreads();
        // z: A[AZ][TY][TX] -> output
        for (int e = tid; e < TZ * TY * TX; e += kSmoothThreads) {
            const int x = e % TX, y = (e / TX) % TY, z = e / (TX * TY);
            const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
            if (gx >= Rx || gy >= Ry || gz >= Rz) continue;
            const float* a = A + (z * TY + y) * TX + x;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc = fmaf(T.w[j], a[j * TY * TX], acc);
            float* o = out + (((size_t)gz * Ry + gy) * Rx + gx) * out_stride;
            *o = accumulate ? *o + acc : acc;
        }
    } else {
        // G^T = Gx^T Gy^T Gz^T.  Output k of a transposed pass gathers the
        // inputs i = k - 2 .. k + 2 with the weight the forward gave node k in
        // its output i.
        // z: A[AZ][AY][AX] -> B[TZ][AY][AX]
        for (int e = tid; e < TZ * AY * AX; e += kSmoothThreads) {
            const int ax = e % AX, ay = (e / AX) % AY, z = e / (AX * AY);
            const int k = z0 + z;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int i = k + j - HALO;
                if (i >= 0 && i < Rz)
                    acc = fmaf(conv_weight(T, k, i, Rz), A[((z + j) * AY + ay) * AX + ax], acc);
            }
            B[e] = acc;
        }
        __syncthreads();
        // y: B[TZ][AY][AX] -> A[TZ][TY][AX]
        for (int e = tid; e < TZ * TY * AX; e += kSmoothThreads) {
            const int ax = e % AX, y = (e / AX) % TY, z = e / (AX * TY);
            const int k = y0 + y;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int i = k + j - HALO;
                if (i >= 0 && i < Ry)
                    acc = fmaf(conv_weight(T, k, i, Ry), B[(z * AY + y + j) * AX + ax], acc);
            }
            A[e] = acc;
        }
        __syncthreads();
        // x: A[TZ][TY][AX] -> output
        for (int e = tid; e < TZ * TY * TX; e += kSmoothThreads) {
            const int x = e % TX, y = (e / TX) % TY, z = e / (TX * TY);
            const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
            if (gx >= Rx || gy >= Ry || gz >= Rz) continue;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int i = gx + j - HALO;
                if (i >= 0 && i < Rx)
                    acc = fmaf(conv_weight(T, gx, i, Rx), A[(z * TY + y) * AX + x + j], acc);
            }
            float* o = out + (((size_t)gz * Ry + gy) * Rx + gx) * out_stride;
            *o = accumulate ? *o + acc : acc;
        }
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
    const float* s_hat;  // dense [R^3]
    const float* s;      // smoothed, element stride s_stride
    int s_stride;
    float* d_s;          // gradient w.r.t. s (accumulated), stride d_stride
    int d_stride;
    float* d_s_hat;      // gradient w.r.t. s_hat (accumulated), dense
    float* loss;         // [3]: L_sdf, L_Eik, L_normal (accumulated)
    int R[3];
    float inv2h[3];      // 1 / (2 h_a)
    float lam_sdf, lam_eik, lam_normal;
};

__device__ __forceinline__ float sv(const SdfReg& P, int x, int y, int z)
{
    return __ldg(P.s + (((size_t)z * P.R[1] + y) * P.R[0] + x) * P.s_stride);
}

__device__ __forceinline__ bool interior(const SdfReg& P, int x, int y, int z)
{
    return x > 0 && y > 0 && z > 0 && x < P.R[0] - 1 && y < P.R[1] - 1 && z < P.R[2] - 1;
}

// Central-difference gradient at an interior node.
__device__ __forceinline__ void cgrad(const SdfReg& P, int x, int y, int z, float g[3])
{
    g[0] = (sv(P, x + 1, y, z) - sv(P, x - 1, y, z)) * P.inv2h[0];
    g[1] = (sv(P, x, y + 1, z) - sv(P, x, y - 1, z)) * P.inv2h[1];
    g[2] = (sv(P, x, y, z + 1) - sv(P, x, y, z - 1)) * P.inv2h[2];
}

__device__ __forceinline__ void unit_normal(const float g[3], float n[3], float& rho)
{
    rho = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + 1e-24f);
    const float r = 1.0f / rho;
    n[0] = g[0] * r;
    n[1] = g[1] * r;
    n[2] = g[2] * r;
}

__global__ void __launch_bounds__(256) sdf_reg_kernel(SdfReg P)
{
    const int64_t n = int64_t(P.R[0]) * P.R[1] * P.R[2];
    float l_sdf = 0.0f, l_eik = 0.0f, l_nrm = 0.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % P.R[0]);
        const int y = static_cast<int>((i / P.R[0]) % P.R[1]);
        const int z = static_cast<int>(i / (int64_t(P.R[0]) * P.R[1]));
        const float s = sv(P, x, y, z);
        const float w = 1.0f / (1.0f + 5.0f * fabsf(s));
        // Eq. 11
        const float r = s - __ldg(P.s_hat + i);
        l_sdf += r * r;
        float ds_own = P.lam_sdf * w * 2.0f * r;
        P.d_s_hat[i] -= P.lam_sdf * w * 2.0f * r;
        if (interior(P, x, y, z)) {
            float g[3], nrm[3], rho;
            cgrad(P, x, y, z, g);
            unit_normal(g, nrm, rho);
            // Eq. 12
            const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            const float e = gn - 1.0f;
            l_eik += e * e;
            const float ce = gn > 0.0f ? P.lam_eik * w * 2.0f * e / gn : 0.0f;
            float dg[3] = {ce * g[0], ce * g[1], ce * g[2]};
            // Eq. 13: pairs (i, i + e_a) owned by node i, and (i - e_a, i) owned
            // by the neighbour, both between interior nodes
            float dn[3] = {0.f, 0.f, 0.f};
            const int off[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int xp = x + off[a][0], yp = y + off[a][1], zp = z + off[a][2];
                if (interior(P, xp, yp, zp)) {
                    float gp[3], np_[3], rp;
                    cgrad(P, xp, yp, zp, gp);
                    unit_normal(gp, np_, rp);
                    const float d0 = np_[0] - nrm[0], d1 = np_[1] - nrm[1], d2 = np_[2] - nrm[2];
                    l_nrm += d0 * d0 + d1 * d1 + d2 * d2;
                    const float c = P.lam_normal * w * 2.0f;
                    dn[0] -= c * d0;
                    dn[1] -= c * d1;
                    dn[2] -= c * d2;
                }
                const int xm = x - off[a][0], ym = y - off[a][1], zm = z - off[a][2];
                if (interior(P, xm, ym, zm)) {
                    float gm[3], nm[3], rm;
                    cgrad(P, xm, ym, zm, gm);
                    unit_normal(gm, nm, rm);
                    const float wm = 1.0f / (1.0f + 5.0f * fabsf(sv(P, xm, ym, zm)));
                    const float c = P.lam_normal * wm * 2.0f;
                    dn[0] += c * (nrm[0] - nm[0]);
                    dn[1] += c * (nrm[1] - nm[1]);
                    dn[2] += c * (nrm[2] - nm[2]);
                }
            }
            const float ndn = nrm[0] * dn[0] + nrm[1] * dn[1] + nrm[2] * dn[2];
            const float ir = 1.0f / rho;
#pragma unroll
            for (int a = 0; a < 3; ++a) dg[a] += (dn[a] - nrm[a] * ndn) * ir;
            // central-difference adjoint into the neighbours
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float v = dg[a] * P.inv2h[a];
                const size_t ip = ((size_t)(z + off[a][2]) * P.R[1] + (y + off[a][1])) * P.R[0] +
                                  (x + off[a][0]);
                const size_t im = ((size_t)(z - off[a][2]) * P.R[1] + (y - off[a][1])) * P.R[0] +
                                  (x - off[a][0]);
                atomicAdd(P.d_s + ip * P.d_stride, v);
                atomicAdd(P.d_s + im * P.d_stride, -v);
            }
        }
        atomicAdd(P.d_s + i * P.d_stride, ds_own);
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

cudaError_t launch_sdf_reg(const int R[3], const float h[3], const float* s_hat, const float* s,
                           int s_stride, float lam_sdf, float lam_eik, float lam_normal,
                           float* d_s, int d_stride, float* d_s_hat, float* loss,
                           cudaStream_t stream)
{
    SdfReg P;
    P.s_hat = s_hat;
    P.s = s;
    P.s_stride = s_stride;
    P.d_s = d_s;
    P.d_stride = d_stride;
    P.d_s_hat = d_s_hat;
    P.loss = loss;
    for (int a = 0; a < 3; ++a) {
        P.R[a] = R[a];
        P.inv2h[a] = 0.5f / h[a];
    }
    P.lam_sdf = lam_sdf;
    P.lam_eik = lam_eik;
    P.lam_normal = lam_normal;
    sdf_reg_kernel<<<blocks(int64_t(R[0]) * R[1] * R[2]), 256, 0, stream>>>(P);
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
