// Learned sample proposal (not in the paper): a per-ray MLP predicts how the
// render's weight is spread over B equal bins of the ray's segment in the
// box, and the samples are placed at the quantiles of that density, so that a
// few samples land where uniform marching would need many.
//
//   occupancy_kernel      coarse occupancy grid from the SDF (|s| < threshold)
//   histogram_kernel      per-bin sums of the uniform render's weights w_k
//                         (SDF gathers only: the weights need no colour)
//   proposal_fwd_kernel   [(o-c)/e, d, occupancy at bin centres] -> W -> W -> B
//                         logits, softmax, mixed density, quantile placement
//   proposal_bwd_kernel   cross-entropy to the normalised histogram and its
//                         gradient with respect to the proposal MLP
//
// One thread per ray for the MLP parts (per-ray work, ~1.7 k FMA), one warp per
// ray for the histogram march.
#include "internal.h"
#include "proposal.h"
#include "sample_eval.cuh"

namespace psdf {

namespace {

constexpr int kPB = 8;    // bins
constexpr int kPW = 32;   // hidden width
constexpr int kPIn = 6 + kPB;
constexpr int kPParams = kPW * kPIn + kPW + kPW * kPW + kPW + kPB * kPW + kPB;

__device__ __forceinline__ float grid_sdf_node(const GridView& g, int idx)
{
    return g.sdf ? __ldg(g.sdf + idx) : __ldg(reinterpret_cast<const float*>(g.nodes + idx));
}

__global__ void occupancy_kernel(GridView g, int rx, int ry, int rz, float threshold,
                                 float* __restrict__ occ)
{
    const int n = rx * ry * rz;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n;
         cell += gridDim.x * blockDim.x) {
        const int c[3] = {cell % rx, (cell / rx) % ry, cell / (rx * ry)};
        const int res[3] = {rx, ry, rz};
        int lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const long long span = g.R[a] - 1;
            lo[a] = static_cast<int>((c[a] * span) / res[a]);
            hi[a] = static_cast<int>(((c[a] + 1) * span + res[a] - 1) / res[a]);
            hi[a] = min(hi[a], g.R[a] - 1);
        }
        float mn = INFINITY;
        for (int iz = lo[2]; iz <= hi[2]; ++iz)
            for (int iy = lo[1]; iy <= hi[1]; ++iy)
                for (int ix = lo[0]; ix <= hi[0]; ++ix)
                    mn = fminf(mn, fabsf(grid_sdf_node(g, (iz * g.R[1] + iy) * g.R[0] + ix)));
        occ[cell] = mn < threshold ? 1.0f : 0.0f;
    }
}

// One warp per ray: the uniform render's opacities from the SDF alone, the
// chunk transmittance by a warp scan, per-bin sums of w_k.
__global__ void histogram_kernel(RenderArgs A, int n_bins, float* __restrict__ hist)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int N = A.n_samples, per_bin = N / n_bins;
    const unsigned FULL = 0xffffffffu;
    for (int64_t ray = warp0; ray < A.n_rays; ray += nwarps) {
        const RayIn R = load_ray(A, ray);
        float o[3], d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = R.o[a];
            d[a] = R.d[a];
        }
        float tn, tf;
        const bool hit = ray_box(o, d, A.grid, tn, tf);
        float bins_acc = 0.0f;  // lane b < n_bins accumulates bin b
        if (hit) {
            const float dt = __fdiv_rn(__fsub_rn(tf, tn), static_cast<float>(N));
            float carry = 0.0f, comp = 0.0f;
            for (int base = 0; base < N; base += 32) {
                const int k = base + lane;
                const bool active = k < N;
                float x[3];
                point_at(o, d, sample_t(active ? k : N, dt, tn), x);
                const float s = sdf_value(A.grid, locate(x, A.grid.bmin, A.grid.sc, A.grid.R));
                float s_next = __shfl_down_sync(FULL, s, 1);
                if (active && (lane == 31 || k + 1 >= N)) {
                    point_at(o, d, sample_t(k + 1, dt, tn), x);
                    s_next = sdf_value(A.grid, locate(x, A.grid.bmin, A.grid.sc, A.grid.R));
                }
                float lam = 0.0f;
                if (active) {
                    const float diff = log_transmittance(A.tau, s, s_next);
                    lam = diff < 0.0f ? diff : 0.0f;
                }
                float incl = lam;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float v = __shfl_up_sync(FULL, incl, off);
                    if (lane >= off) incl += v;
                }
                float excl = __shfl_up_sync(FULL, incl, 1);
                if (lane == 0) excl = 0.0f;
                const float total = __shfl_sync(FULL, incl, 31);
                const float w = active ? expf((carry - comp) + excl) * -expm1f(lam) : 0.0f;
                const int my_bin = active ? k / per_bin : -1;
                for (int b = base / per_bin; b <= min(n_bins - 1, (base + 31) / per_bin); ++b) {
                    float v = my_bin == b ? w : 0.0f;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
                    if (lane == b) bins_acc += v;
                }
                const float y = total - comp;
                const float tt = carry + y;
                comp = (tt - carry) - y;
                carry = tt;
            }
        }
        if (lane < n_bins) hist[ray * n_bins + lane] = bins_acc;
    }
}

struct PropArgs {
    GridView grid;
    int occ_res[3];
    const float* __restrict__ occ;
    const float* __restrict__ params;
    float mix, theta;
    const float* __restrict__ rays_o;
    const float* __restrict__ rays_d;
    int64_t n_rays;
    int n_out;
    float* t_samples;
    float* probs;
    const float* __restrict__ hist;
    float min_mass, scale;
    float* grad;
    float* loss;
};

__device__ __forceinline__ float occ_sample(const PropArgs& P, const float x[3])
{
    int i[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int r = P.occ_res[a];
        float u = (x[a] - P.grid.bmin[a]) / (P.grid.bmax[a] - P.grid.bmin[a]) * r - 0.5f;
        u = fminf(fmaxf(u, 0.0f), static_cast<float>(r - 1));
        int fl = static_cast<int>(floorf(u));
        fl = max(0, min(fl, r - 2));
        i[a] = fl;
        f[a] = r > 1 ? u - fl : 0.0f;
    }
    float v = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        const int jx = P.occ_res[0] > 1 ? i[0] + cx : 0;
        const int jy = P.occ_res[1] > 1 ? i[1] + cy : 0;
        const int jz = P.occ_res[2] > 1 ? i[2] + cz : 0;
        const float w =
            (cx ? f[0] : 1 - f[0]) * (cy ? f[1] : 1 - f[1]) * (cz ? f[2] : 1 - f[2]);
        v = fmaf(w, __ldg(P.occ + (jz * P.occ_res[1] + jy) * P.occ_res[0] + jx), v);
    }
    return v;
}

struct PropState {
    bool hit;
    float tn, tf;
    float x[kPIn], h1[kPW], h2[kPW], p[kPB];
    uint32_t m1, m2;  // ReLU masks
};

__device__ __forceinline__ void proposal_eval(const PropArgs& P, const float* sw, int64_t ray,
                                              PropState& S)
{
    float o[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(P.rays_o + 3 * ray + a);
        d[a] = __ldg(P.rays_d + 3 * ray + a);
    }
    S.hit = ray_box(o, d, P.grid, S.tn, S.tf);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c = 0.5f * (P.grid.bmin[a] + P.grid.bmax[a]);
        S.x[a] = (o[a] - c) / (P.grid.bmax[a] - P.grid.bmin[a]);
        S.x[3 + a] = d[a];
    }
#pragma unroll
    for (int b = 0; b < kPB; ++b) {
        float v = 0.0f;
        if (S.hit) {
            const float tb = S.tn + (b + 0.5f) * (S.tf - S.tn) / kPB;
            float xw[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) xw[a] = fmaf(tb, d[a], o[a]);
            v = occ_sample(P, xw);
        }
        S.x[6 + b] = v;
    }
    const float* W1 = sw;
    const float* b1 = W1 + kPW * kPIn;
    const float* W2 = b1 + kPW;
    const float* b2 = W2 + kPW * kPW;
    const float* W3 = b2 + kPW;
    const float* b3 = W3 + kPB * kPW;
    S.m1 = S.m2 = 0;
#pragma unroll
    for (int u = 0; u < kPW; ++u) {
        float z = b1[u];
#pragma unroll
        for (int i = 0; i < kPIn; ++i) z = fmaf(W1[u * kPIn + i], S.x[i], z);
        S.m1 |= (z > 0.0f ? 1u : 0u) << u;
        S.h1[u] = fmaxf(z, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < kPW; ++u) {
        float z = b2[u];
#pragma unroll
        for (int i = 0; i < kPW; ++i) z = fmaf(W2[u * kPW + i], S.h1[i], z);
        S.m2 |= (z > 0.0f ? 1u : 0u) << u;
        S.h2[u] = fmaxf(z, 0.0f);
    }
    float mx = -INFINITY, l[kPB];
#pragma unroll
    for (int b = 0; b < kPB; ++b) {
        float z = b3[b];
#pragma unroll
        for (int i = 0; i < kPW; ++i) z = fmaf(W3[b * kPW + i], S.h2[i], z);
        l[b] = z;
        mx = fmaxf(mx, z);
    }
    float sum = 0.0f;
#pragma unroll
    for (int b = 0; b < kPB; ++b) {
        S.p[b] = expf(l[b] - mx);
        sum += S.p[b];
    }
    const float inv = 1.0f / sum;
#pragma unroll
    for (int b = 0; b < kPB; ++b) S.p[b] *= inv;
}

__global__ void proposal_fwd_kernel(PropArgs P)
{
    __shared__ float sw[kPParams];
    for (int i = threadIdx.x; i < kPParams; i += blockDim.x) sw[i] = P.params[i];
    __syncthreads();
    for (int64_t ray = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; ray < P.n_rays;
         ray += int64_t(gridDim.x) * blockDim.x) {
        PropState S;
        proposal_eval(P, sw, ray, S);
        float q[kPB], qmax = 0.0f;
#pragma unroll
        for (int b = 0; b < kPB; ++b) {
            q[b] = (1.0f - P.mix) * S.p[b] + P.mix / kPB;
            qmax = fmaxf(qmax, q[b]);
        }
        if (qmax < P.theta) {
#pragma unroll
            for (int b = 0; b < kPB; ++b) q[b] = 1.0f / kPB;
        }
        if (P.probs) {
#pragma unroll
            for (int b = 0; b < kPB; ++b) P.probs[ray * kPB + b] = q[b];
        }
        float* t = P.t_samples + ray * (P.n_out + 1);
        if (!S.hit) {
            for (int k = 0; k <= P.n_out; ++k) t[k] = 0.0f;
            continue;
        }
        // samples at the quantiles k / n_out of the piecewise-constant density
        const float db = (S.tf - S.tn) / kPB;
        int b = 0;
        float c = 0.0f;
        for (int k = 0; k <= P.n_out; ++k) {
            const float u = static_cast<float>(k) / P.n_out;
            while (b < kPB - 1 && c + q[b] <= u) {
                c += q[b];
                ++b;
            }
            const float frac = fminf((u - c) / q[b], 1.0f);
            t[k] = fmaf(b + frac, db, S.tn);
        }
        t[0] = S.tn;
        t[P.n_out] = S.tf;
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void proposal_bwd_kernel(PropArgs P)
{
    __shared__ float sw[kPParams];
    __shared__ float acc[kPParams];
    for (int i = threadIdx.x; i < kPParams; i += blockDim.x) {
        sw[i] = P.params[i];
        acc[i] = 0.0f;
    }
    __syncthreads();
    const float* W2 = sw + kPW * kPIn + kPW;
    const float* W3 = W2 + kPW * kPW + kPW;
    float* gW1 = acc;
    float* gb1 = gW1 + kPW * kPIn;
    float* gW2 = gb1 + kPW;
    float* gb2 = gW2 + kPW * kPW;
    float* gW3 = gb2 + kPW;
    float* gb3 = gW3 + kPB * kPW;
    const int lane = threadIdx.x & 31;
    // whole warps iterate together so that the per-parameter warp sums below
    // see every lane; lanes past the end contribute zeros
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < P.n_rays;
         base += stride) {
        const int64_t ray = base + lane;
        PropState S;
        float dl[kPB];
        bool valid = false;
        if (ray < P.n_rays) {
            float mass = 0.0f;
#pragma unroll
            for (int b = 0; b < kPB; ++b) mass += __ldg(P.hist + ray * kPB + b);
            valid = mass >= P.min_mass;
            float ce = 0.0f;
            if (valid) {
                proposal_eval(P, sw, ray, S);
#pragma unroll
                for (int b = 0; b < kPB; ++b) {
                    const float tgt = __ldg(P.hist + ray * kPB + b) / mass;
                    ce -= tgt * logf(S.p[b]);
                    dl[b] = P.scale * (S.p[b] - tgt);
                }
            }
            if (P.loss) P.loss[ray] = ce;
        }
        if (!valid) {
#pragma unroll
            for (int b = 0; b < kPB; ++b) dl[b] = 0.0f;
#pragma unroll
            for (int i = 0; i < kPW; ++i) S.h1[i] = S.h2[i] = 0.0f;
#pragma unroll
            for (int i = 0; i < kPIn; ++i) S.x[i] = 0.0f;
            S.m1 = S.m2 = 0;
        }
        // layer 3
#pragma unroll
        for (int b = 0; b < kPB; ++b) {
            const float sb = warp_sum(dl[b]);
            if (lane == 0) atomicAdd(gb3 + b, sb);
#pragma unroll
            for (int i = 0; i < kPW; ++i) {
                const float v = warp_sum(dl[b] * S.h2[i]);
                if (lane == 0) atomicAdd(gW3 + b * kPW + i, v);
            }
        }
        float dz2[kPW];
#pragma unroll
        for (int i = 0; i < kPW; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int b = 0; b < kPB; ++b) a = fmaf(W3[b * kPW + i], dl[b], a);
            dz2[i] = ((S.m2 >> i) & 1u) ? a : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kPW; ++u) {
            const float sb = warp_sum(dz2[u]);
            if (lane == 0) atomicAdd(gb2 + u, sb);
#pragma unroll
            for (int i = 0; i < kPW; ++i) {
                const float v = warp_sum(dz2[u] * S.h1[i]);
                if (lane == 0) atomicAdd(gW2 + u * kPW + i, v);
            }
        }
        float dz1[kPW];
#pragma unroll
        for (int i = 0; i < kPW; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int u = 0; u < kPW; ++u) a = fmaf(W2[u * kPW + i], dz2[u], a);
            dz1[i] = ((S.m1 >> i) & 1u) ? a : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kPW; ++u) {
            const float sb = warp_sum(dz1[u]);
            if (lane == 0) atomicAdd(gb1 + u, sb);
#pragma unroll
            for (int i = 0; i < kPIn; ++i) {
                const float v = warp_sum(dz1[u] * S.x[i]);
                if (lane == 0) atomicAdd(gW1 + u * kPIn + i, v);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPParams; i += blockDim.x) red_add(P.grad + i, acc[i]);
}

int blocks_for(int64_t n, int threads, int cap)
{
    const int64_t b = (n + threads - 1) / threads;
    return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

int proposal_param_count() { return kPParams; }
int proposal_bins() { return kPB; }
int proposal_width() { return kPW; }

cudaError_t launch_occupancy(const GridView& g, const int res[3], float threshold, float* occ,
                             cudaStream_t stream)
{
    const int n = res[0] * res[1] * res[2];
    occupancy_kernel<<<blocks_for(n, 128, 8 * sm_count()), 128, 0, stream>>>(
        g, res[0], res[1], res[2], threshold, occ);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const RenderArgs& A, int n_bins, float* hist, cudaStream_t stream)
{
    const int64_t warps = A.n_rays;
    histogram_kernel<<<blocks_for(warps * 32, 256, 16 * sm_count()), 256, 0, stream>>>(
        A, n_bins, hist);
    return cudaGetLastError();
}

cudaError_t launch_proposal_forward(const ProposalLaunch& L, cudaStream_t stream)
{
    PropArgs P;
    P.grid = L.grid;
    for (int a = 0; a < 3; ++a) P.occ_res[a] = L.occ_res[a];
    P.occ = L.occ;
    P.params = L.params;
    P.mix = L.mix;
    P.theta = L.theta;
    P.rays_o = L.rays_o;
    P.rays_d = L.rays_d;
    P.n_rays = L.n_rays;
    P.n_out = L.n_out;
    P.t_samples = L.t_samples;
    P.probs = L.probs;
    P.hist = nullptr;
    P.grad = nullptr;
    P.loss = nullptr;
    proposal_fwd_kernel<<<blocks_for(L.n_rays, 128, 16 * sm_count()), 128, 0, stream>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_proposal_backward(const ProposalLaunch& L, cudaStream_t stream)
{
    PropArgs P;
    P.grid = L.grid;
    for (int a = 0; a < 3; ++a) P.occ_res[a] = L.occ_res[a];
    P.occ = L.occ;
    P.params = L.params;
    P.mix = L.mix;
    P.theta = L.theta;
    P.rays_o = L.rays_o;
    P.rays_d = L.rays_d;
    P.n_rays = L.n_rays;
    P.n_out = 0;
    P.t_samples = nullptr;
    P.probs = nullptr;
    P.hist = L.hist;
    P.min_mass = L.min_mass;
    P.scale = L.scale;
    P.grad = L.grad;
    P.loss = L.loss;
    proposal_bwd_kernel<<<blocks_for(L.n_rays, 128, 4 * sm_count()), 128, 0, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace psdf
