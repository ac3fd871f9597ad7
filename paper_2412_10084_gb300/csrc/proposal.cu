// Learned sample proposal (not in the paper): a per-ray MLP predicts how the
// render's weight is spread over B equal bins of the ray's segment in the
// box, and the samples are placed at the quantiles of that density, so that a
// few samples land where uniform marching would need many.
//
//   occupancy_kernel      coarse occupancy bitmask from the SDF (|s| < threshold)
//   histogram_kernel      per-bin sums of the uniform render's weights w_k
//                         (SDF gathers only: the weights need no colour)
//   proposal_fwd_kernel   [(o-c)/e, d, occupied fraction per bin] -> W -> W -> B
//                         logits, softmax, mixed density, quantile placement
//   proposal_bwd_kernel   mass-weighted cross-entropy -sum_b hist_b log p_b and
//                         its gradient with respect to the proposal MLP
//
// One thread per ray for the MLP parts (per-ray work, ~1.7 k FMA), one warp per
// ray for the histogram march.  The proposal kernels keep the occupancy
// bitmask (at most 64^3 bits = 32 KB) in shared memory.
#include "internal.h"
#include "proposal.h"
#include "sample_eval.cuh"

namespace psdf {

namespace {

constexpr int kPW = 32;  // hidden width

// Compiled proposal shapes: B bins, inputs [o (3), d (3), first occupied
// position (1), occupied fraction of each bin (B), share of each bin before
// the first occupied point (B)].
template <int B>
struct PropShape {
    static constexpr int kIn = 7 + 2 * B;
    static constexpr int kParams = kPW * kIn + kPW + kPW * kPW + kPW + B * kPW + B;
    // W1 rows padded to an even length in shared memory, so that every row
    // starts 8-byte aligned and is read two inputs at a time
    static constexpr int kInP = (kIn + 1) & ~1;
    static_assert((kPW * kIn + kPW) % 4 == 0 && (kPW * kPW + kPW) % 4 == 0,
                  "W2 and W3 rows start 16-byte aligned in the packed parameters");
};

// Parameters into shared memory: the packed vector, and W1 with padded rows.
template <int B>
__device__ __forceinline__ void load_prop_params(const float* __restrict__ g, float* sw,
                                                 float* sw1)
{
    constexpr int kIn = PropShape<B>::kIn, kInP = PropShape<B>::kInP;
    for (int i = threadIdx.x; i < PropShape<B>::kParams; i += blockDim.x) sw[i] = g[i];
    for (int i = threadIdx.x; i < kPW * kInP; i += blockDim.x) {
        const int u = i / kInP, j = i % kInP;
        sw1[i] = j < kIn ? g[u * kIn + j] : 0.0f;
    }
}

// SDF of node (x, y, z); in a sparse grid a node of a brick that is not
// stored reads as empty_sdf.
__device__ __forceinline__ float grid_sdf_node(const GridView& g, int x, int y, int z)
{
    if (g.table) {
        const int64_t rec = brick_record(g, x, y, z);
        return rec < 0 ? g.empty_sdf : __ldg(reinterpret_cast<const float*>(g.nodes + rec));
    }
    const int idx = (z * g.R[1] + y) * g.R[0] + x;
    return g.sdf ? __ldg(g.sdf + idx) : __ldg(reinterpret_cast<const float*>(g.nodes + idx));
}

// One bit per cell (bit c & 31 of word c >> 5, c = (z res_y + y) res_x + x):
// a warp builds one word with a ballot.
__global__ void occupancy_kernel(GridView g, int rx, int ry, int rz, float threshold,
                                 uint32_t* __restrict__ bits)
{
    const int n = rx * ry * rz;
    const int words = (n + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const int res[3] = {rx, ry, rz};
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < words;
         w += (gridDim.x * blockDim.x) >> 5) {
        const int cell = (w << 5) + lane;
        bool occupied = false;
        if (cell < n) {
            const int c[3] = {cell % rx, (cell / rx) % ry, cell / (rx * ry)};
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
                        mn = fminf(mn, fabsf(grid_sdf_node(g, ix, iy, iz)));
            occupied = mn < threshold;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, occupied);
        if (lane == 0) bits[w] = word;
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
    int n_sub;
    const uint32_t* __restrict__ occ_bits;
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

// Occupancy features of a ray (x[6] = first occupied position, x[7 + b] =
// occupied share of bin b, x[7 + B + b] = share of bin b before the first
// occupied point): B n_sub points at the centres of equal
// sub-intervals of [t_n, t_f], each looked up in the cell containing it.
// Positions and cell indices use explicitly rounded FP32 operations (they
// decide integers).
template <int B>
__device__ __forceinline__ void ray_occupancy(const PropArgs& P, const uint32_t* bits,
                                              const float o[3], const float d[3], float tn,
                                              float tf, float* x)
{
    const int S = P.n_sub;
    const float seg = __fdiv_rn(__fsub_rn(tf, tn), static_cast<float>(B * S));
    float inv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        inv[a] = __fdiv_rn(static_cast<float>(P.occ_res[a]),
                           __fsub_rn(P.grid.bmax[a], P.grid.bmin[a]));
    int first = -1;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int count = 0;
        for (int j = 0; j < S; ++j) {
            const int k = b * S + j;
            const float t = __fmaf_rn(static_cast<float>(k) + 0.5f, seg, tn);
            int c[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float xa = __fmaf_rn(t, d[a], o[a]);
                float u = __fmul_rn(__fsub_rn(xa, P.grid.bmin[a]), inv[a]);
                u = fminf(fmaxf(u, 0.0f), static_cast<float>(P.occ_res[a] - 1));
                c[a] = static_cast<int>(floorf(u));
            }
            const int cell = (c[2] * P.occ_res[1] + c[1]) * P.occ_res[0] + c[0];
            const uint32_t hit = (bits[cell >> 5] >> (cell & 31)) & 1u;
            if (hit && first < 0) first = k;
            count += hit;
        }
        x[7 + b] = static_cast<float>(count) / static_cast<float>(S);
    }
    x[6] = first < 0 ? 1.0f
                     : (static_cast<float>(first) + 0.5f) / static_cast<float>(B * S);
#pragma unroll
    for (int b = 0; b < B; ++b) x[7 + B + b] = fminf(fmaxf(B * x[6] - b, 0.0f), 1.0f);
}

template <int B>
struct PropState {
    bool hit;
    float tn, tf;
    float x[PropShape<B>::kIn], h1[kPW], h2[kPW], p[B];
    uint32_t m1, m2;  // ReLU masks
};

template <int B>
__device__ __forceinline__ void proposal_eval(const PropArgs& P, const float* sw,
                                              const float* sw1, const uint32_t* bits,
                                              int64_t ray, PropState<B>& S)
{
    constexpr int kIn = PropShape<B>::kIn, kInP = PropShape<B>::kInP;
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
    if (S.hit) {
        ray_occupancy<B>(P, bits, o, d, S.tn, S.tf, S.x);
    } else {
        S.x[6] = 1.0f;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            S.x[7 + b] = 0.0f;
            S.x[7 + B + b] = 1.0f;
        }
    }
    const float* W1 = sw;
    const float* b1 = W1 + kPW * kIn;
    const float* W2 = b1 + kPW;
    const float* b2 = W2 + kPW * kPW;
    const float* W3 = b2 + kPW;
    const float* b3 = W3 + B * kPW;
    (void)W1;
    S.m1 = S.m2 = 0;
    // each layer sums the even and the odd inputs apart, two per paired FMA
    float2 xp[kInP / 2];
#pragma unroll
    for (int i = 0; i < kInP / 2; ++i)
        xp[i] = make_float2(S.x[2 * i], 2 * i + 1 < kIn ? S.x[2 * i + 1] : 0.0f);
#pragma unroll
    for (int u = 0; u < kPW; ++u) {
        float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < kInP / 2; ++i)
            a = fma2(*reinterpret_cast<const float2*>(sw1 + u * kInP + 2 * i), xp[i], a);
        const float z = b1[u] + (a.x + a.y);
        S.m1 |= (z > 0.0f ? 1u : 0u) << u;
        S.h1[u] = fmaxf(z, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < kPW; ++u) {
        float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < kPW; i += 2)
            a = fma2(*reinterpret_cast<const float2*>(W2 + u * kPW + i),
                     make_float2(S.h1[i], S.h1[i + 1]), a);
        const float z = b2[u] + (a.x + a.y);
        S.m2 |= (z > 0.0f ? 1u : 0u) << u;
        S.h2[u] = fmaxf(z, 0.0f);
    }
    float mx = -INFINITY, l[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < kPW; i += 2)
            a = fma2(*reinterpret_cast<const float2*>(W3 + b * kPW + i),
                     make_float2(S.h2[i], S.h2[i + 1]), a);
        const float z = b3[b] + (a.x + a.y);
        l[b] = z;
        mx = fmaxf(mx, z);
    }
    float sum = 0.0f;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        S.p[b] = expf(l[b] - mx);
        sum += S.p[b];
    }
    const float rsum = 1.0f / sum;
#pragma unroll
    for (int b = 0; b < B; ++b) S.p[b] *= rsum;
}

__device__ __forceinline__ int occ_words(const PropArgs& P)
{
    return (P.occ_res[0] * P.occ_res[1] * P.occ_res[2] + 31) >> 5;
}

// Parameters (and, for the adjoint, their accumulators) in static shared
// memory, the occupancy bitmask in dynamic shared memory.
template <int B>
__global__ void proposal_fwd_kernel(PropArgs P)
{
    constexpr int kParams = PropShape<B>::kParams;
    constexpr int kRow = 2 * B + 4;  // per ray: c_0..c_B, 1/q_0..1/q_{B-1}, hit, t_n, t_f
    __shared__ __align__(16) float sw[kParams];
    __shared__ __align__(16) float sw1[kPW * PropShape<B>::kInP];
    __shared__ float srow[4 * 32 * kRow];
    extern __shared__ uint32_t sbits[];
    load_prop_params<B>(P.params, sw, sw1);
    for (int i = threadIdx.x; i < occ_words(P); i += blockDim.x) sbits[i] = P.occ_bits[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    // whole warps iterate together: each lane evaluates one ray, then the warp
    // writes the 32 rays' sample rows one after another, lane k writing
    // samples k, k + 32, ... (coalesced stores)
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < P.n_rays;
         base += stride) {
        const int64_t ray = base + lane;
        const bool live = ray < P.n_rays;
        PropState<B> S;
        float q[B];
        S.hit = false;
        S.tn = S.tf = 0.0f;
#pragma unroll
        for (int b = 0; b < B; ++b) q[b] = 1.0f / B;
        if (live) {
            proposal_eval<B>(P, sw, sw1, sbits, ray, S);
            // mix share: a quarter on every bin, three quarters on the occupied
            // bins and their neighbours (all of it uniformly when none is
            // occupied)
            float qmax = 0.0f;
            int nr = 0;
            uint32_t near = 0;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const bool nb = S.x[7 + b] > 0.0f || (b > 0 && S.x[6 + b] > 0.0f) ||
                                (b + 1 < B && S.x[8 + b] > 0.0f);
                near |= (nb ? 1u : 0u) << b;
                nr += nb;
            }
            const float share = nr > 0 ? 0.75f * P.mix / nr : 0.0f;
            const float floor_b = nr > 0 ? 0.25f * P.mix / B : P.mix / B;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const float rb = floor_b + (((near >> b) & 1u) ? share : 0.0f);
                q[b] = (1.0f - P.mix) * S.p[b] + rb;
                qmax = fmaxf(qmax, q[b]);
            }
            if (qmax < P.theta) {
#pragma unroll
                for (int b = 0; b < B; ++b) q[b] = 1.0f / B;
            }
            if (P.probs) {
#pragma unroll
                for (int b = 0; b < B; ++b) P.probs[ray * B + b] = q[b];
            }
        }
        if (!P.t_samples) continue;  // densities only (the render places the samples)
        // each lane stages its ray's density q_b and running sums c_b (summed in
        // bin order, as the inverse CDF below defines them) for the row writes
        float* cq = srow + (threadIdx.x >> 5) * 32 * kRow + lane * kRow;
        {
            float c = 0.0f;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                cq[b] = c;
                cq[B + 1 + b] = 1.0f / q[b];
                c += q[b];
            }
            cq[B] = c;
            cq[2 * B + 1] = __int_as_float(S.hit ? 1 : 0);
            cq[2 * B + 2] = S.tn;
            cq[2 * B + 3] = S.tf;
        }
        __syncwarp();
        const int64_t left = P.n_rays - base;
        const int rows = left < 32 ? static_cast<int>(left) : 32;
        for (int r = 0; r < rows; ++r) {
            const float* row = srow + (threadIdx.x >> 5) * 32 * kRow + r * kRow;
            const bool hit = __float_as_int(row[2 * B + 1]) != 0;
            const float tn = row[2 * B + 2], tf = row[2 * B + 3];
            float* t = P.t_samples + (base + r) * (P.n_out + 1);
            // samples at the quantiles k / n_out of the piecewise-constant
            // density: bin b = the last with c_b <= u (binary search), which is
            // where the walk "advance while c_b + q_b <= u" stops; the
            // reciprocals 1 / n_out and 1 / q_b are rounded once (the render's
            // bin-density placement uses the same expressions)
            const float db = (tf - tn) / B;
            const float inv_n = 1.0f / P.n_out;
            for (int k = lane; k <= P.n_out; k += 32) {
                float v = 0.0f;
                if (hit) {
                    const float u = static_cast<float>(k) * inv_n;
                    int b = 0;
#pragma unroll
                    for (int step = B / 2; step > 0; step >>= 1)
                        if (b + step < B && row[b + step] <= u) b += step;
                    const float frac = fminf((u - row[b]) * row[B + 1 + b], 1.0f);
                    v = k == 0 ? tn : (k == P.n_out ? tf : fmaf(b + frac, db, tn));
                }
                t[k] = v;
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int B>
__global__ void proposal_bwd_kernel(PropArgs P)
{
    constexpr int kIn = PropShape<B>::kIn;
    constexpr int kParams = PropShape<B>::kParams;
    __shared__ __align__(16) float sw[kParams];
    __shared__ __align__(16) float sw1[kPW * PropShape<B>::kInP];
    __shared__ float acc[kParams];
    extern __shared__ uint32_t sbits[];
    load_prop_params<B>(P.params, sw, sw1);
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) acc[i] = 0.0f;
    for (int i = threadIdx.x; i < occ_words(P); i += blockDim.x) sbits[i] = P.occ_bits[i];
    __syncthreads();
    const float* W2 = sw + kPW * kIn + kPW;
    const float* W3 = W2 + kPW * kPW + kPW;
    float* gW1 = acc;
    float* gb1 = gW1 + kPW * kIn;
    float* gW2 = gb1 + kPW;
    float* gb2 = gW2 + kPW * kPW;
    float* gW3 = gb2 + kPW;
    float* gb3 = gW3 + B * kPW;
    const int lane = threadIdx.x & 31;
    // whole warps iterate together so that the per-parameter warp sums below
    // see every lane; lanes past the end contribute zeros
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < P.n_rays;
         base += stride) {
        const int64_t ray = base + lane;
        PropState<B> S;
        float dl[B];
        bool valid = false;
        if (ray < P.n_rays) {
            float mass = 0.0f;
#pragma unroll
            for (int b = 0; b < B; ++b) mass += __ldg(P.hist + ray * B + b);
            valid = mass >= P.min_mass;
            float ce = 0.0f;
            if (valid) {
                proposal_eval<B>(P, sw, sw1, sbits, ray, S);
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const float h = __ldg(P.hist + ray * B + b);
                    ce -= h * logf(S.p[b]);
                    dl[b] = P.scale * (mass * S.p[b] - h);
                }
            }
            if (P.loss) P.loss[ray] = ce;
        }
        if (!valid) {
#pragma unroll
            for (int b = 0; b < B; ++b) dl[b] = 0.0f;
#pragma unroll
            for (int i = 0; i < kPW; ++i) S.h1[i] = S.h2[i] = 0.0f;
#pragma unroll
            for (int i = 0; i < kIn; ++i) S.x[i] = 0.0f;
            S.m1 = S.m2 = 0;
        }
        // layer 3
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const float sb = warp_sum(dl[b]);
            if (lane == 0) atomicAdd(gb3 + b, sb);
#pragma unroll 4
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
            for (int b = 0; b < B; ++b) a = fmaf(W3[b * kPW + i], dl[b], a);
            dz2[i] = ((S.m2 >> i) & 1u) ? a : 0.0f;
        }
#pragma unroll 4
        for (int u = 0; u < kPW; ++u) {
            const float sb = warp_sum(dz2[u]);
            if (lane == 0) atomicAdd(gb2 + u, sb);
#pragma unroll 4
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
#pragma unroll 4
        for (int u = 0; u < kPW; ++u) {
            const float sb = warp_sum(dz1[u]);
            if (lane == 0) atomicAdd(gb1 + u, sb);
#pragma unroll
            for (int i = 0; i < kIn; ++i) {
                const float v = warp_sum(dz1[u] * S.x[i]);
                if (lane == 0) atomicAdd(gW1 + u * kIn + i, v);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) red_add(P.grad + i, acc[i]);
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

int proposal_param_count(int n_bins)
{
    switch (n_bins) {
        case 8: return PropShape<8>::kParams;
        case 16: return PropShape<16>::kParams;
        default: return 0;
    }
}
bool proposal_bins_supported(int n_bins) { return n_bins == 8 || n_bins == 16; }
int proposal_width() { return kPW; }

int occupancy_words(const int res[3]) { return (res[0] * res[1] * res[2] + 31) / 32; }

cudaError_t launch_occupancy(const GridView& g, const int res[3], float threshold,
                             uint32_t* bits, cudaStream_t stream)
{
    const int words = occupancy_words(res);
    occupancy_kernel<<<blocks_for(int64_t(words) * 32, 128, 8 * sm_count()), 128, 0, stream>>>(
        g, res[0], res[1], res[2], threshold, bits);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const RenderArgs& A, int n_bins, float* hist, cudaStream_t stream)
{
    const int64_t warps = A.n_rays;
    histogram_kernel<<<blocks_for(warps * 32, 256, 16 * sm_count()), 256, 0, stream>>>(
        A, n_bins, hist);
    return cudaGetLastError();
}

namespace {

PropArgs prop_args(const ProposalLaunch& L)
{
    PropArgs P;
    P.grid = L.grid;
    for (int a = 0; a < 3; ++a) P.occ_res[a] = L.occ_res[a];
    P.n_sub = L.n_sub;
    P.occ_bits = L.occ_bits;
    P.params = L.params;
    P.mix = L.mix;
    P.theta = L.theta;
    P.rays_o = L.rays_o;
    P.rays_d = L.rays_d;
    P.n_rays = L.n_rays;
    P.n_out = L.n_out;
    P.t_samples = L.t_samples;
    P.probs = L.probs;
    P.hist = L.hist;
    P.min_mass = L.min_mass;
    P.scale = L.scale;
    P.grad = L.grad;
    P.loss = L.loss;
    return P;
}

// Static parameter storage plus a bitmask of up to 32 KB can pass the 48 KB
// default: opt in to the dynamic size the launch needs.
template <class K>
cudaError_t allow_smem(K kernel, size_t dynamic)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(dynamic));
}

template <int B>
cudaError_t launch_fwd(const PropArgs& P, cudaStream_t stream)
{
    const size_t smem = sizeof(uint32_t) * occupancy_words(P.occ_res);
    cudaError_t e = allow_smem(proposal_fwd_kernel<B>, smem);
    if (e != cudaSuccess) return e;
    proposal_fwd_kernel<B><<<blocks_for(P.n_rays, 128, 16 * sm_count()), 128, smem, stream>>>(P);
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_bwd(const PropArgs& P, cudaStream_t stream)
{
    const size_t smem = sizeof(uint32_t) * occupancy_words(P.occ_res);
    cudaError_t e = allow_smem(proposal_bwd_kernel<B>, smem);
    if (e != cudaSuccess) return e;
    proposal_bwd_kernel<B><<<blocks_for(P.n_rays, 128, 4 * sm_count()), 128, smem, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_proposal_forward(const ProposalLaunch& L, cudaStream_t stream)
{
    const PropArgs P = prop_args(L);
    return L.n_bins == 16 ? launch_fwd<16>(P, stream) : launch_fwd<8>(P, stream);
}

cudaError_t launch_proposal_backward(const ProposalLaunch& L, cudaStream_t stream)
{
    const PropArgs P = prop_args(L);
    return L.n_bins == 16 ? launch_bwd<16>(P, stream) : launch_bwd<8>(P, stream);
}

}  // namespace psdf
