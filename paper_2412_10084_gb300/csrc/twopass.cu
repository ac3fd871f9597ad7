// Two-pass inference (the paper's viewer, Tab. 8: "shading" gives every voxel
// a colour for the current view, then "render" marches the SDF and the colour
// field), sm_103a.
//
//   shade_kernel<C>       persistent CTAs of 4 warps.  Each round the CTA tests
//                         128 nodes against the band |s| < band: the others get
//                         colour 0, band nodes are appended to a shared-memory
//                         queue; every full 128 queue entries form one M = 128
//                         tile: central-difference normal, view vector to the
//                         camera, node features, probe-blended SH features and
//                         Fresnel inputs, then the MLP on the tensor cores
//                         exactly as in the forward render.  Colours are stored
//                         as FP16 {r, g, b, 0} (8 bytes per node).
//   colour_render_kernel  warp per ray, lane per sample, 32-sample chunks: the
//                         forward's sample placement, opacity and compositing,
//                         with a sample's colour the trilinear blend of the 8
//                         node colours of its cell (gathered only where alpha > 0).
#include <cuda_fp16.h>

#include "internal.h"
#include "mlp_tc.cuh"

namespace psdf {

namespace {

template <class C>
struct ShadeLayout {
    using M = MlpTC<C>;
    static constexpr int K1 = M::K1;
    static constexpr int kXT = 128 * K1 * 2;    // one split of the input tile [128][16]
    static constexpr int kHT = 128 * C::W * 2;  // one split of the hidden tile [128][W]
    static constexpr int oW = 0;
    static constexpr int oF32 = oW + M::kWeightBytes;
    static constexpr int oX = (oF32 + 4 * M::kF32 + 127) & ~127;
    static constexpr int oH = oX + M::kSplit * kXT;
    static constexpr int oQ = oH + M::kSplit * kHT;  // node queue: 256 entries + count
    static constexpr int oBar = oQ + 256 * 4 + 16;
    static constexpr int kBytes = oBar + 16;
    static constexpr uint32_t kTmemCols = 64;  // layer 1 at column 0, layer 2 at 32
};

// SDF of the node with linear index i (x fastest); in a sparse grid a node of
// a brick that is not stored reads as empty_sdf.
__device__ __forceinline__ float node_sdf(const GridView& g, int64_t i)
{
    if (g.table) {
        const int x = static_cast<int>(i % g.R[0]), y = static_cast<int>((i / g.R[0]) % g.R[1]);
        const int z = static_cast<int>(i / (int64_t(g.R[0]) * g.R[1]));
        const int64_t rec = brick_record(g, x, y, z);
        return rec < 0 ? g.empty_sdf : __ldg(reinterpret_cast<const float*>(g.nodes + rec));
    }
    return g.sdf ? __ldg(g.sdf + i) : __ldg(reinterpret_cast<const float*>(g.nodes + i));
}

// MLP inputs of grid node `node` seen from the camera.
template <class C>
__device__ __forceinline__ void node_inputs(const RenderArgs& A, const ShadeArgs& S, int64_t node,
                                            float* x)
{
    const GridView& g = A.grid;
    const int i[3] = {static_cast<int>(node % g.R[0]), static_cast<int>((node / g.R[0]) % g.R[1]),
                      static_cast<int>(node / (int64_t(g.R[0]) * g.R[1]))};
    const int64_t step[3] = {1, g.R[0], int64_t(g.R[0]) * g.R[1]};
    SampleGeom<C> G;
    // gradient: central differences, one-sided on the grid's faces
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int up = i[a] + 1 < g.R[a] ? 1 : 0, dn = i[a] > 0 ? 1 : 0;
        const float sp = node_sdf(g, node + up * step[a]);
        const float sm = node_sdf(g, node - dn * step[a]);
        G.g[a] = (sp - sm) / (static_cast<float>(up + dn) * S.h[a]);
    }
    float xw[3], v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xw[a] = fmaf(static_cast<float>(i[a]), S.h[a], g.bmin[a]);
        v[a] = S.cam[a] - xw[a];
    }
    const float inv = 1.0f / sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] *= inv;
    // the node's spatial features
    if constexpr (C::TP) {
        const float u[3] = {static_cast<float>(i[0]), static_cast<float>(i[1]),
                            static_cast<float>(i[2])};
        TriAt T;
        triplane_locate_u(g, u, T);
        triplane_lookup(g, T, G.x);
    } else if constexpr (C::FB) {
        const uint2 f = __ldg(g.feat16 + node);
        G.x[0] = bf16_lo(f.x);
        G.x[1] = bf16_hi(f.x);
        G.x[2] = bf16_lo(f.y);
    } else if constexpr (C::SP) {
        const int64_t rec = brick_record(g, i[0], i[1], i[2]);
        const float4 r = rec >= 0 ? __ldg(g.nodes + rec) : make_float4(0.f, 0.f, 0.f, 0.f);
        G.x[0] = r.y;
        G.x[1] = r.z;
        G.x[2] = r.w;
    } else {
        const float4 r = __ldg(g.nodes + node);
        G.x[0] = r.y;
        G.x[1] = r.z;
        G.x[2] = r.w;
    }
    eval_appearance_at<C>(A, xw, v, G);
#pragma unroll
    for (int k = 0; k < C::NINP; ++k) x[k] = G.x[k];
}

__device__ __forceinline__ uint2 pack_colour(const float c[3])
{
    const __half2 rg = __floats2half2_rn(c[0], c[1]);
    const __half2 b0 = __floats2half2_rn(c[2], 0.0f);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&rg),
                      *reinterpret_cast<const uint32_t*>(&b0));
}

template <class C>
__global__ void __launch_bounds__(kFwdThreads, 4) shade_kernel(RenderArgs A, ShadeArgs S)
{
    using M = MlpTC<C>;
    using L = ShadeLayout<C>;
    constexpr int W = C::W;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* wt = smem + L::oW;
    float* f32 = reinterpret_cast<float*>(smem + L::oF32);
    uint8_t* xh = smem + L::oX;
    uint8_t* xl = xh + L::kXT;
    uint8_t* hh = smem + L::oH;
    uint8_t* hl = hh + L::kHT;
    int* queue = reinterpret_cast<int*>(smem + L::oQ);
    int* qcount = queue + 256;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::oBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::oBar + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    load_mlp_tc<C>(A.mlp, wt, f32);
    if (warp == 0) tc::tmem_alloc(tslot, L::kTmemCols);
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        *qcount = 0;
    }
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * warp) << 16);
    uint32_t phase = 0;
    bool bad = false;
    const unsigned FULL = 0xffffffffu;
    const int64_t n_nodes = int64_t(A.grid.R[0]) * A.grid.R[1] * A.grid.R[2];

    for (int64_t base = int64_t(blockIdx.x) * 128;; base += int64_t(gridDim.x) * 128) {
        const bool more = base < n_nodes;  // CTA-uniform
        if (more) {
            // band test of 128 nodes; band nodes join the queue (fewer than 128
            // entries are waiting, so the queue never holds more than 255)
            const int64_t node = base + tid;
            bool in_band = false;
            if (node < n_nodes) {
                in_band = fabsf(node_sdf(A.grid, node)) < S.band;
                if (!in_band) S.colours[node] = make_uint2(0u, 0u);
            }
            const unsigned m = __ballot_sync(FULL, in_band);
            int off = 0;
            if (lane == 0 && m) off = atomicAdd(qcount, __popc(m));
            off = __shfl_sync(FULL, off, 0);
            if (in_band) queue[off + __popc(m & ((1u << lane) - 1u))] = static_cast<int>(node);
        }
        __syncthreads();
        int count = *qcount;
        __syncthreads();  // read by all before the next round's appends
        while (count >= 128 || (!more && count > 0)) {
            const int batch = count < 128 ? count : 128;
            const int node = tid < batch ? queue[tid] : -1;
            // ---- inputs of the tile's rows ----
            if (node >= 0) {
                float xin[M::K1];
                float xr[C::NINP];
                node_inputs<C>(A, S, node, xr);
#pragma unroll
                for (int k = 0; k < M::K1; ++k) xin[k] = k < C::NIN ? xr[k] : 0.0f;
                store_row<M::K1, M::kSplit>(xh, xl, tid, 0, M::K1, xin);
            } else {
                zero_row<M::K1, M::kSplit>(xh, xl, tid, 0, M::K1);
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            if (__syncthreads_or(bad)) goto done;
            tc::fence_after();
            // ---- layer 1 on the tensor cores ----
            if (tid == 0) {
                mma_k<M::kSplit>(tmem + 0, xh, xl, M::w1h(wt), M::w1l(wt), 128,
                                 (M::K1 / 8) * 128, 128, (M::K1 / 8) * 128, M::kIdescL, false);
                tc::commit(mbar);
            }
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            {
                float z[W];
                tc::tmem_ld<W>(t_row + 0, z);
                bias_relu<W>(z, f32 + M::kB1);
                store_row<W, M::kSplit>(hh, hl, tid, 0, W, z);
            }
            tc::fence_smem_to_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            // ---- layer 2 on the tensor cores, layer 3 on the CUDA cores ----
            if (tid == 0) {
#pragma unroll
                for (int s = 0; s < W / 16; ++s)
                    mma_k<M::kSplit>(tmem + 32, hh + s * 256, hl + s * 256,
                                     M::w2h(wt) + s * 256, M::w2l(wt) + s * 256, 128,
                                     (W / 8) * 128, 128, (W / 8) * 128, M::kIdescL, s > 0);
                tc::commit(mbar);
            }
            bad |= !tc::mbar_wait(mbar, phase, A.wait_polls);
            phase ^= 1;
            tc::fence_after();
            {
                float z[W];
                tc::tmem_ld<W>(t_row + 32, z);
                bias_relu<W>(z, f32 + M::kB2);
                float col[3];
                mlp_layer3<C>(f32, z, col);
                if (node >= 0) S.colours[node] = pack_colour(col);
            }
            tc::fence_before();
            // ---- drop the tile's entries from the queue ----
            const int rest = count - batch;
            const int moved = tid < rest ? queue[128 + tid] : 0;
            __syncthreads();
            if (tid < rest) queue[tid] = moved;
            if (tid == 0) *qcount = rest;
            __syncthreads();
            count = rest;
        }
        if (!more) break;
    }
done:
    bad = __syncthreads_or(bad);
    if (bad) {
        // an MMA never signalled completion: give it one more bounded wait
        // before the tensor memory is released, and report the failure
        // the last commit's phase has the parity before the final flip
        tc::mbar_wait(mbar, phase ^ 1u);
        if (tid == 0) atomicOr(A.status, 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, L::kTmemCols);
}

constexpr int kRenderWarps = 8;

__global__ void __launch_bounds__(kRenderWarps * 32) colour_render_kernel(
    RenderArgs A, const uint2* __restrict__ colours)
{
    __shared__ float tab[kRenderWarps][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int N = A.n_samples;
    const int sx = 1, sy = A.grid.R[0], sz = A.grid.R[0] * A.grid.R[1];
    const int off[8] = {0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sy + sx};
    const int64_t stride = int64_t(gridDim.x) * kRenderWarps;
    for (int64_t ray = int64_t(blockIdx.x) * kRenderWarps + warp; ray < A.n_rays; ray += stride) {
        const RayIn R = load_ray(A, ray);
        const RaySpan sp = ray_span(A, R, ray, tab[warp]);
        if (!sp.hit) {
            if (lane == 0) {
                A.rgb[3 * ray + 0] = A.bg[0];
                A.rgb[3 * ray + 1] = A.bg[1];
                A.rgb[3 * ray + 2] = A.bg[2];
                A.depth[ray] = 0.0f;
                A.wsum[ray] = 0.0f;
            }
            continue;
        }
        float acc_r = 0.f, acc_g = 0.f, acc_b = 0.f, acc_d = 0.f, acc_w = 0.f;
        float carry = 0.f, comp = 0.f;  // Kahan sum of log T over chunks
        for (int base = 0; base < N; base += 32) {
            const int k = base + lane;
            const bool active = k < N;
            const float t = span_t(sp, active ? k : N - 1);
            float xw[3];
            point_at(R.o, R.d, t, xw);
            const Cell cell = locate(xw, A.grid.bmin, A.grid.sc, A.grid.R);
            const float s = sdf_value(A.grid, cell);
            float s_next = __shfl_down_sync(FULL, s, 1);
            if (active && (lane == 31 || k + 1 >= N)) {
                float xn[3];
                point_at(R.o, R.d, span_t(sp, k + 1), xn);
                s_next = sdf_value(A.grid, locate(xn, A.grid.bmin, A.grid.sc, A.grid.R));
            }
            float lam = 0.0f;
            if (active) {
                const float diff = log_transmittance(A.tau, s, s_next);
                lam = diff < 0.0f ? diff : 0.0f;
            }
            float cr = 0.f, cg = 0.f, cb = 0.f;
            if (lam < 0.0f) {  // alpha > 0: the colour reaches the outputs
                float w[8];
                corner_weights(cell.f, w);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint2 u = __ldg(colours + cell.base + off[q]);
                    const float2 rg = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
                    const float2 b0 = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
                    cr = fmaf(w[q], rg.x, cr);
                    cg = fmaf(w[q], rg.y, cg);
                    cb = fmaf(w[q], b0.x, cb);
                }
            }
            // transmittance of the chunk (Eq. 8): exclusive warp scan of lam
            float incl = lam;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
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
            acc_r = fmaf(wgt, cr, acc_r);
            acc_g = fmaf(wgt, cg, acc_g);
            acc_b = fmaf(wgt, cb, acc_b);
            acc_d = fmaf(wgt, t, acc_d);
            acc_w += wgt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc_r += __shfl_xor_sync(FULL, acc_r, o);
            acc_g += __shfl_xor_sync(FULL, acc_g, o);
            acc_b += __shfl_xor_sync(FULL, acc_b, o);
            acc_d += __shfl_xor_sync(FULL, acc_d, o);
            acc_w += __shfl_xor_sync(FULL, acc_w, o);
        }
        if (lane == 0) {
            const float TN = expf(carry - comp);
            A.rgb[3 * ray + 0] = fmaf(TN, A.bg[0], acc_r);
            A.rgb[3 * ray + 1] = fmaf(TN, A.bg[1], acc_g);
            A.rgb[3 * ray + 2] = fmaf(TN, A.bg[2], acc_b);
            A.depth[ray] = acc_d;
            A.wsum[ray] = acc_w;
        }
    }
}

template <class C>
cudaError_t launch_shade_t(const RenderArgs& A, const ShadeArgs& S, int ctas_per_sm,
                           cudaStream_t stream)
{
    using L = ShadeLayout<C>;
    cudaError_t e = cudaFuncSetAttribute(shade_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, shade_kernel<C>);
    if (e != cudaSuccess) return e;
    const int per_sm = resident_ctas(fa, kFwdThreads, L::kBytes, L::kTmemCols);
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n_nodes = int64_t(A.grid.R[0]) * A.grid.R[1] * A.grid.R[2];
    const int64_t rounds = (n_nodes + 127) / 128;
    const int64_t full = int64_t(sms > 0 ? sms : 1) * (ctas_per_sm > 0 && ctas_per_sm < per_sm
                                                           ? ctas_per_sm
                                                           : per_sm);
    const int ctas = static_cast<int>(rounds < full ? rounds : full);
    shade_kernel<C><<<ctas, kFwdThreads, L::kBytes, stream>>>(A, S);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_shade(const RenderArgs& A, const KernelShape& ks, const ShadeArgs& S,
                         cudaStream_t stream)
{
#define PSDF_SHADE_CASE(NA, L2, W, K, FB, PH, MH)                                            \
    if (ks.match(NA, L2, W, K, FB, PH, MH))                                                  \
        return launch_shade_t<Cfg<NA, L2, W, K, FB, PH, MH>>(A, S, 0, stream);
    PSDF_FOR_EACH_SHAPE(PSDF_SHADE_CASE)
#undef PSDF_SHADE_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_colour_render(const RenderArgs& A, const void* colours, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, colour_render_kernel,
                                                                  kRenderWarps * 32, 0);
    if (e != cudaSuccess) return e;
    const int64_t need = (A.n_rays + kRenderWarps - 1) / kRenderWarps;
    const int64_t full = int64_t(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    const int ctas = static_cast<int>(need < full ? need : full);
    colour_render_kernel<<<ctas, kRenderWarps * 32, 0, stream>>>(
        A, static_cast<const uint2*>(colours));
    return cudaGetLastError();
}

}  // namespace psdf
