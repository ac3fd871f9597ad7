// Colour MLP (Sec. 4) on the tcgen05 tensor cores.
//
// A CTA of 4 warps batches its 128 samples (4 rays x 32 samples) into M = 128
// tiles.  FP32-equivalent mode: every FP32 operand x is split into
// hi = fp16(x) and lo = fp16(x - hi) (about 22 significant bits) and each layer
// is A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 in tensor memory.
// Reduced-precision mode (MH): plain FP16 operands, one product, FP32
// accumulation.  Layer 3 (width -> 3) stays on the CUDA cores.  The adjoint
// reads the same tiles transposed (MN-major).
#pragma once

#include "sample_eval.cuh"
#include "tc_sm100.cuh"

namespace psdf {

template <class C>
struct MlpTC {
    static constexpr int W = C::W;
    static constexpr int K1 = 16;           // layer-1 K: n_in padded to 16
    static_assert(C::NIN < K1, "n_in + a bias column must fit in 16");
    static_assert(W == 16 || W == 32, "hidden width 16 or 32");
    static constexpr int kSplit = C::MH ? 1 : 2;  // FP16 tiles per operand: hi (+ lo)
    static constexpr int kW1 = W * K1 * 2;  // bytes of one split of W1 [W][16]
    static constexpr int kW2 = W * W * 2;   // bytes of one split of W2 [W][W]
    static constexpr int kWeightBytes = kSplit * (kW1 + kW2);
    static __device__ __forceinline__ uint8_t* w1h(uint8_t* wt) { return wt; }
    static __device__ __forceinline__ uint8_t* w1l(uint8_t* wt) { return wt + kW1; }
    static __device__ __forceinline__ uint8_t* w2h(uint8_t* wt) { return wt + kSplit * kW1; }
    static __device__ __forceinline__ uint8_t* w2l(uint8_t* wt) { return wt + kSplit * kW1 + kW2; }
    // FP32 parameters kept for the CUDA-core parts: b1[W] b2[W] W3[3][W] b3[4]
    // (W3 row-major, so that neighbouring hidden units form pairs)
    static constexpr int kB1 = 0, kB2 = W, kW3 = 2 * W, kB3 = 5 * W, kF32 = 5 * W + 4;
    static constexpr uint32_t kIdescL = tc::idesc_f16(128, W, 0, 0);
};

// Cooperative load of the packed FP32 parameters into the split weight tiles
// (hi at w, lo at w + kW1 / + kW2) and the FP32 block.
template <class C>
__device__ __forceinline__ void load_mlp_tc(const float* __restrict__ g, uint8_t* wt, float* f32)
{
    using M = MlpTC<C>;
    constexpr int W = C::W;
    uint8_t* w1h = M::w1h(wt);
    uint8_t* w1l = M::w1l(wt);
    uint8_t* w2h = M::w2h(wt);
    uint8_t* w2l = M::w2l(wt);
    for (int i = threadIdx.x; i < W * M::K1; i += blockDim.x) {
        const int o = i / M::K1, j = i % M::K1;
        const float v = j < C::NIN ? g[C::gW1 + o * C::NIN + j] : 0.0f;
        __half h, l;
        tc::split2(v, h, l);
        const uint32_t off = tc::tile_off(o, j, M::K1);
        *reinterpret_cast<__half*>(w1h + off) = h;
        if constexpr (M::kSplit == 2) *reinterpret_cast<__half*>(w1l + off) = l;
    }
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) {
        const int o = i / W, j = i % W;
        __half h, l;
        tc::split2(g[C::gW2 + i], h, l);
        const uint32_t off = tc::tile_off(o, j, W);
        *reinterpret_cast<__half*>(w2h + off) = h;
        if constexpr (M::kSplit == 2) *reinterpret_cast<__half*>(w2l + off) = l;
    }
    for (int i = threadIdx.x; i < M::kF32; i += blockDim.x) {
        float v;
        if (i < M::kB2) {
            v = g[C::gB1 + i];
        } else if (i < M::kW3) {
            v = g[C::gB2 + (i - M::kB2)];
        } else if (i < M::kB3) {
            v = g[C::gW3 + (i - M::kW3)];
        } else {
            const int c = i - M::kB3;
            v = c < 3 ? g[C::gB3 + c] : 0.0f;
        }
        f32[i] = v;
    }
}

// The three split products of one K-major x K-major k-step.
__device__ __forceinline__ void mma3(uint32_t d, const uint8_t* a_hi, const uint8_t* a_lo,
                                     const uint8_t* b_hi, const uint8_t* b_lo, uint32_t a_lbo,
                                     uint32_t a_sbo, uint32_t b_lbo, uint32_t b_sbo,
                                     uint32_t idesc, bool accumulate)
{
    const uint64_t ah = tc::desc(a_hi, a_lbo, a_sbo), al = tc::desc(a_lo, a_lbo, a_sbo);
    const uint64_t bh = tc::desc(b_hi, b_lbo, b_sbo), bl = tc::desc(b_lo, b_lbo, b_sbo);
    tc::mma_f16(d, ah, bh, idesc, accumulate);
    tc::mma_f16(d, ah, bl, idesc, true);
    tc::mma_f16(d, al, bh, idesc, true);
}

// One k-step: the three split products, or the single FP16 product.
template <int SPLIT>
__device__ __forceinline__ void mma_k(uint32_t d, const uint8_t* a_hi, const uint8_t* a_lo,
                                      const uint8_t* b_hi, const uint8_t* b_lo, uint32_t a_lbo,
                                      uint32_t a_sbo, uint32_t b_lbo, uint32_t b_sbo,
                                      uint32_t idesc, bool accumulate)
{
    if constexpr (SPLIT == 2) {
        mma3(d, a_hi, a_lo, b_hi, b_lo, a_lbo, a_sbo, b_lbo, b_sbo, idesc, accumulate);
    } else {
        tc::mma_f16(d, tc::desc(a_hi, a_lbo, a_sbo), tc::desc(b_hi, b_lbo, b_sbo), idesc,
                    accumulate);
    }
}

// Layer 3 (W -> 3) and the sigmoid on the CUDA cores: h2 already ReLU'd.
template <class C>
__device__ __forceinline__ void mlp_layer3(const float* f32, const float* h2, float col[3])
{
    using M = MlpTC<C>;
    constexpr int W = C::W;
    const float4 b3 = *reinterpret_cast<const float4*>(f32 + M::kB3);
    // even and odd hidden units summed apart, one paired FMA per output and pair
    float2 z0 = make_float2(0.0f, 0.0f), z1 = z0, z2 = z0;
#pragma unroll
    for (int o = 0; o < W; o += 2) {
        const float2 h = make_float2(h2[o], h2[o + 1]);
        z0 = fma2(*reinterpret_cast<const float2*>(f32 + M::kW3 + o), h, z0);
        z1 = fma2(*reinterpret_cast<const float2*>(f32 + M::kW3 + W + o), h, z1);
        z2 = fma2(*reinterpret_cast<const float2*>(f32 + M::kW3 + 2 * W + o), h, z2);
    }
    col[0] = sigmoidf(b3.x + (z0.x + z0.y));
    col[1] = sigmoidf(b3.y + (z1.x + z1.y));
    col[2] = sigmoidf(b3.z + (z2.x + z2.y));
}

// z = max(z + b, 0) over a row of NV hidden units (bias added in pairs).
template <int NV>
__device__ __forceinline__ void bias_relu(float* z, const float* b)
{
#pragma unroll
    for (int o = 0; o < NV; o += 2) {
        const float2 h = add2(make_float2(z[o], z[o + 1]), *reinterpret_cast<const float2*>(b + o));
        z[o] = fmaxf(h.x, 0.0f);
        z[o + 1] = fmaxf(h.y, 0.0f);
    }
}

// bias_relu that also returns the mask of the units with z + b > 0.
template <int NV>
__device__ __forceinline__ uint32_t bias_relu_mask(float* z, const float* b)
{
    uint32_t mask = 0;
#pragma unroll
    for (int o = 0; o < NV; o += 2) {
        const float2 h = add2(make_float2(z[o], z[o + 1]), *reinterpret_cast<const float2*>(b + o));
        mask |= (h.x > 0.0f ? 1u : 0u) << o;
        mask |= (h.y > 0.0f ? 1u : 0u) << (o + 1);
        z[o] = fmaxf(h.x, 0.0f);
        z[o + 1] = fmaxf(h.y, 0.0f);
    }
    return mask;
}

// Writes a row of NV FP32 values (NV a multiple of 8) into columns
// [c0, c0 + NV) of a tile with C columns: split hi/lo FP16, or plain FP16.
template <int NV, int SPLIT>
__device__ __forceinline__ void store_row(uint8_t* hi, uint8_t* lo, int row, int c0, int C,
                                          const float* v)
{
#pragma unroll
    for (int g = 0; g < NV; g += 8) {
        if constexpr (SPLIT == 2)
            tc::store8(hi, lo, row, c0 + g, C, v + g);
        else
            tc::store8_hi(hi, row, c0 + g, C, v + g);
    }
}

template <int NV, int SPLIT>
__device__ __forceinline__ void zero_row(uint8_t* hi, uint8_t* lo, int row, int c0, int C)
{
#pragma unroll
    for (int g = 0; g < NV; g += 8) {
        if constexpr (SPLIT == 2)
            tc::zero8(hi, lo, row, c0 + g, C);
        else
            tc::zero8_hi(hi, row, c0 + g, C);
    }
}

}  // namespace psdf
