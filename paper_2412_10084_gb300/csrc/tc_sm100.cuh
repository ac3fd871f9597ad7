// sm_100-family (sm_103a) tensor-core primitives as inline PTX: tcgen05.mma
// (kind::f16, FP32 accumulation in tensor memory), tcgen05.ld, TMEM
// allocation, shared-memory matrix descriptors, mbarriers.
//
// Operand tiles are "no swizzle" canonical layouts built from core matrices
// of 8 rows x 16 bytes (8 halves).  Descriptor fields: start >> 4 (bits 0-13),
// LBO >> 4 (16-29, stride between core matrices along K), SBO >> 4 (32-45,
// stride between core matrices along M/N), version 1 (46-47), swizzle 0.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace psdf {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t desc(const void* p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = static_cast<uint64_t>((smem_addr(p) & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

// Instruction descriptor, kind::f16 with FP16 A/B and FP32 D.
// a_mn / b_mn select MN-major (transposed) operands.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int a_mn, int b_mn)
{
    return (1u << 4) | (static_cast<uint32_t>(a_mn) << 15) | (static_cast<uint32_t>(b_mn) << 16) |
           (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(static_cast<uint32_t>(accumulate))
        : "memory");
}

__device__ __forceinline__ void commit(uint64_t* mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Default number of polls of a bounded mbarrier wait.
constexpr uint32_t kWaitPolls = 1u << 24;

// Bounded wait for the phase of the given parity to complete.  Returns false
// if the limit ran out (the caller records an error and stops issuing work).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity,
                                          uint32_t limit = kWaitPolls)
{
    const uint32_t a = smem_addr(mbar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Makes this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy).
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp-collective TMEM allocation; the base address is written to *slot.
// `last` gives up the CTA's right to allocate more (set it on the last one).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols, bool last = true)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    if (last)
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// 32 lanes x 16 / 32 consecutive 32-bit columns: lane i of the warp reads
// TMEM lane (taddr.lane + i).  Warp-collective.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v)
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 16 / 4 consecutive 32-bit columns from registers: lane i writes
// TMEM lane (taddr.lane + i).  Warp-collective; tmem_st_wait() before the
// columns are read back.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float* v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                 "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                 : "memory");
}

__device__ __forceinline__ void tmem_st_wait()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v)
{
    static_assert(N % 16 == 0, "16-column granules");
#pragma unroll
    for (int c = 0; c < N; c += 32) {
        if (c + 32 <= N)
            tmem_ld32(taddr + c, v + c);
        else
            tmem_ld16(taddr + c, v + c);
    }
}

// ---------------------------------------------------------------------------
// FP16 operand tiles, "rows x C" halves, K-major along the columns:
// core matrix (row/8, col/8) at (row/8)*(C/8)*128 + (col/8)*128 bytes.
// The same bytes read as an MN-major operand give the transpose (rows become
// K, columns become M or N).
// ---------------------------------------------------------------------------

__host__ __device__ constexpr uint32_t tile_off(int row, int col, int C)
{
    return static_cast<uint32_t>((row >> 3) * (C / 8) * 128 + (col >> 3) * 128 + (row & 7) * 16 +
                                 (col & 7) * 2);
}

// Splits v into hi = fp16(v) and lo = fp16(v - hi): hi + lo carries ~22 bits.
__device__ __forceinline__ void split2(float v, __half& hi, __half& lo)
{
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}

// Splits the pair (a, b) into packed FP16 hi = fp16(a, b) and lo =
// fp16(a - hi.x, b - hi.y), element a in the low half.  The packed
// conversions round exactly as the scalar ones (round to nearest even), so
// the split is the same as split2's, in fewer instructions.
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo)
{
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    float2 r;  // (a - hf.x, b - hf.y), both exact, in one paired subtraction
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a), "f"(b), "f"(hf.x), "f"(hf.y));
    const __half2 l = __floats2half2_rn(r.x, r.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Writes 8 consecutive columns [c0, c0+8) of `row` into the hi and lo tiles.
__device__ __forceinline__ void store8(uint8_t* hi_tile, uint8_t* lo_tile, int row, int c0, int C,
                                       const float* v)
{
    uint4 hv, lv;
    split_pair(v[0], v[1], hv.x, lv.x);
    split_pair(v[2], v[3], hv.y, lv.y);
    split_pair(v[4], v[5], hv.z, lv.z);
    split_pair(v[6], v[7], hv.w, lv.w);
    const uint32_t off = tile_off(row, c0, C);
    *reinterpret_cast<uint4*>(hi_tile + off) = hv;
    *reinterpret_cast<uint4*>(lo_tile + off) = lv;
}

// Writes 8 consecutive columns as plain FP16 (hi tile only).
__device__ __forceinline__ void store8_hi(uint8_t* hi_tile, int row, int c0, int C, const float* v)
{
    uint4 hv;
    const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    const __half2 c = __floats2half2_rn(v[4], v[5]), d = __floats2half2_rn(v[6], v[7]);
    hv.x = *reinterpret_cast<const uint32_t*>(&a);
    hv.y = *reinterpret_cast<const uint32_t*>(&b);
    hv.z = *reinterpret_cast<const uint32_t*>(&c);
    hv.w = *reinterpret_cast<const uint32_t*>(&d);
    *reinterpret_cast<uint4*>(hi_tile + tile_off(row, c0, C)) = hv;
}

__device__ __forceinline__ void zero8_hi(uint8_t* hi_tile, int row, int c0, int C)
{
    *reinterpret_cast<uint4*>(hi_tile + tile_off(row, c0, C)) = make_uint4(0, 0, 0, 0);
}

// Zeroes 8 consecutive columns of a row in both tiles.
__device__ __forceinline__ void zero8(uint8_t* hi_tile, uint8_t* lo_tile, int row, int c0, int C)
{
    const uint32_t off = tile_off(row, c0, C);
    *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(0, 0, 0, 0);
    *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(0, 0, 0, 0);
}

}  // namespace tc
}  // namespace psdf
