// Small sm_103a helpers shared by the tensor-core kernels: shared-memory
// addresses, bounded mbarrier waits, tcgen05 fences, shared-memory matrix and
// instruction descriptors for kind::f16 (BF16 in, FP32 accumulate), MMA issue
// and commit, TMEM loads, and the BF16 piece split of FP32 operands; the
// FP16 instruction descriptor for the pruning network's layers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace {

constexpr int TC_KB = 64;                      // K block: 64 BF16 = one 128-byte swizzle row

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `bar` with the given parity; false after ~2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0 && global_ns() - t0 > 2000000000ull) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzle layout: rows of 128 bytes, groups of 8 rows 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t desc = 0;
    desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    desc |= (uint64_t)1 << 16;                     // leading byte offset (unused here)
    desc |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    desc |= (uint64_t)1 << 46;                     // descriptor version
    desc |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return desc;
}

// Shared-memory matrix descriptor of an MN-major operand in the 128-byte
// swizzle layout: atoms of 8 K rows x 64 16-bit MN elements (1 KB, each K row
// 128 bytes), atoms along MN `lbo` bytes apart, groups of 8 K rows `sbo`
// bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t desc = 0;
    desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    desc |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    desc |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    desc |= (uint64_t)1 << 46;
    desc |= (uint64_t)2 << 61;
    return desc;
}

// Byte offset of element (k, mn) of an MN-major swizzled operand with MN
// atoms 1 KB apart and 8-row K groups `sbo` bytes apart (the 16-byte chunks
// of a 128-byte row are exchanged by k mod 8, as in the K-major layout).
__device__ __forceinline__ uint32_t sw128_mn_off(int k, int mn, uint32_t sbo) {
    return (uint32_t)(k >> 3) * sbo + (uint32_t)(mn >> 6) * 1024u + (uint32_t)(k & 7) * 128u +
           ((((uint32_t)(mn & 63) >> 3) ^ (uint32_t)(k & 7)) << 4) + (uint32_t)(mn & 7) * 2u;
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16: BF16 A and B, both MN-major, FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16_f32_mn(int M, int N) {
    return idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);
}

// Instruction descriptor of kind::f16: FP16 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// (kind::f16 covers both 16-bit input types; the instruction descriptor says which)
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per lane).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per lane).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element k (0..63) of row r inside a swizzled K block.
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint2 pack_bf16x4(float a, float b, float c, float d) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b);
    __nv_bfloat162 hi = __floats2bfloat162_rn(c, d);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&lo);
    u.y = *reinterpret_cast<uint32_t*>(&hi);
    return u;
}

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Writes four FP32 values as NS BF16 pieces (hi, then the rounded remainders),
// piece p at dst + p * stride: v = hi + mid + lo exactly for NS = 3.
template <int NS>
__device__ __forceinline__ void store_pieces(uint8_t* dst, size_t stride, float a, float b, float c, float d) {
#pragma unroll
    for (int p = 0; p < NS; ++p) {
        *reinterpret_cast<uint2*>(dst + p * stride) = pack_bf16x4(a, b, c, d);
        if (p + 1 < NS) {
            a -= bf16_round(a);
            b -= bf16_round(b);
            c -= bf16_round(c);
            d -= bf16_round(d);
        }
    }
}


}  // namespace
