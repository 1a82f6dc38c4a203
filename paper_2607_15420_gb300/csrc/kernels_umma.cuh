// kernels_umma.cuh -- the warm-start network's forward products on the fifth-generation
// tensor cores (tcgen05, kind::f16), accumulators in tensor memory.
//
// C[m][n] = sum_k A[m][k] W[n][k] for the layers with K a multiple of 64 (the 256-wide
// ones): A FP32 row-major [M][K] (the previous layer's activations), W bfloat16 row-major
// [N][K] (the layer's rounded weights), FP32 accumulation.  An MMA takes both operands in
// one type, so each FP32 activation enters as the sum of three bfloat16 terms
// a = h + m + l (h the rounding of a, m of a - h, l of a - h - m: 24 significand bits),
// and the three products with the bfloat16 weight are exact in the FP32 accumulator: the
// layer's product at FP32 accuracy from three MMAs per K step.
//
// Block: 256 threads; tile 128 rows x 64 columns; K in chunks of 64 staged in shared
// memory by the threads (FP32 loads, the split, 8-byte stores) in the no-swizzle K-major
// layout of 8-row x 16-byte core matrices, each half-warp filling whole core matrices (no
// bank conflicts).  One thread issues the chunk's 12 MMAs (4 K steps x 3 terms) and
// commits them to an mbarrier; every thread waits on it (bounded) before the chunk's
// shared memory is refilled.  The accumulator (128 lanes x 64 FP32 columns of tensor
// memory) is read back by tcgen05.ld -- warp w its lanes 32 (w % 4) + 0..31 = its rows,
// columns 32 (w / 4) + 0..31 -- for the fused epilogue.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace umma {

constexpr int TM = 128, TN = 64, KC = 64, T = 256;
constexpr int A_PLANE = TM * KC * 2;              // one bfloat16 term of the A chunk: 16 KB
constexpr int B_BYTES = TN * KC * 2;              // the W chunk: 8 KB
// dynamic shared memory: the chunk (56 KB) + 1 KB alignment slack; at most three blocks
// per SM, 192 of the 512 tensor-memory columns
constexpr int SMEM = 3 * A_PLANE + B_BYTES + 1024;
// core-matrix strides (bytes): A [kc][16 row groups], B [kc][8 row groups]; adjacent
// core matrices along K ("leading") and along M / N ("stride")
constexpr uint32_t A_LBO = (TM / 8) * 128, A_SBO = 128, B_LBO = (TN / 8) * 128, B_SBO = 128;
constexpr long long WAIT_LIMIT = 1ll << 22;      // mbarrier polls before a wait gives up
static_assert(TM == 128 && TN % 16 == 0 && TN >= 32 && TN <= 256 && (TN & (TN - 1)) == 0,
              "an M = 128 MMA shape; tensor-memory columns a power of two >= 32");
static_assert((TM * KC / 4) % T == 0 && (TN * KC / 8) % T == 0 && (TN / 2) % 16 == 0, "staging and epilogue split");

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4),
// descriptor version 1 at bits 46-47, base offset 0, no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// the threads' shared-memory stores become visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier completes its phase when every MMA this thread issued so far is done
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of phase `parity` (at most `limit` polls); false when it
// gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

// 16 consecutive accumulator columns of this thread's lane (32x32b shape: lane = row)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (r, k) of a K-major chunk in core-matrix layout with `groups`
// 8-row groups per 8-column K block
__device__ __forceinline__ uint32_t core_off(int r, int k, int groups) {
    return (uint32_t)((((k >> 3) * groups + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

}  // namespace umma
