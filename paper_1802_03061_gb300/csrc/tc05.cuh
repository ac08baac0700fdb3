// Thin wrappers over the sm_100-family tensor-core instructions used by the
// learned guess's convolutions: TMEM allocation (tcgen05.alloc/dealloc), the
// BF16 MMA with FP32 accumulation in TMEM (tcgen05.mma .kind::f16), its
// completion through an mbarrier (tcgen05.commit), TMEM loads (tcgen05.ld)
// and the descriptors of K-major, non-swizzled shared-memory operands.
//
// Operand layout ("core matrices"): a K-major operand of R rows x K bf16 sits
// in shared memory as 8-row x 16-byte core matrices, each 128 contiguous
// bytes (row r of the core at byte 16 r); the core of row group g and K
// chunk c (8 elements) at byte (g * (K / 8) + c) * 128.  So the K-adjacent
// core stride (the descriptor's leading byte offset) is 128 bytes and the
// row-group stride (stride byte offset) is K / 8 * 128 bytes.
#pragma once
#include <stdint.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), the fixed version field (bit 46) of the tcgen05
// format, no swizzle.  K-major operands: leading = the K-adjacent core
// stride, stride = the row-group (M or N) stride.  M/N-major operands (a
// core matrix is then 8 K-rows of 8 consecutive M or N elements, 16 bytes
// each, still 128 contiguous bytes): leading = the K-adjacent core stride,
// stride = the M/N-adjacent core stride.
__device__ __forceinline__ uint64_t tc_desc_kmajor(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of .kind::f16: BF16 A and B, FP32 accumulator,
// M x N tile; mn_major: both operands M/N-major (the M or N index contiguous
// in a core-matrix row) instead of K-major
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N, bool mn_major = false) {
    return (1u << 4)                       // accumulator format: F32
           | (1u << 7)                     // A format: BF16
           | (1u << 10)                    // B format: BF16
           | (mn_major ? (1u << 15) : 0u)  // A major-ness
           | (mn_major ? (1u << 16) : 0u)  // B major-ness
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void tc_alloc(uint32_t* slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (TMEM) = A B^T (+ D when accumulate): one MMA, issued by one thread
__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier completes one phase once all earlier MMAs of this thread are done
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// waits for the phase of the given parity; gives up after `limit` polls
// (returns false) so that a lost arrival cannot hang the GPU
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long limit) {
    const uint32_t a = smem_u32(mbar);
    for (long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: warp
// w of the CTA reads lanes 32 (w % 4) .. + 31)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills the 16
// bytes with zeros (src must still be a valid address)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
