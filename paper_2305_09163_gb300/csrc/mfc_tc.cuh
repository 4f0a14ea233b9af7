// Fifth-generation tensor cores (tcgen05, sm_100 family: sm_103a here) as
// inline PTX: tensor-memory (TMEM) allocation, shared-memory matrix
// descriptors, the kind::f16 instruction descriptor, MMA issue by one thread
// with completion through an mbarrier, and TMEM loads.
//
// Operand layout used throughout: K-major without swizzling.  A tile of R rows
// and K (bf16) columns is stored as core matrices of 8 rows x 16 bytes (8
// elements), each 128 contiguous bytes; core matrices adjacent along K are 128
// bytes apart (the descriptor's leading-dimension byte offset) and groups of 8
// rows are 16 K bytes apart (the stride-dimension byte offset).  An MMA with
// K = 16 reads two core matrices per row group; the next K step starts 256
// bytes further.  The accumulator D (M = 128 rows) lives in TMEM with row m in
// lane m; the four warps of a warpgroup each access their 32 lanes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mfc {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in a K-major tile of K columns (see above).
__host__ __device__ constexpr int kmajor_offset(int row, int k, int K) {
    return (row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor of a K-major, unswizzled tile of K columns
// starting at `tile` (16-byte aligned), advanced by `kstep` K steps of 16.
// Fields: start address >> 4 (bits 0-13), leading-dimension byte offset >> 4
// (16-29), stride-dimension byte offset >> 4 (32-45), descriptor version 1
// (46-47), base offset 0, relative leading offsets, no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t desc_kmajor(const void* tile, int K, int kstep) {
    const uint32_t a = smem_u32(tile) + (uint32_t)kstep * 256u;
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)((uint32_t)(16 * K) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both K-major,
// dense: D format (bits 4-5) = 1, A format (7-9) = 1, B format (10-12) = 1,
// N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp;
// the base address is written to *slot in shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Thread-synchronisation fences around tcgen05 operations, and the fence that
// makes generic-proxy shared-memory writes visible to the tensor core.
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (TMEM) = A * B^T (+ D if accumulate), issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier arrives once when every tcgen05 operation this thread issued
// before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits until the phase of the given parity has completed, polling without
// blocking at most max_polls times with a short sleep between polls; returns
// false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_polls) {
    const uint32_t a = smem_u32(mbar);
    for (uint32_t i = 0; i < max_polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(32);
    }
    return false;
}

// Eight consecutive FP32 columns of this thread's TMEM lane; the values are
// valid after tmem_wait (which takes them as operands so that no use moves
// above it).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait(uint32_t (&r)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}

// n (a multiple of 8) FP32 columns starting at column col of this thread's lane
// (warp w of the warpgroup reads lanes 32 w .. 32 w + 31).
template <int N>
__device__ __forceinline__ void tmem_load_row(uint32_t tmem_base, int warp, int col, float (&out)[N]) {
    static_assert(N % 8 == 0, "columns in groups of eight");
    const uint32_t t = tmem_base + ((uint32_t)(32 * warp) << 16) + (uint32_t)col;
#pragma unroll
    for (int j = 0; j < N / 8; ++j) {
        uint32_t r[8];
        tmem_ld8(t + 8 * j, r);
        tmem_wait(r);
#pragma unroll
        for (int e = 0; e < 8; ++e) out[8 * j + e] = __uint_as_float(r[e]);
    }
}

}  // namespace tc
}  // namespace mfc
