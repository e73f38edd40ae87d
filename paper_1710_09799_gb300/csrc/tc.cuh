// Fifth-generation tensor core primitives for sm_103a (internal header):
// tensor memory allocation, tcgen05.mma of kind::tf32 (A in tensor or shared
// memory, B in shared memory), completion through an mbarrier, accumulator
// reads and writes, and bulk global-to-shared copies.
//
// Operand layout (both A and B "K-major", no swizzle): a matrix of R rows and
// K columns (K a multiple of 4) is stored as 8-row x 16-byte core matrices;
// element (r, k) of a 4-byte type sits at
//   (r / 8) * (K * 32) + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4
// bytes from the base. Core matrices adjacent along K are 128 bytes apart (the
// descriptor's leading-dimension byte offset) and 8-row groups K * 32 bytes
// apart (its stride-dimension byte offset). One MMA consumes K = 8 (two core
// matrices along K); the k-th block of 8 starts k * 256 bytes after the base.
#pragma once

#include <cstdint>

namespace mln {
namespace tc {

__host__ __device__ constexpr int core_offset(int r, int k, int K) {
    return (r / 8) * (K * 32) + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4;
}

// Round an FP32 value to TF32 (10 explicit mantissa bits), nearest with ties
// away from zero, as a bit pattern with the 13 low bits clear (finite inputs).
__host__ __device__ inline uint32_t tf32_bits(uint32_t b) { return (b + 0x1000u) & 0xFFFFE000u; }

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator, TF32 A
// and B, both K-major, M = 128, N given (multiple of 16, 16 .. 256).
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4)                                  // D format: F32
           | (2u << 7)                                // A format: TF32
           | (2u << 10)                               // B format: TF32
           | (static_cast<uint32_t>(n >> 3) << 17)    // N / 8
           | (static_cast<uint32_t>(128 >> 4) << 24); // M / 16
}

// Byte offset of element (r, k) of a 2-byte K-major operand with K columns (a
// multiple of 8): 8-row x 16-byte core matrices of 8 elements along K, core
// matrices adjacent along K 128 bytes apart, 8-row groups K * 16 bytes apart;
// one kind::f16 MMA consumes K = 16 (two core matrices), the k-th block of 16
// starting k * 256 bytes after the base.
__host__ __device__ constexpr int core_offset16(int r, int k, int K) {
    return (r / 8) * (K * 16) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

// Instruction descriptor of tcgen05.mma kind::f16 with FP16 A and B, FP32
// accumulator, both K-major, M = 128, N given (multiple of 16, 16 .. 256).
__host__ __device__ constexpr uint32_t idesc_f16(int n) {
    return (1u << 4)                                  // D format: F32
           | (0u << 7)                                // A format: F16
           | (0u << 10)                               // B format: F16
           | (static_cast<uint32_t>(n >> 3) << 17)    // N / 8
           | (static_cast<uint32_t>(128 >> 4) << 24); // M / 16
}

// Shared-memory matrix descriptor (no swizzle): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// --- tensor memory -------------------------------------------------------

// One full warp: allocate ncols columns (power of two >= 32); the TMEM address
// is written to shared memory at dst.
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

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Make this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// --- MMA -------------------------------------------------------------------

// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, kind::tf32, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T, M = 128, kind::tf32: row i of A is TMEM
// lane i, its K elements consecutive 32-bit columns from a_tmem.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T, M = 128, kind::f16 (FP16 A and B, FP32
// D): row i of A is TMEM lane i, its K elements packed two per 32-bit column
// (element 2c in the low half of column c, 2c + 1 in the high half).
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One lane of the (converged) warp: true for the elected leader.
__device__ __forceinline__ bool elect_one() {
    uint32_t e;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(e));
    return e != 0;
}

// Two FP32 values to a packed FP16 pair, round to nearest even: lo in the low
// half, hi in the high half.
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Arrive once on the mbarrier when every MMA issued so far by this thread is complete.
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// --- mbarrier --------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Wait for the phase with the given parity to complete; gives up after a
// bounded number of polls (each poll may suspend the thread for a short,
// hardware-chosen time) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int i = 0; i < (1 << 20); ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// As mbar_wait, but each poll suspends the thread until the phase completes
// or `hint_ns` nanoseconds pass, so a waiting warp issues a few polls instead
// of spinning; gives up after `polls` polls (bounded: polls x hint_ns at most).
__device__ __forceinline__ bool mbar_wait_hint(uint32_t mbar, uint32_t parity, uint32_t hint_ns, int polls) {
    for (int i = 0; i < polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(mbar), "r"(parity), "r"(hint_ns)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// --- bulk copies (the asynchronous copy engine) -------------------------------

// Arm the mbarrier for `bytes` of incoming transactions (this thread's arrival).
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to this CTA's shared memory; completion is counted on the mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// --- accumulator reads -------------------------------------------------------

// Warp-collective: lane i of the warp reads 32 (resp. 8, 4) consecutive FP32
// columns of TMEM lane (lane base + i), starting at taddr (lane base in bits
// 31..16, column in bits 15..0). Complete with ld_wait before use.
__device__ __forceinline__ void ld_x32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld_x8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// Warp-collective: lane i writes 8 consecutive 32-bit columns of TMEM lane
// (lane base + i) from v. Complete with st_wait.
__device__ __forceinline__ void st_x8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Named barrier over `count` threads (a multiple of 32).
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

}  // namespace tc
}  // namespace mln
