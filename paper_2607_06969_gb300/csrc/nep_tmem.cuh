// Tensor memory (TMEM) and 5th-generation tensor-core (tcgen05) primitives
// for the sm_100 family, as inline PTX.
//
// TMEM is a 128-lane x 512-column array of 32-bit cells per SM.  A CTA
// allocates a power-of-two number of columns (>= 32) with one warp and frees
// them with the same warp.  In a 128-thread CTA, warp w reaches lanes
// 32w..32w+31 (the 32x32b shapes move one lane per thread), so thread t of
// the CTA owns lane t.  The evaluation kernels use TMEM two ways:
//   * as per-thread scratch: an atom's S_nlm row is parked in its thread's
//     lane while the network runs, instead of in shared memory;
//   * as the FP32 accumulator of tcgen05.mma (kind::f16, M = 128), whose
//     row r lands in lane r.
// Every instruction here with .sync.aligned must be executed by all 32
// threads of the warp together; callers reconverge with __syncwarp() first.
#pragma once
#include <cstdint>

namespace nep {
namespace tc5 {

// The PTX is emitted only in the device compilation pass; the host pass
// sees empty bodies (these functions are never called from host code).
#if defined(__CUDA_ARCH__)
#define NEP_PTX(...) asm volatile(__VA_ARGS__)
#else
#define NEP_PTX(...) ((void)0)
#endif

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
#if defined(__CUDA_ARCH__)
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
#else
    (void)p;
    return 0u;
#endif
}

// --- allocation (one warp) ---------------------------------------------------
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncols) {
    NEP_PTX("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    NEP_PTX("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t base, uint32_t ncols) {
    NEP_PTX("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// --- ordering of tcgen05 operations around thread synchronisation ------------
__device__ __forceinline__ void fence_before() {
    NEP_PTX("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    NEP_PTX("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() {
    NEP_PTX("fence.proxy.async.shared::cta;" ::: "memory");
}

// --- per-thread lane access, 32x32b shape -------------------------------------
// address of column c of the calling warp's lane quarter
__device__ __forceinline__ uint32_t lane_addr(uint32_t base, int warp, int col) {
    return base + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(col);
}
__device__ __forceinline__ void st8(uint32_t ta, const float* v) {
    NEP_PTX(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
        : "memory");
}
__device__ __forceinline__ void ld8(uint32_t ta, float* v) {
    uint32_t r[8] = {};
    NEP_PTX("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(ta)
                 : "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void ld16(uint32_t ta, float* v) {
    uint32_t r[16] = {};
    NEP_PTX(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta)
        : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void wait_st() { NEP_PTX("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { NEP_PTX("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// --- mbarrier -------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    NEP_PTX("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    NEP_PTX("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// wait for the phase with the given parity to complete, at most `limit`
// polls; returns false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < limit; ++it) {
        uint32_t done = 0;
        NEP_PTX(
            "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// --- matrix multiply ------------------------------------------------------------
// Shared-memory operand descriptor, no swizzle, K-major: the operand is a
// grid of 8-row x 16-byte core matrices (128 contiguous bytes each); lbo is
// the byte distance between core matrices adjacent along K, sbo between
// core matrices adjacent along M (or N).  Bits 46-47 carry the descriptor
// version (1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
           (static_cast<uint64_t>(sbo >> 4) << 32) | (static_cast<uint64_t>(1) << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A
// and B both FP16 (0) or both BF16 (1) in bits 7-9 and 10-12, both K-major
// (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}
// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        bool accumulate) {
    NEP_PTX(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}
// the mbarrier completes one arrival once every earlier MMA of this thread is done
__device__ __forceinline__ void commit(uint64_t* bar) {
    NEP_PTX("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// element offset of (row r, column k) in a no-swizzle K-major operand whose
// K extent is Kp (a multiple of 8): core matrices adjacent along K are 128
// bytes apart, 8-row groups Kp * 16 bytes apart
__host__ __device__ constexpr int cm_offset(int r, int k, int Kp) {
    return (r >> 3) * (Kp * 8) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// smallest legal TMEM allocation holding n columns
__host__ __device__ constexpr uint32_t tmem_cols(int n) {
    return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : n <= 256 ? 256u : 512u;
}

}  // namespace tc5
}  // namespace nep
