// Tensor memory (TMEM) and tcgen05 helpers (sm_103a inline PTX).
//
// A CTA allocates a power-of-two number of TMEM columns (>= 32) with
// tcgen05.alloc; every one of the 128 lanes has those columns, 32 bits each.
// A warp reaches only the lanes of its quarter (warp w: lanes 32 (w % 4) ..
// 32 (w % 4) + 31), thread t of the warp lane 32 (w % 4) + t.  An address is
// (lane << 16) | column.
#pragma once

#include <stdint.h>

namespace lbmk {

__device__ __forceinline__ void tm_alloc(uint32_t* dst, uint32_t ncols)  // whole warp
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(a), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols)  // whole warp
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// 12 consecutive columns of the thread's lane (one population triple of four cells)
__device__ __forceinline__ void tm_st12(uint32_t ta, const float (&v)[3][4])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%9], {%10, %11, %12, %13};\n" ::"r"(ta),
        "r"(__float_as_uint(v[0][0])), "r"(__float_as_uint(v[0][1])), "r"(__float_as_uint(v[0][2])),
        "r"(__float_as_uint(v[0][3])), "r"(__float_as_uint(v[1][0])), "r"(__float_as_uint(v[1][1])),
        "r"(__float_as_uint(v[1][2])), "r"(__float_as_uint(v[1][3])), "r"(ta + 8u), "r"(__float_as_uint(v[2][0])),
        "r"(__float_as_uint(v[2][1])), "r"(__float_as_uint(v[2][2])), "r"(__float_as_uint(v[2][3]))
        : "memory");
}

// 12 consecutive columns back, waited for inside the same statement so that
// no use of the values can be scheduled before they have arrived
__device__ __forceinline__ void tm_ld12(uint32_t ta, float (&v)[3][4])
{
    uint32_t r[12];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%13];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
        : "r"(ta), "r"(ta + 8u)
        : "memory");
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k / 4][k % 4] = __uint_as_float(r[k]);
}

// The same 12 columns in two statements: the load, then (after independent
// work) the wait, which takes the destination registers as operands so that no
// use of them can be placed between the two.
__device__ __forceinline__ void tm_ld12_issue(uint32_t ta, uint32_t (&r)[12])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%13];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
        : "r"(ta), "r"(ta + 8u)
        : "memory");
}
__device__ __forceinline__ void tm_ld12_wait(uint32_t (&r)[12])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11])
                 :
                 : "memory");
}

// one column of the thread's lane: load issued (wait with tm_ld_wait9 before
// use) / store
__device__ __forceinline__ void tm_ld1_issue(uint32_t ta, uint32_t& r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n" : "=r"(r) : "r"(ta) : "memory");
}
__device__ __forceinline__ void tm_st1(uint32_t ta, uint32_t v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};\n" ::"r"(ta), "r"(v) : "memory");
}
// waits for all of the thread's loads issued so far; r: nine of their
// destination registers, which are not read before this
__device__ __forceinline__ void tm_ld_wait9(uint32_t* r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8])
                 :
                 : "memory");
}

// 8 consecutive columns of the thread's lane, 32-bit values
__device__ __forceinline__ void tm_st8(uint32_t ta, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(ta),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// 8 / 16 consecutive FP32 columns of the thread's lane, waited for in the statement
__device__ __forceinline__ void tm_ld8(uint32_t ta, float (&v)[8])
{
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(ta)
        : "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tm_ld16(uint32_t ta, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta)
        : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// 32 consecutive FP32 columns of the thread's lane (two x16 loads, one wait)
__device__ __forceinline__ void tm_ld32(uint32_t ta, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31}, [%33];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta), "r"(ta + 16u)
        : "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Generic-proxy writes to shared memory made visible to the tensor cores
// (the async proxy), before the barrier that precedes their MMA.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a tcgen05 operand, no swizzle: the matrix
// is tiled into core matrices of 8 rows x 16 bytes (128 contiguous bytes);
// lbo = byte distance between core matrices adjacent along K (the leading
// dimension of a K-major operand), sbo = between core matrices adjacent along
// M or N.  Fields: start address >> 4 (bits 0-13), lbo >> 4 (16-29), sbo >> 4
// (32-45), descriptor version 1 (bits 46-47), base offset 0, layout 0 (no
// swizzle, bits 61-63).
__device__ __forceinline__ uint64_t tc_smem_desc(const void* smem_ptr, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem_ptr);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of a dense kind::f16 MMA with BF16 A and B (both
// K-major), FP32 accumulation: D format F32 (bits 4-5 = 1), A and B format BF16
// (bits 7-9 and 10-12 = 1), no negation or transposition, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
template <int M, int N>
__host__ __device__ constexpr uint32_t tc_idesc_bf16()
{
    static_assert(M == 128, "one CTA, 128 lanes");
    static_assert(N % 16 == 0 && N >= 16 && N <= 256, "N for M = 128");
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[tmem] x B[smem]: A (M x 16, BF16, row i in lane i, pairs of
// K packed in 32-bit columns), B (N x 16 K-major) by descriptor; issued by one
// thread.  accumulate = 0 overwrites D.
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// one arrival on the mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(a) : "memory");
}

}  // namespace lbmk
