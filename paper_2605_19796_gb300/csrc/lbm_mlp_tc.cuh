// The learned closure's network on the 5th-generation tensor cores (tcgen05)
// for a CTA of 128 cells, one per thread: the network runs as one 128-row
// GEMM per layer instead of per-warp fragment chains.
//
//  * Row i of every layer's A operand and accumulator is TMEM lane i, the cell
//    of thread i (warp w, lane t: i = 32 w + t; four warps, one per TMEM lane
//    quarter).  Each thread writes its own row: the 16 standardised inputs (10
//    used) as 8 BF16-pair columns, later the 64 hidden activations as 32.
//  * One thread issues the layer's MMAs (tcgen05.mma kind::f16, A from TMEM,
//    B = the layer's weights from shared memory, M = 128, N = 64, one
//    instruction per 16 inputs) and commits them to an mbarrier; every thread
//    waits for it and reads its row of the FP32 accumulator back
//    (tcgen05.ld), adds the bias, applies SiLU and packs BF16 pairs into the
//    next layer's A columns (the accumulator and the A columns are disjoint).
//  * The output layer (N = 16, outputs 6..15 zero-weighted) lands in its own
//    16 columns; thread i reads its cell's 6 outputs.
// Weights and biases are the fused inference's (MlpLayout: BF16 weights, the
// hidden layers' weights and biases times 1/2, so that the accumulator plus
// bias is the SiLU's half argument), re-laid out per CTA into the core-matrix
// order the MMA descriptors address.  The arithmetic is that of
// mlp_warp_forward up to the FP32 summation order (the bias is added after the
// products rather than before).
#pragma once

#include <stdint.h>

#include "lbm_mbarrier.cuh"
#include "lbm_mlp_infer.cuh"
#include "lbm_tmem.cuh"

namespace lbmk {

struct MlpTcLayout {
    // B operands, BF16, K-major, core matrices of 8 rows x 16 bytes, no
    // swizzle: element (n, k) at (n / 8) SBO + (k / 8) 128 + (n % 8) 16 + (k % 8) 2
    static constexpr int LBO = 128;
    static constexpr int W1 = 0, SBO1 = 256;            // N 64 x K 16, 2 KB
    static constexpr int W2 = 2048, SBO = 1024;         // N 64 x K 64, 8 KB
    static constexpr int W3 = W2 + 8192;                // N 64 x K 64
    static constexpr int W4 = W3 + 8192;                // N 16 x K 64 (rows 6..15 zero), 2 KB
    static constexpr int B1 = W4 + 2048;                // f32 [64], times 1/2; B2, B3 likewise
    static constexpr int B2 = B1 + 256;
    static constexpr int B3 = B2 + 256;
    static constexpr int B4 = B3 + 256;                 // f32 [16] (6 used)
    static constexpr int XMU = B4 + 64;                 // f32: input mean [10], 1/std [10], output mean [6], std [6]
    static constexpr int XIS = XMU + 40;
    static constexpr int YMU = XIS + 40;
    static constexpr int YSD = YMU + 24;
    static constexpr int MBAR = (YSD + 24 + 7) / 8 * 8;  // MMA-completion mbarrier
    static constexpr int TMEM_SLOT = MBAR + 8;           // base address written by tcgen05.alloc
    static constexpr int BYTES = (TMEM_SLOT + 4 + 127) / 128 * 128;
    // TMEM columns of the CTA (128): hidden accumulator [0, 64), A operand
    // [64, 96) (the inputs use [64, 72)), output accumulator [96, 112)
    static constexpr uint32_t TM_COLS = 128, D_COL = 0, A_COL = 64, D4_COL = 96;
    static_assert(MlpLayout::XIS == MlpLayout::XMU + 40 && MlpLayout::YMU == MlpLayout::XIS + 40 &&
                      MlpLayout::YSD == MlpLayout::YMU + 24,
                  "standardisation values contiguous in both layouts");
    static_assert(MlpLayout::XMU % 16 == 0 && XMU % 16 == 0, "16-byte copies");
};

// Re-lays the packed network block (global memory, MlpLayout) out into `dst`
// (shared memory, MlpTcLayout) with 16-byte copies by threads tid of nt; the
// caller fences the async proxy and synchronises before the first MMA.
__device__ __forceinline__ void mlp_tc_repack(const unsigned char* src, unsigned char* dst, int tid, int nt)
{
    using L = MlpLayout;
    using T = MlpTcLayout;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    auto put = [&](int off, const uint4& v) { *reinterpret_cast<uint4*>(dst + off) = v; };
    auto get = [&](int off) { return __ldg(reinterpret_cast<const uint4*>(src + off)); };
    // W1: 64 rows (pitch 48 bytes) x 2 chunks of 8 inputs
    for (int c = tid; c < 64 * 2; c += nt) {
        const int n = c >> 1, j = c & 1;
        put(T::W1 + (n >> 3) * T::SBO1 + j * T::LBO + (n & 7) * 16, get(L::W1 + n * L::LD1 * 2 + j * 16));
    }
    // W2, W3: 64 rows (pitch 144 bytes) x 8 chunks
    for (int c = tid; c < 2 * 64 * 8; c += nt) {
        const int l = c >> 9, n = (c >> 3) & 63, j = c & 7;
        put((l ? T::W3 : T::W2) + (n >> 3) * T::SBO + j * T::LBO + (n & 7) * 16,
            get((l ? L::W3 : L::W2) + n * L::LD * 2 + j * 16));
    }
    // W4: 16 rows, of which the first 8 are MlpLayout's (6 used, 2 zero)
    for (int c = tid; c < 16 * 8; c += nt) {
        const int n = c >> 3, j = c & 7;
        put(T::W4 + (n >> 3) * T::SBO + j * T::LBO + (n & 7) * 16, n < 8 ? get(L::W4 + n * L::LD * 2 + j * 16) : zero);
    }
    // biases (3 x 64 + 8 floats, the last 8 of B4 zero) and the 32 standardisation values
    for (int c = tid; c < 48 + 4 + 8; c += nt) {
        if (c < 48)
            put(T::B1 + c * 16, get(L::B1 + c * 16));
        else if (c < 52)
            put(T::B4 + (c - 48) * 16, c < 50 ? get(L::B4 + (c - 48) * 16) : zero);
        else
            put(T::XMU + (c - 52) * 16, get(L::XMU + (c - 52) * 16));
    }
}

// Publishes the A columns every thread has written, then one thread issues
// KS MMAs (16 inputs each) of N outputs into column dcol and commits them;
// every thread waits for the commit.  ok_in false on any thread, or a wait
// that gives up, returns false on every thread of the CTA (the first through
// the barrier, the second through the caller's next barrier).
template <int KS, int N>
__device__ __forceinline__ bool mlp_tc_issue(const unsigned char* sm, uint32_t tm_base, int woff, int sbo,
                                             uint32_t dcol, unsigned& phase, int tid, bool ok_in)
{
    using T = MlpTcLayout;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(const_cast<unsigned char*>(sm) + T::MBAR);
    tm_wait_st();
    tm_fence_before();
    if (!__syncthreads_and(ok_in)) return false;
    if (tid == 0) {
        tm_fence_after();
        constexpr uint32_t idesc = tc_idesc_bf16<128, N>();
#pragma unroll
        for (int s = 0; s < KS; ++s)
            tc_mma_ts(tm_base + dcol, tm_base + T::A_COL + 8u * s, tc_smem_desc(sm + woff + s * 2 * T::LBO, T::LBO, sbo),
                      idesc, s > 0 ? 1u : 0u);
        tc_commit(mbar);
    }
    const bool done = __all_sync(0xffffffffu, mbar_wait_bounded(mbar, phase));
    phase ^= 1u;
    tm_fence_after();
    return done;
}

// hidden-layer epilogue of the thread's row: accumulator + bias (both halved)
// -> SiLU -> BF16 pairs into the A columns
__device__ __forceinline__ void mlp_tc_hidden_epilogue(const unsigned char* sm, int boff, uint32_t tm_row)
{
    using T = MlpTcLayout;
    const float2* bias = reinterpret_cast<const float2*>(sm + boff);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        float acc[32];
        tm_ld32(tm_row + T::D_COL + 32u * j, acc);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t out[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 v = __fadd2_rn(make_float2(acc[16 * h + 2 * q], acc[16 * h + 2 * q + 1]),
                                            bias[16 * j + 8 * h + q]);
                out[q] = mlp_silu_pack(v.x, v.y);
            }
            tm_st8(tm_row + T::A_COL + 16u * j + 8u * h, out);
        }
    }
}

// The network for the CTA's 128 rows.  xin: the thread's 16 standardised BF16
// inputs as 8 pairs (pairs 5..7 zero); y: its 6 standardised outputs.  All 128
// threads call it together; returns false (on every thread) when an MMA wait
// gave up, y then undefined.
__device__ __forceinline__ bool mlp_cta_forward_tc(const unsigned char* sm, uint32_t tm_base, uint32_t tm_row,
                                                   const uint32_t (&xin)[8], float (&y)[6], unsigned& phase, int tid,
                                                   bool ok)
{
    using T = MlpTcLayout;
    tm_st8(tm_row + T::A_COL, xin);
    ok = mlp_tc_issue<1, 64>(sm, tm_base, T::W1, T::SBO1, T::D_COL, phase, tid, ok);
    if (ok) mlp_tc_hidden_epilogue(sm, T::B1, tm_row);
    ok = mlp_tc_issue<4, 64>(sm, tm_base, T::W2, T::SBO, T::D_COL, phase, tid, ok);
    if (ok) mlp_tc_hidden_epilogue(sm, T::B2, tm_row);
    ok = mlp_tc_issue<4, 64>(sm, tm_base, T::W3, T::SBO, T::D_COL, phase, tid, ok);
    if (ok) mlp_tc_hidden_epilogue(sm, T::B3, tm_row);
    ok = mlp_tc_issue<4, 16>(sm, tm_base, T::W4, T::SBO, T::D4_COL, phase, tid, ok);
    if (ok) {
        float acc[8];
        tm_ld8(tm_row + T::D4_COL, acc);
        const float* b4 = reinterpret_cast<const float*>(sm + T::B4);
#pragma unroll
        for (int q = 0; q < 6; ++q) y[q] = acc[q] + b4[q];
    }
    return ok;
}

}  // namespace lbmk
