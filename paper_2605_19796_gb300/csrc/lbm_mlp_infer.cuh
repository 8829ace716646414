// Fused inference of the learned closure's network inside the step kernel.
//
// The 32 cells of a warp (one x-row of the CTA tile) form the M dimension of
// the per-layer GEMMs, run on the tensor cores with mma.sync m16n8k16 (BF16
// inputs, FP32 accumulation): two 16-row tiles per warp, layers 10(->16) x 64,
// 64 x 64, 64 x 64, 64 x 8(6 used).  The FP32 accumulator fragment of one
// layer (rows g, g+8; columns 2t, 2t+1 of an 8-column tile) is, after bias and
// SiLU and packing to BF16 pairs, exactly the A fragment of the next layer
// (k-step s = n-tiles 2s, 2s+1), so activations never leave registers; only the
// 10 inputs and 6 outputs go through a per-warp shared-memory exchange.
//
// Packed parameter block (prepared by the host, copied to shared memory):
//   W1 [64][24] bf16 (inputs 10, zero padded; row pitch 24 keeps the B-fragment
//   loads bank-conflict free), W2, W3 [64][72] bf16, W4 [8][72] bf16 (rows 6, 7
//   zero), biases b1 b2 b3 [64] f32, b4 [8] f32, input mean [10], input 1/std
//   [10], output mean [6], output std [6] (f32, padded to 48).  W1..W3 and
//   b1..b3 are stored times 1/2 (the SiLU's half argument, below).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lbmk {

struct MlpLayout {
    static constexpr int LD1 = 24, LD = 72;
    static constexpr int W1 = 0;                        // byte offsets
    static constexpr int W2 = W1 + 64 * LD1 * 2;
    static constexpr int W3 = W2 + 64 * LD * 2;
    static constexpr int W4 = W3 + 64 * LD * 2;
    static constexpr int B1 = W4 + 8 * LD * 2;
    static constexpr int B2 = B1 + 64 * 4;
    static constexpr int B3 = B2 + 64 * 4;
    static constexpr int B4 = B3 + 64 * 4;
    static constexpr int XMU = B4 + 8 * 4;
    static constexpr int XIS = XMU + 10 * 4;
    static constexpr int YMU = XIS + 10 * 4;
    static constexpr int YSD = YMU + 6 * 4;
    static constexpr int BYTES = (YSD + 6 * 4 + 127) / 128 * 128;
    // per-warp exchange: inputs [32][XLD] bf16 (16 used); the outputs [32][8]
    // f32 overlay its first 1 KB (rows of a 16-row tile are written only after
    // the warp has read that tile's inputs, and the second tile's inputs lie at
    // bytes 768 and up, past the first tile's outputs)
    static constexpr int XLD = 24;
    static constexpr int XCH_BYTES = 32 * XLD * 2;
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// SiLU a * sigmoid(a) = h + h tanh(h), h = a / 2, on the hardware tanh (one
// MUFU operation, relative error about 2^-11, below the BF16 rounding that
// follows).  The hidden layers' weights and biases are packed times 1/2 (exact
// in BF16 and FP32), so the accumulator already holds h; the two columns of a
// fragment row take one packed FP32 FMA.
__device__ __forceinline__ float mlp_tanh(float v)
{
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ uint32_t mlp_silu_pack(float h0, float h1)
{
    const float2 h = make_float2(h0, h1);
    const float2 y = __ffma2_rn(h, make_float2(mlp_tanh(h0), mlp_tanh(h1)), h);
    return pack_bf16(y.x, y.y);
}

// B fragments of the m16n8k16 products from the packed [n][k] weight rows with
// ldmatrix: 8x8 BF16 matrices whose rows are output units n and whose columns
// are 8 consecutive inputs k, so lane l receives W[n0 + l/4][k0 + 2(l%4) ..+1],
// the fragment layout of the "col" B operand.  x2: matrices at k0 = 16 s and
// 16 s + 8 (one k-step, b0 and b1); x4: two k-steps.  Lane l gives the address
// of row l%8 of matrix l/8.  Row pitches of 48 and 144 bytes keep the 16-byte
// rows 16-byte aligned and the eight rows of a matrix on distinct banks.  The
// hidden layers take x2 loads (x4 raises the register peak of the fused step
// kernel past its 128-register budget), the output layer x4.
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

// shared-memory address of this lane's ldmatrix row: output row n0 + lane%8,
// input column k0 + 8 (lane/8) (x4: two k-steps; x2 uses lanes 0-15)
template <int LDW>
__device__ __forceinline__ uint32_t ldsm_row(uint32_t wbase, int n0, int k0, int lane)
{
    return wbase + (uint32_t)(((n0 + (lane & 7)) * LDW + k0 + 8 * (lane >> 3)) * 2);
}

// One hidden layer (64 outputs) for one 16-row tile: A fragments of the input
// (KS k-steps) -> A fragments of the output (4 k-steps of the next layer).
// The accumulators start at the bias.
template <int KS, int LDW>
__device__ __forceinline__ void mlp_hidden(const unsigned char* sm, int woff, int boff, const uint32_t (&ain)[KS][4],
                                           uint32_t (&aout)[4][4], int lane)
{
    const int t = lane & 3;
    const uint32_t wbase = (uint32_t)__cvta_generic_to_shared(sm + woff);
    const float2* B = reinterpret_cast<const float2*>(sm + boff);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 bb = B[4 * nt + t];  // columns 8 nt + 2t, 8 nt + 2t + 1
        float c[4] = {bb.x, bb.y, bb.x, bb.y};
        if constexpr (KS == 1) {
            uint32_t b0, b1;
            ldsm_x2(ldsm_row<LDW>(wbase, 8 * nt, 0, lane & 15), b0, b1);
            mma_bf16_16816(c, ain[0], b0, b1);
        } else {
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                uint32_t b0, b1;
                ldsm_x2(ldsm_row<LDW>(wbase, 8 * nt, 16 * s, lane & 15), b0, b1);
                mma_bf16_16816(c, ain[s], b0, b1);
            }
        }
        const uint32_t lo = mlp_silu_pack(c[0], c[1]);  // row g
        const uint32_t hi = mlp_silu_pack(c[2], c[3]);  // row g + 8
        if (nt & 1) {
            aout[nt >> 1][2] = lo;
            aout[nt >> 1][3] = hi;
        } else {
            aout[nt >> 1][0] = lo;
            aout[nt >> 1][1] = hi;
        }
    }
}

// The same layer for both 16-row tiles of the warp at once: each B fragment
// is loaded once and feeds two independent MMAs, so the layer issues half the
// ldmatrix operations and has two accumulator chains in flight (twice the
// fragment registers: taken where the kernel can afford them).
template <int KS, int LDW>
__device__ __forceinline__ void mlp_hidden2(const unsigned char* sm, int woff, int boff, const uint32_t (&ain0)[KS][4],
                                            const uint32_t (&ain1)[KS][4], uint32_t (&aout0)[4][4],
                                            uint32_t (&aout1)[4][4], int lane)
{
    const int t = lane & 3;
    const uint32_t wbase = (uint32_t)__cvta_generic_to_shared(sm + woff);
    const float2* B = reinterpret_cast<const float2*>(sm + boff);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 bb = B[4 * nt + t];
        float c0[4] = {bb.x, bb.y, bb.x, bb.y};
        float c1[4] = {bb.x, bb.y, bb.x, bb.y};
#pragma unroll
        for (int s = 0; s < KS; ++s) {
            uint32_t b0, b1;
            ldsm_x2(ldsm_row<LDW>(wbase, 8 * nt, 16 * s, lane & 15), b0, b1);
            mma_bf16_16816(c0, ain0[s], b0, b1);
            mma_bf16_16816(c1, ain1[s], b0, b1);
        }
        const int j = nt >> 1, o = (nt & 1) * 2;
        aout0[j][o] = mlp_silu_pack(c0[0], c0[1]);
        aout0[j][o + 1] = mlp_silu_pack(c0[2], c0[3]);
        aout1[j][o] = mlp_silu_pack(c1[0], c1[1]);
        aout1[j][o + 1] = mlp_silu_pack(c1[2], c1[3]);
    }
}

// Network forward for the warp's 32 cells, both 16-row tiles together (see
// mlp_hidden2); all inputs are read before the first output is written.
__device__ __forceinline__ void mlp_warp_forward_dual(const unsigned char* sm, const __nv_bfloat16* X, float* Y,
                                                      int lane)
{
    using L = MlpLayout;
    const int g = lane >> 2, t = lane & 3;
    const uint32_t* Xw = reinterpret_cast<const uint32_t*>(X);
    uint32_t a[2][1][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        a[mt][0][0] = Xw[(r0 * L::XLD + 2 * t) / 2];
        a[mt][0][1] = Xw[(r1 * L::XLD + 2 * t) / 2];
        a[mt][0][2] = Xw[(r0 * L::XLD + 2 * t + 8) / 2];
        a[mt][0][3] = Xw[(r1 * L::XLD + 2 * t + 8) / 2];
    }
    uint32_t p1[4][4], q1[4][4], p2[4][4], q2[4][4];
    mlp_hidden2<1, L::LD1>(sm, L::W1, L::B1, a[0], a[1], p1, q1, lane);
    mlp_hidden2<4, L::LD>(sm, L::W2, L::B2, p1, q1, p2, q2, lane);
    mlp_hidden2<4, L::LD>(sm, L::W3, L::B3, p2, q2, p1, q1, lane);
    const uint32_t w4 = (uint32_t)__cvta_generic_to_shared(sm + L::W4);
    const float2 b4 = reinterpret_cast<const float2*>(sm + L::B4)[t];
    float c0[4] = {b4.x, b4.y, b4.x, b4.y};
    float c1[4] = {b4.x, b4.y, b4.x, b4.y};
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        uint32_t b[4];
        ldsm_x4(ldsm_row<L::LD>(w4, 0, 32 * sp, lane), b);
        mma_bf16_16816(c0, p1[2 * sp], b[0], b[1]);
        mma_bf16_16816(c0, p1[2 * sp + 1], b[2], b[3]);
        mma_bf16_16816(c1, q1[2 * sp], b[0], b[1]);
        mma_bf16_16816(c1, q1[2 * sp + 1], b[2], b[3]);
    }
    __syncwarp();  // every lane has read both tiles' inputs
    *reinterpret_cast<float2*>(Y + g * 8 + 2 * t) = make_float2(c0[0], c0[1]);
    *reinterpret_cast<float2*>(Y + (g + 8) * 8 + 2 * t) = make_float2(c0[2], c0[3]);
    *reinterpret_cast<float2*>(Y + (g + 16) * 8 + 2 * t) = make_float2(c1[0], c1[1]);
    *reinterpret_cast<float2*>(Y + (g + 24) * 8 + 2 * t) = make_float2(c1[2], c1[3]);
}

// Network forward for the warp's 32 cells: X [32][XLD] bf16 (standardised
// inputs, columns 10..15 zero) -> Y [32][8] f32 (standardised outputs 0..5);
// Y may alias X (the exchange layout above).
__device__ __forceinline__ void mlp_warp_forward(const unsigned char* sm, const __nv_bfloat16* X, float* Y, int lane)
{
    using L = MlpLayout;
    const int g = lane >> 2, t = lane & 3;
    const uint32_t* Xw = reinterpret_cast<const uint32_t*>(X);
    const uint32_t w4 = (uint32_t)__cvta_generic_to_shared(sm + L::W4);
    const float2 b4 = reinterpret_cast<const float2*>(sm + L::B4)[t];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        uint32_t a0[1][4];
        a0[0][0] = Xw[(r0 * L::XLD + 2 * t) / 2];
        a0[0][1] = Xw[(r1 * L::XLD + 2 * t) / 2];
        a0[0][2] = Xw[(r0 * L::XLD + 2 * t + 8) / 2];
        a0[0][3] = Xw[(r1 * L::XLD + 2 * t + 8) / 2];
        uint32_t h1[4][4], h2[4][4];
        mlp_hidden<1, L::LD1>(sm, L::W1, L::B1, a0, h1, lane);
        mlp_hidden<4, L::LD>(sm, L::W2, L::B2, h1, h2, lane);
        mlp_hidden<4, L::LD>(sm, L::W3, L::B3, h2, h1, lane);
        // output layer: one 8-column tile, no activation
        float c[4] = {b4.x, b4.y, b4.x, b4.y};
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            uint32_t b[4];
            ldsm_x4(ldsm_row<L::LD>(w4, 0, 32 * sp, lane), b);
            mma_bf16_16816(c, h1[2 * sp], b[0], b[1]);
            mma_bf16_16816(c, h1[2 * sp + 1], b[2], b[3]);
        }
        __syncwarp();  // every lane has read this tile's inputs
        *reinterpret_cast<float2*>(Y + r0 * 8 + 2 * t) = make_float2(c[0], c[1]);
        *reinterpret_cast<float2*>(Y + r1 * 8 + 2 * t) = make_float2(c[2], c[3]);
    }
}

}  // namespace lbmk
