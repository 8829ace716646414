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
//   [10], output mean [6], output std [6] (f32, padded to 48).
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

// SiLU a * sigmoid(a) through sigmoid(a) = (1 + tanh(a / 2)) / 2 on the
// hardware tanh (one MUFU operation, relative error about 2^-11, below the BF16
// rounding that follows)
__device__ __forceinline__ float mlp_tanh(float v)
{
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float mlp_silu(float a)
{
    const float h = 0.5f * a;
    return fmaf(h, mlp_tanh(h), h);
}

// One hidden layer (64 outputs) for one 16-row tile: A fragments of the input
// (KS k-steps) -> A fragments of the output (4 k-steps of the next layer).
template <int KS, int LDW>
__device__ __forceinline__ void mlp_hidden(const unsigned char* sm, int woff, int boff, const uint32_t (&ain)[KS][4],
                                           uint32_t (&aout)[4][4], int g, int t)
{
    const uint32_t* W = reinterpret_cast<const uint32_t*>(sm + woff);
    const float* B = reinterpret_cast<const float*>(sm + boff);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const int row = 8 * nt + g;
#pragma unroll
        for (int s = 0; s < KS; ++s) {
            const uint32_t b0 = W[(row * LDW + 16 * s + 2 * t) / 2];
            const uint32_t b1 = W[(row * LDW + 16 * s + 2 * t + 8) / 2];
            mma_bf16_16816(c, ain[s], b0, b1);
        }
        const float bb0 = B[8 * nt + 2 * t], bb1 = B[8 * nt + 2 * t + 1];
        const uint32_t lo = pack_bf16(mlp_silu(c[0] + bb0), mlp_silu(c[1] + bb1));  // row g
        const uint32_t hi = pack_bf16(mlp_silu(c[2] + bb0), mlp_silu(c[3] + bb1));  // row g + 8
        if (nt & 1) {
            aout[nt >> 1][2] = lo;
            aout[nt >> 1][3] = hi;
        } else {
            aout[nt >> 1][0] = lo;
            aout[nt >> 1][1] = hi;
        }
    }
}

// Network forward for the warp's 32 cells: X [32][XLD] bf16 (standardised
// inputs, columns 10..15 zero) -> Y [32][8] f32 (standardised outputs 0..5);
// Y may alias X (the exchange layout above).
__device__ __forceinline__ void mlp_warp_forward(const unsigned char* sm, const __nv_bfloat16* X, float* Y, int lane)
{
    using L = MlpLayout;
    const int g = lane >> 2, t = lane & 3;
    const uint32_t* Xw = reinterpret_cast<const uint32_t*>(X);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        uint32_t a0[1][4];
        a0[0][0] = Xw[(r0 * L::XLD + 2 * t) / 2];
        a0[0][1] = Xw[(r1 * L::XLD + 2 * t) / 2];
        a0[0][2] = Xw[(r0 * L::XLD + 2 * t + 8) / 2];
        a0[0][3] = Xw[(r1 * L::XLD + 2 * t + 8) / 2];
        uint32_t h1[4][4], h2[4][4];
        mlp_hidden<1, L::LD1>(sm, L::W1, L::B1, a0, h1, g, t);
        mlp_hidden<4, L::LD>(sm, L::W2, L::B2, h1, h2, g, t);
        mlp_hidden<4, L::LD>(sm, L::W3, L::B3, h2, h1, g, t);
        // output layer: one 8-column tile, no activation
        const uint32_t* W = reinterpret_cast<const uint32_t*>(sm + L::W4);
        const float* B = reinterpret_cast<const float*>(sm + L::B4);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const uint32_t b0 = W[(g * L::LD + 16 * s + 2 * t) / 2];
            const uint32_t b1 = W[(g * L::LD + 16 * s + 2 * t + 8) / 2];
            mma_bf16_16816(c, h1[s], b0, b1);
        }
        __syncwarp();  // every lane has read this tile's inputs
        Y[r0 * 8 + 2 * t] = c[0] + B[2 * t];
        Y[r0 * 8 + 2 * t + 1] = c[1] + B[2 * t + 1];
        Y[r1 * 8 + 2 * t] = c[2] + B[2 * t];
        Y[r1 * 8 + 2 * t + 1] = c[3] + B[2 * t + 1];
    }
}

}  // namespace lbmk
