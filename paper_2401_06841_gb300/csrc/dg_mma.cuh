// dg_mma.cuh -- BF16 tensor-core helpers shared by the tile kernels and the
// learned sensor: the m16n8k16 mma.sync, BF16 packing, and the evaluation of
// the sensor network (D -> 64 -> 64 -> 1, GELU) for 16 samples by one warp.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace dg {

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

constexpr int MLP_H = 64;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// GELU of the BF16 inference paths, with erf from Abramowitz & Stegun 7.1.26
// (Hastings' approximation: for x >= 0, erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 +
// t a5)))) exp(-x^2), t = 1/(1 + p x), absolute error <= 1.5e-7), far below the
// BF16 rounding (2^-9 relative) that the activation then takes:
//   gelu(z) = z - z erfc(|z|/sqrt 2)/2  (z >= 0),   z erfc(|z|/sqrt 2)/2  (z < 0)
__device__ __forceinline__ float gelu_infer(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float q = fmaf(t, 1.061405429f, -1.453152027f);
    q = fmaf(t, q, 1.421413741f);
    q = fmaf(t, q, -0.284496736f);
    q = fmaf(t, q, 0.254829592f);
    q *= t * __expf(-x * x);
    const float hz = 0.5f * z * q;
    return z >= 0.f ? z - hz : hz;
}

// packed inference weights: B1 = W1^T [KD][64], B2 = W2^T [64][64], B3 = W3 as
// [64][8] (column 0), each as fragments [K/16][N/8][32 lanes][2 words], then
// b1, b2, b3 as floats
template <int D>
struct MlpPack {
    static constexpr int KD = (D + 15) / 16 * 16;
    static constexpr int w1 = 0;                              // words
    static constexpr int w2 = w1 + (KD / 16) * 8 * 64;
    static constexpr int w3 = w2 + 4 * 8 * 64;
    static constexpr int bias = w3 + 4 * 1 * 64;              // floats b1[64], b2[64], b3
    static constexpr int words = bias + 2 * MLP_H + 1;
};

// One warp evaluates the network for the 16 samples r = 0..15 with BF16
// inputs, weights and hidden activations and FP32 accumulation; feat(r, k)
// gives input k of sample r (0 past the inputs).  On return the lanes with
// (lane & 3) == 0 hold y for samples lane/4 (y0) and lane/4 + 8 (y1).
// `packed` (shared or global) holds the MlpPack<D> block.
template <int D, typename F>
__device__ __forceinline__ void mlp_infer_warp(F&& feat, const uint32_t* packed, float& y0, float& y1)
{
    using PK = MlpPack<D>;
    constexpr int KT1 = PK::KD / 16;
    const uint2* B1 = reinterpret_cast<const uint2*>(packed + PK::w1);
    const uint2* B2 = reinterpret_cast<const uint2*>(packed + PK::w2);
    const uint2* B3 = reinterpret_cast<const uint2*>(packed + PK::w3);
    const float* bias = reinterpret_cast<const float*>(packed + PK::bias);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc1[j][0] = acc1[j][1] = acc1[j][2] = acc1[j][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KT1; ++kt) {
        const int k0 = kt * 16 + 2 * t;
        uint32_t A[4];
        A[0] = pack_bf16x2(feat(g, k0), feat(g, k0 + 1));
        A[1] = pack_bf16x2(feat(g + 8, k0), feat(g + 8, k0 + 1));
        A[2] = pack_bf16x2(feat(g, k0 + 8), feat(g, k0 + 9));
        A[3] = pack_bf16x2(feat(g + 8, k0 + 8), feat(g + 8, k0 + 9));
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint2 bw = B1[(kt * 8 + nt) * 32 + lane];
            mma_bf16(acc1[nt], A, bw.x, bw.y);
        }
    }
    // bias + GELU; the m16n8 accumulator tiles 2j, 2j+1 form the A operand of k-chunk j
    uint32_t A2[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float h[2][4];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int nt = 2 * j + s, c = nt * 8 + 2 * t;
            h[s][0] = gelu_infer(acc1[nt][0] + bias[c]);
            h[s][1] = gelu_infer(acc1[nt][1] + bias[c + 1]);
            h[s][2] = gelu_infer(acc1[nt][2] + bias[c]);
            h[s][3] = gelu_infer(acc1[nt][3] + bias[c + 1]);
        }
        A2[j][0] = pack_bf16x2(h[0][0], h[0][1]);
        A2[j][1] = pack_bf16x2(h[0][2], h[0][3]);
        A2[j][2] = pack_bf16x2(h[1][0], h[1][1]);
        A2[j][3] = pack_bf16x2(h[1][2], h[1][3]);
    }
    float acc2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc2[j][0] = acc2[j][1] = acc2[j][2] = acc2[j][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint2 bw = B2[(kt * 8 + nt) * 32 + lane];
            mma_bf16(acc2[nt], A2[kt], bw.x, bw.y);
        }
    uint32_t A3[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float h[2][4];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int nt = 2 * j + s, c = MLP_H + nt * 8 + 2 * t;
            h[s][0] = gelu_infer(acc2[nt][0] + bias[c]);
            h[s][1] = gelu_infer(acc2[nt][1] + bias[c + 1]);
            h[s][2] = gelu_infer(acc2[nt][2] + bias[c]);
            h[s][3] = gelu_infer(acc2[nt][3] + bias[c + 1]);
        }
        A3[j][0] = pack_bf16x2(h[0][0], h[0][1]);
        A3[j][1] = pack_bf16x2(h[0][2], h[0][3]);
        A3[j][2] = pack_bf16x2(h[1][0], h[1][1]);
        A3[j][3] = pack_bf16x2(h[1][2], h[1][3]);
    }
    float acc3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        const uint2 bw = B3[kt * 32 + lane];
        mma_bf16(acc3, A3[kt], bw.x, bw.y);
    }
    const float b3 = bias[2 * MLP_H];
    y0 = acc3[0] + b3;
    y1 = acc3[2] + b3;
}

}  // namespace dg
