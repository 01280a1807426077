// The learned brancher's network on the device: 16 features -> 64 -> 64 -> 1 score, ReLU,
// bfloat16 weights and activations, fp32 accumulation.  A warp scores 16 rows (variables)
// at a time with mma.sync m16n8k16 (the tensor-core path that a single warp can drive from
// inside the search kernel).
//
// Weights live in a "packed" block laid out in mma fragment order, so each lane loads its
// B fragment with one 8-byte load:
//   P1 [8 n-tiles][32 lanes][2 words]          W1 (16 x 64)
//   P2 [4 k-steps][8 n-tiles][32 lanes][2]     W2 (64 x 64)
//   P3 [4 k-steps][32 lanes][2]                w3 (64 x 1, column 0 of an 8-wide tile)
//   b1[64], b2[64], b3 as fp32
// Flat parameter order (the ABI's bf16 array): W1 row-major [in][out], b1, W2 [in][out], b2,
// w3, b3 — 5313 values.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace cubics {

constexpr int MLP_IN = 16, MLP_H = 64;
constexpr int MLP_PARAMS = 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1;     // 5313
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 1024, MLP_OFF_W2 = 1088, MLP_OFF_B2 = 5184,
              MLP_OFF_W3 = 5248, MLP_OFF_B3 = 5312;
constexpr int PK_P1 = 0, PK_P2 = 512, PK_P3 = 2560, PK_B1 = 2816, PK_B2 = 2880, PK_B3 = 2944;
constexpr int PK_WORDS = 2948;                                       // multiple of 4

__device__ __forceinline__ float bf16_to_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);     // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Packed word `i` of the fragment block from the flat bf16 parameters (one thread per word).
__device__ __forceinline__ uint32_t pack_word(const uint16_t *p, int i) {
    auto pair = [&](int off_lo, int off_hi) -> uint32_t {
        return (uint32_t)p[off_lo] | ((uint32_t)p[off_hi] << 16);
    };
    if (i < PK_P2) {                                    // W1: n-tile j, lane l, word w
        const int j = i / 64, l = (i / 2) % 32, w = i % 2;
        const int k = 2 * (l % 4) + 8 * w, n = 8 * j + l / 4;
        return pair(MLP_OFF_W1 + k * 64 + n, MLP_OFF_W1 + (k + 1) * 64 + n);
    }
    if (i < PK_P3) {                                    // W2: k-step kk, n-tile j, lane, word
        const int r = i - PK_P2;
        const int kk = r / 512, j = (r / 64) % 8, l = (r / 2) % 32, w = r % 2;
        const int k = 16 * kk + 2 * (l % 4) + 8 * w, n = 8 * j + l / 4;
        return pair(MLP_OFF_W2 + k * 64 + n, MLP_OFF_W2 + (k + 1) * 64 + n);
    }
    if (i < PK_B1) {                                    // w3 in column 0 of an 8-wide tile
        const int r = i - PK_P3;
        const int kk = r / 64, l = (r / 2) % 32, w = r % 2;
        if (l / 4 != 0) return 0u;
        const int k = 16 * kk + 2 * (l % 4) + 8 * w;
        return pair(MLP_OFF_W3 + k, MLP_OFF_W3 + k + 1);
    }
    if (i < PK_B2) return __float_as_uint(bf16_to_f(p[MLP_OFF_B1 + i - PK_B1]));
    if (i < PK_B3) return __float_as_uint(bf16_to_f(p[MLP_OFF_B2 + i - PK_B2]));
    if (i == PK_B3) return __float_as_uint(bf16_to_f(p[MLP_OFF_B3]));
    return 0u;
}

// Scores of 16 rows.  `x(r, c)` returns the bf16x2 pair of features (c, c + 1) of row r of
// the tile; `pk(i)` returns packed word i.  Lanes with (lane & 3) == 0 receive the scores
// of rows lane/4 (s_lo) and lane/4 + 8 (s_hi).
template <typename XF, typename PF>
__device__ __forceinline__ void mlp_tile(XF x, PF pk, float &s_lo, float &s_hi) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t a0 = x(g, 2 * t), a1 = x(g + 8, 2 * t), a2 = x(g, 2 * t + 8), a3 = x(g + 8, 2 * t + 8);
    float h1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        h1[j][0] = h1[j][1] = h1[j][2] = h1[j][3] = 0.f;
        mma_bf16(h1[j], a0, a1, a2, a3, pk(PK_P1 + 64 * j + 2 * lane), pk(PK_P1 + 64 * j + 2 * lane + 1));
    }
    // bias, ReLU and bf16: the accumulator of n-tiles 2kk, 2kk + 1 is the A fragment of k-step kk
    uint32_t A2[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * kk + h;
            const float bl = __uint_as_float(pk(PK_B1 + 8 * j + 2 * t));
            const float bh = __uint_as_float(pk(PK_B1 + 8 * j + 2 * t + 1));
            A2[kk][2 * h + 0] = pack_bf16(fmaxf(h1[j][0] + bl, 0.f), fmaxf(h1[j][1] + bh, 0.f));
            A2[kk][2 * h + 1] = pack_bf16(fmaxf(h1[j][2] + bl, 0.f), fmaxf(h1[j][3] + bh, 0.f));
        }
    }
    float h2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        h2[j][0] = h2[j][1] = h2[j][2] = h2[j][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int o = PK_P2 + 512 * kk + 64 * j + 2 * lane;
            mma_bf16(h2[j], A2[kk][0], A2[kk][1], A2[kk][2], A2[kk][3], pk(o), pk(o + 1));
        }
    }
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        uint32_t a[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * kk + h;
            const float bl = __uint_as_float(pk(PK_B2 + 8 * j + 2 * t));
            const float bh = __uint_as_float(pk(PK_B2 + 8 * j + 2 * t + 1));
            a[2 * h + 0] = pack_bf16(fmaxf(h2[j][0] + bl, 0.f), fmaxf(h2[j][1] + bh, 0.f));
            a[2 * h + 1] = pack_bf16(fmaxf(h2[j][2] + bl, 0.f), fmaxf(h2[j][3] + bh, 0.f));
        }
        const int o = PK_P3 + 64 * kk + 2 * lane;
        mma_bf16(s, a[0], a[1], a[2], a[3], pk(o), pk(o + 1));
    }
    const float b3 = __uint_as_float(pk(PK_B3));
    s_lo = s[0] + b3;
    s_hi = s[2] + b3;
}

}  // namespace cubics
