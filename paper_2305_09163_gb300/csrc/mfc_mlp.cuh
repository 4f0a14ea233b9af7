// Learned WENO weights: warp-level BF16 tensor-core building blocks.
//
// The paper has no learned part.  This network replaces the WENO5-JS
// nonlinear weights of Sec. 3.2: for a five-cell stencil v_{i-2..i+2} and the
// edge at i+1/2, inputs x_k = (v_{i+k} - v_i)/s with s = max_k |v_{i+k} - v_i|
// (+1e-30), layers 5 -> 32 -> 32 (ReLU) -> 3 (softmax), and the edge value
// v_i + sum_r omega_r (p_r - v_i) with the three WENO5 candidates p_r.
//
// Every layer runs on the tensor cores as mma.sync with BF16 operands and FP32
// accumulation, 16 stencils (one tile) per warp instruction stream: layer 1 is
// m16n8k8 (5 inputs padded to 8), layers 2 and 3 are m16n8k16.  The
// accumulator of one layer becomes the A operand of the next in registers
// (two adjacent n8 accumulator tiles have exactly the A-fragment layout), so a
// tile never leaves the register file between layers.
//
// Parameter blob (float32): W1[32][5], b1[32], W2[32][32], b2[32], W3[3][32], b3[3].
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mfc {

constexpr int kMlpH = 32;
constexpr int kMlpIn = 5;
constexpr int kMlpOut = 3;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpH * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpOut * kMlpH;
constexpr int kMlpParams = kOffB3 + kMlpOut;  // 1347

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// D += A(16x16, row) * B(16x8, col), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// D += A(16x8, row) * B(8x8, col), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma1688(float* d, const uint32_t* a, uint32_t b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b));
}

// D = A(16x16, row) * B(16x8, col) + C with C = (c0, c1) in both row halves:
// a bias enters as the accumulator input, with no register copies.
__device__ __forceinline__ void mma16816_bias(float* d, const uint32_t* a, const uint32_t* b, float c0, float c1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%10,%11};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(c0), "f"(c1));
}

// D = A(16x8, row) * B(8x8, col) + C, C as in mma16816_bias.
__device__ __forceinline__ void mma1688_bias(float* d, const uint32_t* a, uint32_t b, float c0, float c1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%7,%8};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b), "f"(c0), "f"(c1));
}

// Per-thread B fragments of the three layers and the biases of the columns
// this thread accumulates.  Lane = 4 g + t: a thread holds accumulator rows g,
// g+8 and columns 2t, 2t+1 of each n8 tile.
struct MlpWeights {
    uint32_t w1[4];         // layer 1, n-tiles 0..3: B[k][n] = W1[n][k], k < 5
    uint32_t w2[2][4][2];   // layer 2, k-steps 0..1, n-tiles 0..3: B[k][n] = W2[n][k]
    uint32_t w3[2][2];      // layer 3, k-steps 0..1, one n-tile (n < 3): B[k][n] = W3[n][k]
    float b1[4][2], b2[4][2], b3[2];
};

__device__ __forceinline__ void mlp_load_weights(const float* __restrict__ P, MlpWeights& W, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n = 8 * j + g;
        const int k = 2 * t;
        W.w1[j] = pack_bf16(k < kMlpIn ? P[kOffW1 + n * kMlpIn + k] : 0.f,
                            k + 1 < kMlpIn ? P[kOffW1 + n * kMlpIn + k + 1] : 0.f);
        W.b1[j][0] = P[kOffB1 + 8 * j + 2 * t];
        W.b1[j][1] = P[kOffB1 + 8 * j + 2 * t + 1];
        W.b2[j][0] = P[kOffB2 + 8 * j + 2 * t];
        W.b2[j][1] = P[kOffB2 + 8 * j + 2 * t + 1];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int k0 = 16 * s + 2 * t;
            W.w2[s][j][0] = pack_bf16(P[kOffW2 + n * kMlpH + k0], P[kOffW2 + n * kMlpH + k0 + 1]);
            W.w2[s][j][1] = pack_bf16(P[kOffW2 + n * kMlpH + k0 + 8], P[kOffW2 + n * kMlpH + k0 + 9]);
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int k0 = 16 * s + 2 * t;
        const bool ok = g < kMlpOut;
        W.w3[s][0] = ok ? pack_bf16(P[kOffW3 + g * kMlpH + k0], P[kOffW3 + g * kMlpH + k0 + 1]) : 0u;
        W.w3[s][1] = ok ? pack_bf16(P[kOffW3 + g * kMlpH + k0 + 8], P[kOffW3 + g * kMlpH + k0 + 9]) : 0u;
    }
    W.b3[0] = 2 * t < kMlpOut ? P[kOffB3 + 2 * t] : 0.f;
    W.b3[1] = 2 * t + 1 < kMlpOut ? P[kOffB3 + 2 * t + 1] : 0.f;
}

// The per-lane fragments of MlpWeights packed for one warp: word k of lane l
// at frag[k / 4][l] component k % 4, so each lane reads 11 16-byte words and
// a warp's 32 lanes read 512 contiguous bytes per word.  Built once per
// parameter set; the sweeps load it only when a warp has stencils for the
// network.
constexpr int kMlpFragVec = 11;   // uint4 per lane (42 words used)
constexpr int kMlpFragBytes = kMlpFragVec * 32 * 16;
static_assert(sizeof(MlpWeights) == 42 * 4, "MlpWeights is 42 words");

union MlpWeightsWords {
    MlpWeights w;
    uint4 v[kMlpFragVec];
};

__device__ __forceinline__ void mlp_weights_to_frag(const MlpWeights& W, uint4* __restrict__ F, int lane) {
    MlpWeightsWords u;
    u.v[kMlpFragVec - 1] = make_uint4(0u, 0u, 0u, 0u);
    u.w = W;
#pragma unroll
    for (int k = 0; k < kMlpFragVec; ++k) F[k * 32 + lane] = u.v[k];
}

__device__ __forceinline__ void mlp_weights_from_frag(const uint4* __restrict__ F, MlpWeights& W, int lane) {
    MlpWeightsWords u;
#pragma unroll
    for (int k = 0; k < kMlpFragVec; ++k) u.v[k] = __ldg(F + k * 32 + lane);
    W = u.w;
}

// max(lo, 0), max(hi, 0) rounded to BF16 and packed, in one conversion.
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Accumulator pair (two adjacent n8 tiles) after ReLU -> A fragment of the next layer.
__device__ __forceinline__ void relu_to_a(const float* c0, const float* c1, uint32_t* a) {
    a[0] = pack_bf16_relu(c0[0], c0[1]);
    a[1] = pack_bf16_relu(c0[2], c0[3]);
    a[2] = pack_bf16_relu(c1[0], c1[1]);
    a[3] = pack_bf16_relu(c1[2], c1[3]);
}

// Forward pass of one 16-stencil tile.  a_in is the m16n8k8 A fragment of the
// inputs (row g / g+8, columns 2t, 2t+1).  On return z holds the output
// logits (rows g, g+8; columns 2t, 2t+1; columns >= 3 are padding), c1/c2 the
// pre-activations and a1/a2 the BF16 activations (for backpropagation).
__device__ __forceinline__ void mlp_tile_forward(const MlpWeights& W, const uint32_t* a_in, float (&c1)[4][4],
                                                 uint32_t (&a1)[2][4], float (&c2)[4][4], uint32_t (&a2)[2][4],
                                                 float (&z)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c1[j][0] = c1[j][2] = W.b1[j][0];
        c1[j][1] = c1[j][3] = W.b1[j][1];
        mma1688(c1[j], a_in, W.w1[j]);
    }
    relu_to_a(c1[0], c1[1], a1[0]);
    relu_to_a(c1[2], c1[3], a1[1]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c2[j][0] = c2[j][2] = W.b2[j][0];
        c2[j][1] = c2[j][3] = W.b2[j][1];
        mma16816(c2[j], a1[0], W.w2[0][j]);
        mma16816(c2[j], a1[1], W.w2[1][j]);
    }
    relu_to_a(c2[0], c2[1], a2[0]);
    relu_to_a(c2[2], c2[3], a2[1]);
    z[0] = z[2] = W.b3[0];
    z[1] = z[3] = W.b3[1];
    mma16816(z, a2[0], W.w3[0]);
    mma16816(z, a2[1], W.w3[1]);
}

// Logits of one 16-stencil tile for inference (same arithmetic as
// mlp_tile_forward, without keeping the intermediate layers).
__device__ __forceinline__ void mlp_tile_logits(const MlpWeights& W, const uint32_t* a_in, float (&z)[4]) {
    float c[4][4];
    uint32_t a1[2][4], a2[2][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) mma1688_bias(c[j], a_in, W.w1[j], W.b1[j][0], W.b1[j][1]);
    relu_to_a(c[0], c[1], a1[0]);
    relu_to_a(c[2], c[3], a1[1]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        mma16816_bias(c[j], a1[0], W.w2[0][j], W.b2[j][0], W.b2[j][1]);
        mma16816(c[j], a1[1], W.w2[1][j]);
    }
    relu_to_a(c[0], c[1], a2[0]);
    relu_to_a(c[2], c[3], a2[1]);
    mma16816_bias(z, a2[0], W.w3[0], W.b3[0], W.b3[1]);
    mma16816(z, a2[1], W.w3[1]);
}

// Softmax of the three logits of rows g and g+8; valid in lanes with t == 0
// (the logit of column 2 lives in lane+1).  All 32 lanes must call it.
__device__ __forceinline__ void mlp_softmax_rows(const float (&z)[4], float (&om_g)[3], float (&om_g8)[3]) {
    const float z2g = __shfl_down_sync(0xffffffffu, z[0], 1);
    const float z2g8 = __shfl_down_sync(0xffffffffu, z[2], 1);
    {
        const float m = fmaxf(z[0], fmaxf(z[1], z2g));
        const float e0 = __expf(z[0] - m), e1 = __expf(z[1] - m), e2 = __expf(z2g - m);
        const float inv = __fdividef(1.f, e0 + e1 + e2);
        om_g[0] = e0 * inv; om_g[1] = e1 * inv; om_g[2] = e2 * inv;
    }
    {
        const float m = fmaxf(z[2], fmaxf(z[3], z2g8));
        const float e0 = __expf(z[2] - m), e1 = __expf(z[3] - m), e2 = __expf(z2g8 - m);
        const float inv = __fdividef(1.f, e0 + e1 + e2);
        om_g8[0] = e0 * inv; om_g8[1] = e1 * inv; om_g8[2] = e2 * inv;
    }
}

}  // namespace mfc
