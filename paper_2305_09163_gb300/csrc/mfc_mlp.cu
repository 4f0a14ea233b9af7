// Learned WENO weights: training kernels and their C ABI (include/mfc.h).
//
//   mfc_mlp_forward  weights omega for a batch of normalised stencils
//   mfc_mlp_grad_mma loss and gradient of a batch (forward + backpropagation)
//                    on warp-level mma.sync; mfc_mlp_grad (mfc_mlp_tc.cu) is
//                    the same on the fifth-generation tensor cores
//   mfc_mlp_adam     Adam update of the parameter blob
//   mfc_harvest      training samples from a fine primitive field: coarse
//                    (2x restricted) stencils, WENO5 candidates, the fine-grid
//                    face value as target, the WENO5-JS value and a sensor flag
//
// The paper has no learned part; the network replaces the WENO5-JS nonlinear
// weights of Sec. 3.2.  Every matrix product of the forward and backward pass
// (including the batch reductions that form the weight gradients) runs on the
// tensor cores as mma.sync with BF16 operands and FP32 accumulation.
#include <cmath>
#include <cstdint>

#include "../../include/mfc.h"
#include "mfc_device.cuh"
#include "mfc_mlp.cuh"

using namespace mfc;

namespace {

constexpr int kGradWarps = 4;
constexpr int kGradBlocks = MFC_MLP_GRAD_BLOCKS;
constexpr int kGradStride = kMlpParams + 1;  // parameters + loss
static_assert(kMlpParams == MFC_MLP_PARAMS, "parameter count");
static_assert((long long)kGradBlocks * kGradWarps * kGradStride == MFC_MLP_WORK_FLOATS, "workspace size");

__device__ __constant__ float kIdeal[3] = {0.1f, 0.6f, 0.3f};

// A fragment (m16n8k8) of the inputs of rows row0+g and row0+g+8.
__device__ __forceinline__ void load_inputs(const float* __restrict__ x, long long B, long long row0, int g, int t,
                                            uint32_t* a) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long r = row0 + g + 8 * h;
        const int k = 2 * t;
        float v0 = 0.f, v1 = 0.f;
        if (r < B) {
            if (k < kMlpIn) v0 = x[r * kMlpIn + k];
            if (k + 1 < kMlpIn) v1 = x[r * kMlpIn + k + 1];
        }
        a[h] = pack_bf16(v0, v1);
    }
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ x,
                                                          long long B, float* __restrict__ omega) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    MlpWeights W;
    mlp_load_weights(P, W, lane);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long tile = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < B; tile += nw) {
        uint32_t a_in[2];
        load_inputs(x, B, tile * 16, g, t, a_in);
        float c1[4][4], c2[4][4], z[4];
        uint32_t a1[2][4], a2[2][4];
        mlp_tile_forward(W, a_in, c1, a1, c2, a2, z);
        float og[3], og8[3];
        mlp_softmax_rows(z, og, og8);
        if (t == 0) {
            const long long r = tile * 16 + g;
            if (r < B)
                for (int q = 0; q < 3; ++q) omega[r * 3 + q] = og[q];
            if (r + 8 < B)
                for (int q = 0; q < 3; ++q) omega[(r + 8) * 3 + q] = og8[q];
        }
    }
}

// bf16 element (row, col) of a row-major tile stored as 32-bit pairs.
__device__ __forceinline__ uint32_t elem16(const uint32_t* tile, int words_per_row, int row, int col) {
    const uint32_t w = tile[row * words_per_row + (col >> 1)];
    return (col & 1) ? (w >> 16) : (w & 0xFFFFu);
}

__device__ __forceinline__ uint32_t pair16(uint32_t lo, uint32_t hi) { return lo | (hi << 16); }

// A fragment (m16n8k16) of the transpose of a [16 samples][cols] tile:
// A[m][k] = tile[k][col0 + m], rows m >= mmax are zero.
__device__ __forceinline__ void transposed_a(const uint32_t* tile, int wpr, int col0, int mmax, int g, int t,
                                             uint32_t* a) {
    const int m0 = g, m1 = g + 8;
    const int k0 = 2 * t, k1 = 2 * t + 8;
    a[0] = m0 < mmax ? pair16(elem16(tile, wpr, k0, col0 + m0), elem16(tile, wpr, k0 + 1, col0 + m0)) : 0u;
    a[1] = m1 < mmax ? pair16(elem16(tile, wpr, k0, col0 + m1), elem16(tile, wpr, k0 + 1, col0 + m1)) : 0u;
    a[2] = m0 < mmax ? pair16(elem16(tile, wpr, k1, col0 + m0), elem16(tile, wpr, k1 + 1, col0 + m0)) : 0u;
    a[3] = m1 < mmax ? pair16(elem16(tile, wpr, k1, col0 + m1), elem16(tile, wpr, k1 + 1, col0 + m1)) : 0u;
}

// B fragment (m16n8k16) of a [16 samples][cols] tile: B[k][n] = tile[k][col0 + n].
__device__ __forceinline__ void tile_b(const uint32_t* tile, int wpr, int col0, int g, int t, uint32_t* b) {
    const int k0 = 2 * t, k1 = 2 * t + 8;
    b[0] = pair16(elem16(tile, wpr, k0, col0 + g), elem16(tile, wpr, k0 + 1, col0 + g));
    b[1] = pair16(elem16(tile, wpr, k1, col0 + g), elem16(tile, wpr, k1 + 1, col0 + g));
}

__device__ __forceinline__ void to_a(const float* c0, const float* c1, uint32_t* a) {
    a[0] = pack_bf16(c0[0], c0[1]);
    a[1] = pack_bf16(c0[2], c0[3]);
    a[2] = pack_bf16(c1[0], c1[1]);
    a[3] = pack_bf16(c1[2], c1[3]);
}

// Store an A fragment pair (16 x 32 bf16 tile in two k-steps) to a row-major tile.
__device__ __forceinline__ void store_a32(uint32_t* tile, const uint32_t (&a)[2][4], int g, int t) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        tile[g * 16 + 8 * s + t] = a[s][0];
        tile[(g + 8) * 16 + 8 * s + t] = a[s][1];
        tile[g * 16 + 8 * s + 4 + t] = a[s][2];
        tile[(g + 8) * 16 + 8 * s + 4 + t] = a[s][3];
    }
}

struct GradShared {
    uint32_t h1[16 * 16], h2[16 * 16], da2[16 * 16], da1[16 * 16];  // [16 rows][32 bf16]
    uint32_t dz[16 * 4], xin[16 * 4];                                // [16 rows][8 bf16]
};

__global__ void __launch_bounds__(kGradWarps * 32) mlp_grad_kernel(
    const float* __restrict__ P, const float* __restrict__ x, const float* __restrict__ phat,
    const float* __restrict__ target, const float* __restrict__ mask, long long B, float lam,
    float* __restrict__ work) {
    __shared__ GradShared sh[kGradWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    GradShared& S = sh[warp];
    MlpWeights W;
    mlp_load_weights(P, W, lane);
    // backward B fragments: dh2 = dz W3 (B[k][n] = W3[k][n], k < 3) and dh1 = da2 W2 (B[k][n] = W2[k][n])
    uint32_t w3t[4][2], w2t[2][4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n = 8 * j + g;
        const int k = 2 * t;
        w3t[j][0] = pack_bf16(k < 3 ? P[kOffW3 + k * kMlpH + n] : 0.f, k + 1 < 3 ? P[kOffW3 + (k + 1) * kMlpH + n] : 0.f);
        w3t[j][1] = 0u;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int k0 = 16 * s + 2 * t;
            w2t[s][j][0] = pack_bf16(P[kOffW2 + k0 * kMlpH + n], P[kOffW2 + (k0 + 1) * kMlpH + n]);
            w2t[s][j][1] = pack_bf16(P[kOffW2 + (k0 + 8) * kMlpH + n], P[kOffW2 + (k0 + 9) * kMlpH + n]);
        }
    }
    float gW3[4][4], gW2[2][4][4], gW1[2][4], gb1[4][2], gb2[4][2], gb3[3] = {0.f, 0.f, 0.f}, lsum = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        gb1[j][0] = gb1[j][1] = gb2[j][0] = gb2[j][1] = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) { gW3[j][e] = 0.f; gW2[0][j][e] = 0.f; gW2[1][j][e] = 0.f; }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) { gW1[0][e] = 0.f; gW1[1][e] = 0.f; }
    const float invB = 1.0f / (float)B;

    const long long nw = (long long)gridDim.x * kGradWarps;
    for (long long tile = (long long)blockIdx.x * kGradWarps + warp; tile * 16 < B; tile += nw) {
        const long long row0 = tile * 16;
        uint32_t a_in[2];
        load_inputs(x, B, row0, g, t, a_in);
        float c1[4][4], c2[4][4], z[4];
        uint32_t a1[2][4], a2[2][4];
        mlp_tile_forward(W, a_in, c1, a1, c2, a2, z);
        float og[3], og8[3];
        mlp_softmax_rows(z, og, og8);
        // loss and dL/dz on the t == 0 lanes for rows g and g+8
        float dzg[3] = {0.f, 0.f, 0.f}, dzg8[3] = {0.f, 0.f, 0.f};
        if (t == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long r = row0 + g + 8 * h;
                if (r < B) {
                    const float* om = h ? og8 : og;
                    float* dz = h ? dzg8 : dzg;
                    const float p0 = phat[r * 3], p1 = phat[r * 3 + 1], p2 = phat[r * 3 + 2];
                    const float tt = target[r], mk = mask[r];
                    const float y = om[0] * p0 + om[1] * p1 + om[2] * p2;
                    const float e = y - tt;
                    float dom[3];
                    const float pp[3] = {p0, p1, p2};
                    float reg = 0.f;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float dd = om[q] - kIdeal[q];
                        reg += dd * dd;
                        dom[q] = 2.f * invB * (e * pp[q] + lam * mk * dd);
                    }
                    lsum += invB * (e * e + lam * mk * reg);
                    const float sdot = om[0] * dom[0] + om[1] * dom[1] + om[2] * dom[2];
#pragma unroll
                    for (int q = 0; q < 3; ++q) dz[q] = om[q] * (dom[q] - sdot);
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) gb3[q] += dzg[q] + dzg8[q];
        }
        // dz as an A fragment (columns 0..2): lane t=1 takes column 2 from lane t=0
        const float v2g = __shfl_up_sync(0xffffffffu, dzg[2], 1);
        const float v2g8 = __shfl_up_sync(0xffffffffu, dzg8[2], 1);
        uint32_t a_dz[4];
        a_dz[0] = t == 0 ? pack_bf16(dzg[0], dzg[1]) : (t == 1 ? pack_bf16(v2g, 0.f) : 0u);
        a_dz[1] = t == 0 ? pack_bf16(dzg8[0], dzg8[1]) : (t == 1 ? pack_bf16(v2g8, 0.f) : 0u);
        a_dz[2] = 0u;
        a_dz[3] = 0u;
        // dh2 = dz W3, da2 = dh2 * (a2 > 0)
        float da2[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816(d, a_dz, w3t[j]);
#pragma unroll
            for (int e = 0; e < 4; ++e) da2[j][e] = c2[j][e] > 0.f ? d[e] : 0.f;
            gb2[j][0] += da2[j][0] + da2[j][2];
            gb2[j][1] += da2[j][1] + da2[j][3];
        }
        uint32_t a_da2[2][4];
        to_a(da2[0], da2[1], a_da2[0]);
        to_a(da2[2], da2[3], a_da2[1]);
        // dh1 = da2 W2, da1 = dh1 * (a1 > 0)
        float da1[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816(d, a_da2[0], w2t[0][j]);
            mma16816(d, a_da2[1], w2t[1][j]);
#pragma unroll
            for (int e = 0; e < 4; ++e) da1[j][e] = c1[j][e] > 0.f ? d[e] : 0.f;
            gb1[j][0] += da1[j][0] + da1[j][2];
            gb1[j][1] += da1[j][1] + da1[j][3];
        }
        uint32_t a_da1[2][4];
        to_a(da1[0], da1[1], a_da1[0]);
        to_a(da1[2], da1[3], a_da1[1]);
        // stage the tiles whose transposes form the weight gradients
        store_a32(S.h1, a1, g, t);
        store_a32(S.h2, a2, g, t);
        store_a32(S.da2, a_da2, g, t);
        store_a32(S.da1, a_da1, g, t);
        S.dz[g * 4 + t] = a_dz[0];
        S.dz[(g + 8) * 4 + t] = a_dz[1];
        S.xin[g * 4 + t] = a_in[0];
        S.xin[(g + 8) * 4 + t] = a_in[1];
        __syncwarp();
        // dW3 += dz^T h2  (16 x 32, rows 0..2 meaningful)
        {
            uint32_t a[4];
            transposed_a(S.dz, 4, 0, 3, g, t, a);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t b[2];
                tile_b(S.h2, 16, 8 * j, g, t, b);
                mma16816(gW3[j], a, b);
            }
        }
        // dW2 += da2^T h1 (32 x 32) and dW1 += da1^T x (32 x 8)
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            uint32_t a[4];
            transposed_a(S.da2, 16, 16 * mi, 16, g, t, a);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t b[2];
                tile_b(S.h1, 16, 8 * j, g, t, b);
                mma16816(gW2[mi][j], a, b);
            }
            uint32_t a1t[4], bx[2];
            transposed_a(S.da1, 16, 16 * mi, 16, g, t, a1t);
            tile_b(S.xin, 4, 0, g, t, bx);
            mma16816(gW1[mi], a1t, bx);
        }
        __syncwarp();
    }
    // reduce the bias partials and the loss over the eight row groups (lane bits 2..4)
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            gb1[j][0] += __shfl_xor_sync(0xffffffffu, gb1[j][0], o);
            gb1[j][1] += __shfl_xor_sync(0xffffffffu, gb1[j][1], o);
            gb2[j][0] += __shfl_xor_sync(0xffffffffu, gb2[j][0], o);
            gb2[j][1] += __shfl_xor_sync(0xffffffffu, gb2[j][1], o);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) gb3[q] += __shfl_xor_sync(0xffffffffu, gb3[q], o);
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    float* out = work + ((long long)blockIdx.x * kGradWarps + warp) * kGradStride;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (g < 3) {
            out[kOffW3 + g * kMlpH + 8 * j + 2 * t] = gW3[j][0];
            out[kOffW3 + g * kMlpH + 8 * j + 2 * t + 1] = gW3[j][1];
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const int r0 = 16 * mi + g, r1 = r0 + 8, c = 8 * j + 2 * t;
            out[kOffW2 + r0 * kMlpH + c] = gW2[mi][j][0];
            out[kOffW2 + r0 * kMlpH + c + 1] = gW2[mi][j][1];
            out[kOffW2 + r1 * kMlpH + c] = gW2[mi][j][2];
            out[kOffW2 + r1 * kMlpH + c + 1] = gW2[mi][j][3];
        }
        if (g == 0) {
            out[kOffB1 + 8 * j + 2 * t] = gb1[j][0];
            out[kOffB1 + 8 * j + 2 * t + 1] = gb1[j][1];
            out[kOffB2 + 8 * j + 2 * t] = gb2[j][0];
            out[kOffB2 + 8 * j + 2 * t + 1] = gb2[j][1];
        }
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int r0 = 16 * mi + g, r1 = r0 + 8;
        const int c = 2 * t;
        if (c < kMlpIn) {
            out[kOffW1 + r0 * kMlpIn + c] = gW1[mi][0];
            out[kOffW1 + r1 * kMlpIn + c] = gW1[mi][2];
        }
        if (c + 1 < kMlpIn) {
            out[kOffW1 + r0 * kMlpIn + c + 1] = gW1[mi][1];
            out[kOffW1 + r1 * kMlpIn + c + 1] = gW1[mi][3];
        }
    }
    if (lane == 0) {
        for (int q = 0; q < 3; ++q) out[kOffB3 + q] = gb3[q];
        out[kMlpParams] = lsum;
    }
}

// Deterministic sum of the per-warp partials: one thread per slot.
__global__ void mlp_reduce_kernel(const float* __restrict__ work, int parts, float* __restrict__ grad,
                                  float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    float s = 0.f;
    for (int w = 0; w < parts; ++w) s += work[(long long)w * kGradStride + p];
    if (p < kMlpParams) grad[p] = s;
    else if (loss) *loss = s;
}

// Adam (Kingma & Ba 2015): bias corrections c1 = 1/(1-b1^t), c2 = 1/(1-b2^t).
__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                                float* __restrict__ V, int n, float lr, float b1, float b2, float eps, float c1,
                                float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = G[i];
    const float m = b1 * M[i] + (1.f - b1) * gi;
    const float v = b2 * V[i] + (1.f - b2) * gi * gi;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

// ---------------------------------------------------------------------------
// Sample harvest.  Sample k picks (by a counter-based hash of seed and k) an
// active direction d, a coarse face I+1/2 of the 2x-restricted grid, the
// transverse coarse cell, a variable and a side: side 0 is the edge of cell I
// (stencil I-2..I+2), side 1 the edge of cell I+1 (stencil I+3..I-1, reversed).
// The coarse value of a cell is the mean of the primitives of its 2^ndim fine
// children.  The target is the fine-grid face value at the coincident fine face,
// 1/2 (left + right WENO5-JS edge values of the fine run), averaged over the
// 2^(ndim-1) fine faces that tile the coarse face.  All in FP64, stored FP32
// and normalised by the stencil scale s.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Textbook WENO5-JS value at the right edge of the middle cell of v[0..4].
__device__ double weno5_js(const double* v, double eps) {
    const double p0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
    const double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
    const double p2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
    double q;
    q = v[0] - 2.0 * v[1] + v[2];
    double b0 = 13.0 / 12.0 * q * q;
    q = v[0] - 4.0 * v[1] + 3.0 * v[2];
    b0 += 0.25 * q * q;
    q = v[1] - 2.0 * v[2] + v[3];
    double b1 = 13.0 / 12.0 * q * q;
    q = v[1] - v[3];
    b1 += 0.25 * q * q;
    q = v[2] - 2.0 * v[3] + v[4];
    double b2 = 13.0 / 12.0 * q * q;
    q = 3.0 * v[2] - 4.0 * v[3] + v[4];
    b2 += 0.25 * q * q;
    const double a0 = 0.1 / ((eps + b0) * (eps + b0));
    const double a1 = 0.6 / ((eps + b1) * (eps + b1));
    const double a2 = 0.3 / ((eps + b2) * (eps + b2));
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

__global__ void harvest_kernel(const double* __restrict__ wf, int nxf, int nyf, int nzf, int ndim, int ns,
                               double eps, double tau, long long nsamp, unsigned long long seed,
                               float* __restrict__ xo, float* __restrict__ po, float* __restrict__ to,
                               float* __restrict__ so, float* __restrict__ jo) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsamp) return;
    const long long nf = (long long)nxf * nyf * nzf;
    const int nfd[3] = {nxf, nyf, nzf};
    int nc[3];
    for (int a = 0; a < 3; ++a) nc[a] = a < ndim ? nfd[a] / 2 : 1;
    const unsigned long long h0 = mix64(seed ^ mix64((unsigned long long)k));
    const unsigned long long h1 = mix64(h0), h2 = mix64(h1), h3 = mix64(h2);
    const int d = (int)(h0 % (unsigned long long)ndim);
    const int side = (int)((h0 >> 20) & 1ULL);
    const int var = (int)((h0 >> 24) % (unsigned long long)ns);
    const int I = 2 + (int)(h1 % (unsigned long long)(nc[d] - 6));
    int cc[3];
    cc[0] = (int)(h2 % (unsigned long long)nc[0]);
    cc[1] = (int)((h2 >> 21) % (unsigned long long)nc[1]);
    cc[2] = (int)((h3) % (unsigned long long)nc[2]);
    const long long sf[3] = {1, (long long)nxf, (long long)nxf * nyf};
    const double* wv = wf + (long long)var * nf;
    const int nchild = 1 << ndim;
    // coarse values of cells I-2..I+3 along d
    double W[6];
    for (int m = 0; m < 6; ++m) {
        int c[3] = {cc[0], cc[1], cc[2]};
        c[d] = I - 2 + m;
        double s = 0.0;
        for (int ch = 0; ch < nchild; ++ch) {
            long long idx = 0;
            for (int a = 0; a < 3; ++a) {
                const int f = a < ndim ? 2 * c[a] + ((ch >> a) & 1) : 0;
                idx += f * sf[a];
            }
            s += wv[idx];
        }
        W[m] = s / nchild;
    }
    double st[5];
    for (int m = 0; m < 5; ++m) st[m] = side == 0 ? W[m] : W[5 - m];
    // fine target: faces between fine cells 2I+1 and 2I+2 along d
    double tgt = 0.0;
    const int ntr = nchild / 2;
    for (int ch = 0; ch < ntr; ++ch) {
        long long base = 0;
        int bit = 0;
        for (int a = 0; a < 3; ++a) {
            if (a == d) continue;
            const int f = a < ndim ? 2 * cc[a] + ((ch >> bit) & 1) : 0;
            if (a < ndim) ++bit;
            base += f * sf[a];
        }
        double f6[6];
        for (int m = 0; m < 6; ++m) f6[m] = wv[base + (long long)(2 * I - 1 + m) * sf[d]];
        const double l = weno5_js(f6, eps);
        const double rv[5] = {f6[5], f6[4], f6[3], f6[2], f6[1]};
        const double r = weno5_js(rv, eps);
        tgt += 0.5 * (l + r);
    }
    tgt /= ntr;
    const double c = st[2];
    double s = 0.0;
    for (int m = 0; m < 5; ++m) s = fmax(s, fabs(st[m] - c));
    const double tn = (tgt - c) / (s + 1e-30);
    // A stencil flat to FP32 resolution of its centre value carries no shape to
    // learn (its normalised target would be round-off); such samples, and any
    // whose fine target lies far outside the stencil's range, are stored as
    // zeros with smooth = 0 so they add nothing to the loss.
    if (!(s > 1e-7 * fabs(c)) || !(s > 1e-300) || !(fabs(tn) <= 8.0)) {
        for (int m = 0; m < 5; ++m) xo[k * 5 + m] = 0.f;
        po[k * 3 + 0] = po[k * 3 + 1] = po[k * 3 + 2] = 0.f;
        to[k] = 0.f;
        jo[k] = 0.f;
        so[k] = 0.f;
        return;
    }
    s += 1e-30;
    for (int m = 0; m < 5; ++m) xo[k * 5 + m] = (float)((st[m] - c) / s);
    const double p0 = (2.0 * st[0] - 7.0 * st[1] + 11.0 * st[2]) / 6.0;
    const double p1 = (-st[1] + 5.0 * st[2] + 2.0 * st[3]) / 6.0;
    const double p2 = (2.0 * st[2] + 5.0 * st[3] - st[4]) / 6.0;
    po[k * 3 + 0] = (float)((p0 - c) / s);
    po[k * 3 + 1] = (float)((p1 - c) / s);
    po[k * 3 + 2] = (float)((p2 - c) / s);
    to[k] = (float)tn;
    jo[k] = (float)((weno5_js(st, eps) - c) / s);
    // discontinuity sensor (the same test the learned sweep applies)
    const double D0 = st[1] - st[0], D1 = st[2] - st[1], D2 = st[3] - st[2], D3 = st[4] - st[3];
    const double bb0 = 2.5 * D1 * D1 - 2.75 * D1 * D0 + D0 * D0;
    const double bb1 = D1 * D1 + D2 * D2 - 1.25 * D1 * D2;
    const double bb2 = 2.5 * D2 * D2 - 2.75 * D2 * D3 + D3 * D3;
    const double bmax = fmax(bb0, fmax(bb1, bb2)), bmin = fmin(bb0, fmin(bb1, bb2));
    so[k] = bmax > tau * (bmin + 1e-6 * s * s) ? 0.f : 1.f;
}

__global__ void __launch_bounds__(256) prims_out_kernel(const double* __restrict__ q, double* __restrict__ w,
                                                        long long nc, int nf, int ndim, EosConst e, int six) {
    // generic (runtime NF, NDIM) FP64 primitive recovery for output; the
    // six-equation model (six) appends the phase pressures
    // p_k = (a_k r_k e_k / a_k - P_k)/G_k
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
         i += (long long)gridDim.x * blockDim.x) {
        const int ns = 2 * nf + ndim, IM = nf, IE = nf + ndim, IA = nf + ndim + 1;
        double rho = 0.0;
        for (int k2 = 0; k2 < nf; ++k2) rho += q[k2 * nc + i];
        double G = e.G_N, Pm = e.P_N;
        for (int k2 = 0; k2 < nf - 1; ++k2) {
            G = fma(q[(IA + k2) * nc + i], e.dG[k2], G);
            Pm = fma(q[(IA + k2) * nc + i], e.dP[k2], Pm);
        }
        double ke = 0.0;
        for (int a = 0; a < ndim; ++a) {
            const double u = q[(IM + a) * nc + i] / rho;
            w[(IM + a) * nc + i] = u;
            ke = fma(q[(IM + a) * nc + i], u, ke);
        }
        for (int k2 = 0; k2 < nf; ++k2) w[k2 * nc + i] = q[k2 * nc + i];
        w[IE * nc + i] = (q[IE * nc + i] - 0.5 * ke - Pm) / G;
        for (int k2 = IA; k2 < ns; ++k2) w[k2 * nc + i] = q[k2 * nc + i];
        if (six) {
            double aN = 1.0;
            for (int k2 = 0; k2 < nf; ++k2) {
                const double ak = k2 < nf - 1 ? q[(IA + k2) * nc + i] : aN;
                if (k2 < nf - 1) aN -= ak;
                const double Gk = k2 < nf - 1 ? e.G_N + e.dG[k2] : e.G_N;
                const double Pk = k2 < nf - 1 ? e.P_N + e.dP[k2] : e.P_N;
                w[(ns + k2) * nc + i] = (q[(ns + k2) * nc + i] / ak - Pk) / Gk;
            }
        }
    }
}

// One warp: the per-lane MMA fragments of a parameter blob, for the sweeps.
__global__ void __launch_bounds__(32) mlp_pack_kernel(const float* __restrict__ P, uint4* __restrict__ frag) {
    MlpWeights W;
    mlp_load_weights(P, W, threadIdx.x);
    mlp_weights_to_frag(W, frag, threadIdx.x);
}

}  // namespace

// Host launcher used by mfc_set_mlp: frag holds kMlpFragBytes.
cudaError_t mfc_launch_mlp_pack(const float* P, void* frag, cudaStream_t s) {
    mlp_pack_kernel<<<1, 32, 0, s>>>(P, static_cast<uint4*>(frag));
    return cudaGetLastError();
}

// Host launcher used by mfc_get_prims in the context code.
cudaError_t mfc_launch_prims_out(const double* q, double* w, long long nc, int nf, int ndim, const EosConst& e,
                                 int six, cudaStream_t s) {
    long long b = (nc + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    prims_out_kernel<<<(unsigned)b, 256, 0, s>>>(q, w, nc, nf, ndim, e, six);
    return cudaGetLastError();
}

extern "C" {

mfc_status mfc_mlp_forward(const float* params, const float* x, long long batch, float* omega, void* stream) {
    if (!params || !x || !omega || batch <= 0) return MFC_ERR_ARG;
    const long long tiles = (batch + 15) / 16;
    long long blocks = (tiles + 3) / 4;
    if (blocks > 152 * 8) blocks = 152 * 8;
    mlp_forward_kernel<<<(unsigned)blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(params, x, batch, omega);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ERR_CUDA;
}

mfc_status mfc_mlp_grad_mma(const float* params, const float* x, const float* phat, const float* target,
                            const float* mask, long long batch, float lam, float* grad, float* loss, float* work,
                            void* stream) {
    if (!params || !x || !phat || !target || !mask || !grad || !work || batch <= 0 || !(lam >= 0.f))
        return MFC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mlp_grad_kernel<<<kGradBlocks, kGradWarps * 32, 0, s>>>(params, x, phat, target, mask, batch, lam, work);
    if (cudaGetLastError() != cudaSuccess) return MFC_ERR_CUDA;
    mlp_reduce_kernel<<<(kGradStride + 127) / 128, 128, 0, s>>>(work, kGradBlocks * kGradWarps, grad, loss);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ERR_CUDA;
}

mfc_status mfc_mlp_adam(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1,
                        float beta2, float eps, int step, void* stream) {
    if (!params || !grad || !m || !v || n <= 0 || step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
        return MFC_ERR_ARG;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
    mlp_adam_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, n, lr, beta1,
                                                                                  beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ERR_CUDA;
}

mfc_status mfc_harvest(const double* w_fine, int nxf, int nyf, int nzf, int num_fluids, double weno_eps, double tau,
                       long long n_samples, unsigned long long seed, float* x, float* phat, float* target,
                       float* smooth, float* js, void* stream) {
    if (!w_fine || !x || !phat || !target || !smooth || !js || n_samples <= 0) return MFC_ERR_ARG;
    if (num_fluids < 1 || num_fluids > 3 || !(weno_eps > 0.0) || !(tau > 0.0)) return MFC_ERR_ARG;
    const int ndim = nzf > 1 ? 3 : (nyf > 1 ? 2 : 1);
    const int nfd[3] = {nxf, nyf, nzf};
    for (int a = 0; a < 3; ++a) {
        if (a < ndim && (nfd[a] % 2 != 0 || nfd[a] / 2 < 8)) return MFC_ERR_ARG;
        if (a >= ndim && nfd[a] != 1) return MFC_ERR_ARG;
    }
    const int ns = 2 * num_fluids + ndim;
    const long long blocks = (n_samples + 127) / 128;
    harvest_kernel<<<(unsigned)blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        w_fine, nxf, nyf, nzf, ndim, ns, weno_eps, tau, n_samples, seed, x, phat, target, smooth, js);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ERR_CUDA;
}

}  // extern "C"
