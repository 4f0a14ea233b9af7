// Learned WENO weights on the fifth-generation tensor cores (tcgen05): the
// forward pass and the training gradient of the 5 -> 32 -> 32 -> 3 network
// (include/mfc.h: mfc_mlp_forward_tc, mfc_mlp_grad).  The paper has no learned
// part; the network replaces the WENO5-JS nonlinear weights of Sec. 3.2.
//
// One CTA of four warps (one warpgroup) works on tiles of 128 samples, one
// sample per thread.  Every matrix product is one tcgen05.mma chain issued by
// thread 0 (M = 128 samples, BF16 operands in shared memory, FP32 accumulators
// in tensor memory), completed through an mbarrier; the threads read their row
// of the accumulator with tcgen05.ld, apply bias, ReLU or the loss derivative
// in FP32 and write the next operand (BF16) back to shared memory:
//
//   forward   H1 = X W1^T (K 16: 5 inputs padded), H2 = H1 W2^T (K 32),
//             Z  = H2 W3^T (N 16: 3 outputs padded)
//   backward  dH2 = dZ W3 (K 16), dH1 = dZ2 W2 (K 32), with dZ2 = dH2 * (H2 > 0)
//             and dZ1 = dH1 * (H1 > 0)
//   weights   one chain over the batch (K = 128, eight steps) of
//             [dZ2^T; dZ1^T; dZ3^T] [H1^T; H2^T; X^T]^T, whose diagonal blocks
//             are dW2, dW1 and dW3; it accumulates in tensor memory over all
//             tiles of the CTA and is read out once.
//
// Bias gradients and the loss are FP32 sums in registers.  Every wait on the
// mbarrier is bounded; a wait that gives up sets an error flag (read by
// mfc_mlp_tc_status), the CTA waits once more for its MMAs, frees its tensor
// memory and returns.
#include <cuda_bf16.h>
#include <cstdint>

#include "../../include/mfc.h"
#include "mfc_mlp.cuh"
#include "mfc_tc.cuh"

using namespace mfc;

namespace {

constexpr int kTile = 128;                  // samples per tile (MMA M)
constexpr int kTcStride = kMlpParams + 1;   // partial gradient + loss per CTA
constexpr uint32_t kMaxPolls = 1u << 22;    // ~0.2-0.5 s of polling per wait

static __device__ unsigned int g_tc_error;  // set when a bounded wait gave up

__device__ __constant__ float kIdealTc[3] = {0.1f, 0.6f, 0.3f};

// Shared-memory operand tiles (bytes; each a multiple of 128).
constexpr int kW1B = 32 * 16 * 2;    // B: W1 [n 32][k 16]
constexpr int kW2B = 32 * 32 * 2;    // B: W2 [n 32][k 32]
constexpr int kW3B = 16 * 32 * 2;    // B: W3 [n 16][k 32] (rows >= 3 zero)
constexpr int kXA = kTile * 16 * 2;  // A: X [128][16] (columns >= 5 zero)
constexpr int kHA = kTile * 32 * 2;  // A: H1, H2 [128][32]
constexpr int kW3tB = 32 * 16 * 2;   // B: W3^T [n 32][k 16] (k >= 3 zero)
constexpr int kW2tB = 32 * 32 * 2;   // B: W2^T [n 32][k 32]
constexpr int kDZ3A = kTile * 16 * 2;
constexpr int kAW = 128 * kTile * 2;  // A: [dZ2^T; dZ1^T; dZ3^T; 0] [128][batch 128]
constexpr int kBWN = 80;
constexpr int kBW = kBWN * kTile * 2;  // B: [H1^T; H2^T; X^T; 0] [80][batch 128]

struct FwdLayout {
    static constexpr int w1 = 0, w2 = w1 + kW1B, w3 = w2 + kW2B, x = w3 + kW3B, h1 = x + kXA, h2 = h1 + kHA;
    static constexpr int end = h2 + kHA;
};
struct GradLayout {
    static constexpr int w1 = 0, w2 = w1 + kW1B, w3 = w2 + kW2B, x = w3 + kW3B, h1 = x + kXA, h2 = h1 + kHA;
    static constexpr int w3t = h2 + kHA, w2t = w3t + kW3tB, dz3 = w2t + kW2tB, dz2 = dz3 + kDZ3A;
    static constexpr int aw = dz2 + kHA, bw = aw + kAW;
    static constexpr int end = bw + kBW;
};
// The forward kernel pads its shared memory so that at most four CTAs share an
// SM (4 x 128 tensor-memory columns); the gradient kernel's 91 KB allows two
// (2 x 256 columns).
constexpr int kFwdSmem = 57344;
constexpr int kGradSmem = GradLayout::end;
static_assert(FwdLayout::end <= kFwdSmem, "forward tiles");
static_assert(kGradSmem * 3 > 232448 && kGradSmem <= 232448, "two gradient CTAs per SM");

struct Ctrl {
    uint64_t mbar;
    uint32_t tmem;
    float red[4][68];   // cross-warp sums: b1 (32), b2 (32), b3 (3), loss
};

__device__ __forceinline__ uint16_t bf16_bits(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__device__ __forceinline__ void put_bf16(unsigned char* tile, int K, int row, int k, float v) {
    *reinterpret_cast<uint16_t*>(tile + tc::kmajor_offset(row, k, K)) = bf16_bits(v);
}

// Eight values of one row (columns 8 j .. 8 j + 7) as one 16-byte store.
__device__ __forceinline__ void put_row8(unsigned char* tile, int K, int row, int j, const float* v) {
    uint4 u;
    u.x = (uint32_t)bf16_bits(v[0]) | ((uint32_t)bf16_bits(v[1]) << 16);
    u.y = (uint32_t)bf16_bits(v[2]) | ((uint32_t)bf16_bits(v[3]) << 16);
    u.z = (uint32_t)bf16_bits(v[4]) | ((uint32_t)bf16_bits(v[5]) << 16);
    u.w = (uint32_t)bf16_bits(v[6]) | ((uint32_t)bf16_bits(v[7]) << 16);
    *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(row, 8 * j, K)) = u;
}

// Zero the dynamic shared memory and load the weight operands (BF16).
__device__ void load_weights(unsigned char* sm, int bytes, const float* __restrict__ P, bool transposed) {
    for (int i = threadIdx.x * 16; i < bytes; i += blockDim.x * 16)
        *reinterpret_cast<uint4*>(sm + i) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int i = threadIdx.x; i < kMlpH * kMlpH; i += blockDim.x) {
        const int n = i / kMlpH, k = i % kMlpH;
        put_bf16(sm + FwdLayout::w2, 32, n, k, P[kOffW2 + n * kMlpH + k]);
        if (transposed) put_bf16(sm + GradLayout::w2t, 32, n, k, P[kOffW2 + k * kMlpH + n]);
        if (k < kMlpIn) put_bf16(sm + FwdLayout::w1, 16, n, k, P[kOffW1 + n * kMlpIn + k]);
        if (n < kMlpOut) put_bf16(sm + FwdLayout::w3, 32, n, k, P[kOffW3 + n * kMlpH + k]);
        if (transposed && k < kMlpOut) put_bf16(sm + GradLayout::w3t, 16, n, k, P[kOffW3 + k * kMlpH + n]);
    }
}

// Thread 0 issues the MMAs of `issue`, commits them to the mbarrier; every
// thread waits for completion.  Returns false (all threads) if the wait gave up.
template <typename F>
__device__ __forceinline__ bool run_mma(Ctrl& c, uint32_t& phase, F&& issue) {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        issue();
        tc::mma_commit(&c.mbar);
    }
    const bool ok = tc::mbar_wait(&c.mbar, phase, kMaxPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    return !__syncthreads_or(!ok);
}

// After a wait gave up: flag it, give the MMAs in flight one more bounded wait.
__device__ void give_up(Ctrl& c, uint32_t phase) {
    if (threadIdx.x == 0) atomicExch(&g_tc_error, 1u);
    tc::mbar_wait(&c.mbar, phase ^ 1u, kMaxPolls);
}

// Forward of one tile: on return h1/h2 hold this thread's activations (FP32,
// after ReLU) and z its three logits; the BF16 operands are in shared memory.
__device__ __forceinline__ bool tile_forward(unsigned char* sm, Ctrl& c, uint32_t& phase, uint32_t tm, int warp,
                                             int row, const float* __restrict__ P, const float (&xin)[5],
                                             float (&h1)[32], float (&h2)[32], float (&z)[3], bool grad) {
    {
        const float v[8] = {xin[0], xin[1], xin[2], xin[3], xin[4], 0.f, 0.f, 0.f};
        put_row8(sm + FwdLayout::x, 16, row, 0, v);
        if (grad)
            for (int k = 0; k < kMlpIn; ++k) put_bf16(sm + GradLayout::bw, kTile, 64 + k, row, xin[k]);
    }
    if (!run_mma(c, phase, [&] {
            tc::mma_bf16(tm + 0, tc::desc_kmajor(sm + FwdLayout::x, 16, 0), tc::desc_kmajor(sm + FwdLayout::w1, 16, 0),
                         tc::idesc_bf16(kTile, 32), 0u);
        }))
        return false;
    float acc[32];
    tc::tmem_load_row<32>(tm, warp, 0, acc);
#pragma unroll
    for (int j = 0; j < 32; ++j) h1[j] = fmaxf(acc[j] + P[kOffB1 + j], 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) put_row8(sm + FwdLayout::h1, 32, row, j, h1 + 8 * j);
    if (grad)
        for (int k = 0; k < kMlpH; ++k) put_bf16(sm + GradLayout::bw, kTile, k, row, h1[k]);
    if (!run_mma(c, phase, [&] {
            for (int s = 0; s < 2; ++s)
                tc::mma_bf16(tm + 32, tc::desc_kmajor(sm + FwdLayout::h1, 32, s),
                             tc::desc_kmajor(sm + FwdLayout::w2, 32, s), tc::idesc_bf16(kTile, 32), (uint32_t)s);
        }))
        return false;
    tc::tmem_load_row<32>(tm, warp, 32, acc);
#pragma unroll
    for (int j = 0; j < 32; ++j) h2[j] = fmaxf(acc[j] + P[kOffB2 + j], 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) put_row8(sm + FwdLayout::h2, 32, row, j, h2 + 8 * j);
    if (grad)
        for (int k = 0; k < kMlpH; ++k) put_bf16(sm + GradLayout::bw, kTile, 32 + k, row, h2[k]);
    if (!run_mma(c, phase, [&] {
            for (int s = 0; s < 2; ++s)
                tc::mma_bf16(tm + 64, tc::desc_kmajor(sm + FwdLayout::h2, 32, s),
                             tc::desc_kmajor(sm + FwdLayout::w3, 32, s), tc::idesc_bf16(kTile, 16), (uint32_t)s);
        }))
        return false;
    float lz[8];
    {
        float tmp[8];
        tc::tmem_load_row<8>(tm, warp, 64, tmp);
#pragma unroll
        for (int e = 0; e < 8; ++e) lz[e] = tmp[e];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) z[q] = lz[q] + P[kOffB3 + q];
    return true;
}

__device__ __forceinline__ void softmax3(const float (&z)[3], float (&om)[3]) {
    const float m = fmaxf(z[0], fmaxf(z[1], z[2]));
    const float e0 = __expf(z[0] - m), e1 = __expf(z[1] - m), e2 = __expf(z[2] - m);
    const float inv = __fdividef(1.f, e0 + e1 + e2);
    om[0] = e0 * inv;
    om[1] = e1 * inv;
    om[2] = e2 * inv;
}

__global__ void __launch_bounds__(kTile) mlp_forward_tc_kernel(const float* __restrict__ P,
                                                               const float* __restrict__ x, long long B,
                                                               float* __restrict__ omega) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ Ctrl c;
    const int warp = threadIdx.x >> 5, row = threadIdx.x;
    load_weights(sm, FwdLayout::end, P, false);
    if (threadIdx.x == 0) tc::mbar_init(&c.mbar, 1);
    if (warp == 0) tc::tmem_alloc(&c.tmem, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = c.tmem;
    uint32_t phase = 0;
    for (long long t0 = (long long)blockIdx.x * kTile; t0 < B; t0 += (long long)gridDim.x * kTile) {
        const long long r = t0 + row;
        float xin[5];
        for (int k = 0; k < 5; ++k) xin[k] = r < B ? x[r * kMlpIn + k] : 0.f;
        float h1[32], h2[32], z[3];
        if (!tile_forward(sm, c, phase, tm, warp, row, P, xin, h1, h2, z, false)) {
            give_up(c, phase);
            break;
        }
        if (r < B) {
            float om[3];
            softmax3(z, om);
            for (int q = 0; q < 3; ++q) omega[r * 3 + q] = om[q];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 128);
}

__global__ void __launch_bounds__(kTile) mlp_grad_tc_kernel(const float* __restrict__ P, const float* __restrict__ x,
                                                            const float* __restrict__ phat,
                                                            const float* __restrict__ target,
                                                            const float* __restrict__ mask, long long B, float lam,
                                                            float* __restrict__ work) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ Ctrl c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, row = threadIdx.x;
    load_weights(sm, GradLayout::end, P, true);
    if (threadIdx.x == 0) tc::mbar_init(&c.mbar, 1);
    if (warp == 0) tc::tmem_alloc(&c.tmem, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // columns: H1 0, H2 32, Z 64, dH2 80, dH1 112, weight gradients 144 (80 wide)
    const uint32_t tm = c.tmem;
    uint32_t phase = 0;
    const float invB = 1.0f / (float)B;
    float gb1[32], gb2[32], gb3[3] = {0.f, 0.f, 0.f}, lsum = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) gb1[j] = gb2[j] = 0.f;
    bool ok = true;
    uint32_t acc_w = 0;
    for (long long t0 = (long long)blockIdx.x * kTile; t0 < B && ok; t0 += (long long)gridDim.x * kTile) {
        const long long r = t0 + row;
        const bool live = r < B;
        float xin[5];
        for (int k = 0; k < 5; ++k) xin[k] = live ? x[r * kMlpIn + k] : 0.f;
        float h1[32], h2[32], z[3];
        if (!(ok = tile_forward(sm, c, phase, tm, warp, row, P, xin, h1, h2, z, true))) break;
        // loss and dL/dz (zero for rows past the batch)
        float dz[3] = {0.f, 0.f, 0.f};
        if (live) {
            float om[3];
            softmax3(z, om);
            const float pp[3] = {phat[r * 3], phat[r * 3 + 1], phat[r * 3 + 2]};
            const float tt = target[r], mk = mask[r];
            const float e = om[0] * pp[0] + om[1] * pp[1] + om[2] * pp[2] - tt;
            float dom[3], reg = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float dd = om[q] - kIdealTc[q];
                reg += dd * dd;
                dom[q] = 2.f * invB * (e * pp[q] + lam * mk * dd);
            }
            lsum += invB * (e * e + lam * mk * reg);
            const float sdot = om[0] * dom[0] + om[1] * dom[1] + om[2] * dom[2];
#pragma unroll
            for (int q = 0; q < 3; ++q) dz[q] = om[q] * (dom[q] - sdot);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) gb3[q] += dz[q];
        {
            const float v[8] = {dz[0], dz[1], dz[2], 0.f, 0.f, 0.f, 0.f, 0.f};
            put_row8(sm + GradLayout::dz3, 16, row, 0, v);
            for (int q = 0; q < 3; ++q) put_bf16(sm + GradLayout::aw, kTile, 64 + q, row, dz[q]);
        }
        // dH2 = dZ W3, dZ2 = dH2 * (H2 > 0)
        if (!(ok = run_mma(c, phase, [&] {
                  tc::mma_bf16(tm + 80, tc::desc_kmajor(sm + GradLayout::dz3, 16, 0),
                               tc::desc_kmajor(sm + GradLayout::w3t, 16, 0), tc::idesc_bf16(kTile, 32), 0u);
              })))
            break;
        float d[32];
        tc::tmem_load_row<32>(tm, warp, 80, d);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            d[j] = h2[j] > 0.f ? d[j] : 0.f;
            gb2[j] += d[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) put_row8(sm + GradLayout::dz2, 32, row, j, d + 8 * j);
        for (int k = 0; k < kMlpH; ++k) put_bf16(sm + GradLayout::aw, kTile, k, row, d[k]);
        // dH1 = dZ2 W2, dZ1 = dH1 * (H1 > 0)
        if (!(ok = run_mma(c, phase, [&] {
                  for (int s = 0; s < 2; ++s)
                      tc::mma_bf16(tm + 112, tc::desc_kmajor(sm + GradLayout::dz2, 32, s),
                                   tc::desc_kmajor(sm + GradLayout::w2t, 32, s), tc::idesc_bf16(kTile, 32),
                                   (uint32_t)s);
              })))
            break;
        tc::tmem_load_row<32>(tm, warp, 112, d);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            d[j] = h1[j] > 0.f ? d[j] : 0.f;
            gb1[j] += d[j];
        }
        for (int k = 0; k < kMlpH; ++k) put_bf16(sm + GradLayout::aw, kTile, 32 + k, row, d[k]);
        // weight gradients: accumulate over the batch (eight K steps of 16 samples)
        if (!(ok = run_mma(c, phase, [&] {
                  for (int s = 0; s < kTile / 16; ++s)
                      tc::mma_bf16(tm + 144, tc::desc_kmajor(sm + GradLayout::aw, kTile, s),
                                   tc::desc_kmajor(sm + GradLayout::bw, kTile, s), tc::idesc_bf16(kTile, kBWN),
                                   acc_w | (uint32_t)s);
              })))
            break;
        acc_w = 1u;
    }
    if (!ok) {
        give_up(c, phase);
    } else {
        float* out = work + (long long)blockIdx.x * kTcStride;
        // weight gradients: warp 0 rows dW2, warp 1 rows dW1, warp 2 lanes 0..2 rows dW3
        if (acc_w && warp < 3) {
            float dw[32];
            tc::tmem_load_row<32>(tm, warp, 144 + (warp == 0 ? 0 : warp == 1 ? 64 : 32), dw);
            if (warp == 0) {
                for (int k = 0; k < kMlpH; ++k) out[kOffW2 + lane * kMlpH + k] = dw[k];
            } else if (warp == 1) {
                for (int k = 0; k < kMlpIn; ++k) out[kOffW1 + lane * kMlpIn + k] = dw[k];
            } else if (lane < kMlpOut) {
                for (int k = 0; k < kMlpH; ++k) out[kOffW3 + lane * kMlpH + k] = dw[k];
            }
        } else if (!acc_w) {   // no tile: zero partial
            for (int i = threadIdx.x; i < kOffB3; i += blockDim.x)
                if (!(i >= kOffB1 && i < kOffW2) && !(i >= kOffB2 && i < kOffW3)) out[i] = 0.f;
        }
        // bias gradients and loss: warp sums, then across the four warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                gb1[j] += __shfl_xor_sync(0xffffffffu, gb1[j], o);
                gb2[j] += __shfl_xor_sync(0xffffffffu, gb2[j], o);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) gb3[q] += __shfl_xor_sync(0xffffffffu, gb3[q], o);
            lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        }
        if (lane == 0) {
            for (int j = 0; j < 32; ++j) {
                c.red[warp][j] = gb1[j];
                c.red[warp][32 + j] = gb2[j];
            }
            for (int q = 0; q < 3; ++q) c.red[warp][64 + q] = gb3[q];
            c.red[warp][67] = lsum;
        }
        __syncthreads();
        if (threadIdx.x < 68) {
            const int i = threadIdx.x;
            const float s = c.red[0][i] + c.red[1][i] + c.red[2][i] + c.red[3][i];
            const int dst = i < 32 ? kOffB1 + i : i < 64 ? kOffB2 + (i - 32) : i < 67 ? kOffB3 + (i - 64) : kMlpParams;
            out[dst] = s;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 256);
}

// Deterministic sum of the per-CTA partials, one thread per slot.
__global__ void mlp_tc_reduce_kernel(const float* __restrict__ work, int parts, float* __restrict__ grad,
                                     float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    float s = 0.f;
    for (int w = 0; w < parts; ++w) s += work[(long long)w * kTcStride + p];
    if (p < kMlpParams) grad[p] = s;
    else if (loss) *loss = s;
}

unsigned grid_for(long long B, int per_sm) {
    long long tiles = (B + kTile - 1) / kTile;
    const long long cap = 152LL * per_sm;
    return (unsigned)(tiles < cap ? tiles : cap);
}

}  // namespace

extern "C" {

mfc_status mfc_mlp_forward_tc(const float* params, const float* x, long long batch, float* omega, void* stream) {
    if (!params || !x || !omega || batch <= 0) return MFC_ERR_ARG;
    if (cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem) !=
        cudaSuccess)
        return MFC_ERR_CUDA;
    mlp_forward_tc_kernel<<<grid_for(batch, 4), kTile, kFwdSmem, static_cast<cudaStream_t>(stream)>>>(params, x,
                                                                                                     batch, omega);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ERR_CUDA;
}

mfc_status mfc_mlp_grad(const float* params, const float* x, const float* phat, const float* target,
                        const float* mask, long long batch, float lam, float* grad, float* loss, float* work,
                        void* stream) {
    if (!params || !x || !phat || !target || !mask || !grad || !work || batch <= 0 || !(lam >= 0.f))
        return MFC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaFuncSetAttribute(mlp_grad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGradSmem) !=
        cudaSuccess)
        return MFC_ERR_CUDA;
    const unsigned blocks = grid_for(batch, 2);
    static_assert(2LL * 152 * kTcStride <= MFC_MLP_WORK_FLOATS, "workspace holds every CTA's partial");
    mlp_grad_tc_kernel<<<blocks, kTile, kGradSmem, s>>>(params, x, phat, target, mask, batch, lam, work);
    if (cudaGetLastError() != cudaSuccess) return MFC_ERR_CUDA;
    mlp_tc_reduce_kernel<<<(kTcStride + 127) / 128, 128, 0, s>>>(work, (int)blocks, grad, loss);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ERR_CUDA;
}

int mfc_mlp_tc_status(void) {
    unsigned int flag = 0, zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(&flag, g_tc_error, sizeof flag) != cudaSuccess) return -1;
    if (flag && cudaMemcpyToSymbol(g_tc_error, &zero, sizeof zero) != cudaSuccess) return -1;
    return flag ? 1 : 0;
}

}  // extern "C"
