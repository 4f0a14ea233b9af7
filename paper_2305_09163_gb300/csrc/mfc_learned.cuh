// The learned form: WENO5-JS weights replaced by a small network evaluated on
// the tensor cores for the edges the sensor lets through, and its face flux.
#pragma once
#include "mfc_riemann.cuh"

namespace mfc {

// ---------------------------------------------------------------------------
// Learned form (the paper has no learned part; the network replaces the
// WENO5-JS nonlinear weights of Sec. 3.2).  Per cell and variable the FP32
// WENO5 pieces are formed as in the mixed path.  WENO5-JS weights are kept
// where the discontinuity sensor trips (max_r b_r > tau (min_r b_r + 1e-6 s^2),
// b the smoothness indicators without their 4/3 factor), where the stencil is
// flat to FP32 resolution (s <= 1e-7 |v_c|), and where the learned edge value
// would leave the range of cells c-1, c, c+1.  Only the stencils whose learned
// value can be used go to the network: per variable the warp packs them
// (ballot and prefix count) into shared memory as BF16 rows of the five
// normalised differences, one row per edge, evaluates the network on the
// tensor cores 16 rows per tile, and each lane turns its rows' logits into
// weights and edge values while its stencil is still in registers.  A warp
// whose 32 stencils of a variable all keep the JS weights skips the network.
// All 32 lanes must call these functions.
// ---------------------------------------------------------------------------
#ifndef MFC_LEARN_TILES
#define MFC_LEARN_TILES 1
#endif
constexpr int kLearnTiles = MFC_LEARN_TILES;

struct LearnRows {
    // one row per network evaluation (both edges of up to 32 cells of one
    // variable): BF16 inputs in columns 0..4, then overwritten by the logits
    uint4 row[64];
};

// Network over rows 0..nrows-1 of sm; each row's inputs are replaced by its
// three logits (FP32, words 0..2).
__device__ __forceinline__ void learned_logits(const uint4* __restrict__ frag, LearnRows& sm, int nrows, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const int nt = (nrows + 15) >> 4;
    const uint32_t* rw = reinterpret_cast<const uint32_t*>(sm.row);
    float* rf = reinterpret_cast<float*>(sm.row);
    __syncwarp();
    if (nt == 0) return;
    MlpWeights W;
    mlp_weights_from_frag(frag, W, lane);
    // kLearnTiles independent tiles at a time so their tensor-core chains overlap
#pragma unroll 1
    for (int t0 = 0; t0 < nt; t0 += kLearnTiles) {
        float z[kLearnTiles][4];
#pragma unroll
        for (int u = 0; u < kLearnTiles; ++u) {
            if (t0 + u < nt) {
                const int r0 = 16 * (t0 + u);
                const uint32_t a_in[2] = {rw[4 * (r0 + g) + t], rw[4 * (r0 + g + 8) + t]};
                mlp_tile_logits(W, a_in, z[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kLearnTiles; ++u) {
            if (t0 + u < nt && t < 2) {
                const int r0 = 16 * (t0 + u);
                *reinterpret_cast<float2*>(rf + 4 * (r0 + g) + 2 * t) = make_float2(z[u][0], z[u][1]);
                *reinterpret_cast<float2*>(rf + 4 * (r0 + g + 8) + 2 * t) = make_float2(z[u][2], z[u][3]);
            }
        }
    }
    __syncwarp();
}

// Increment sum_r omega_r d_r with omega the softmax of the logits in words
// 0..2 of a row.
__device__ __forceinline__ float learned_increment(const uint4& row, float d0, float d1, float d2) {
    const float z0 = __uint_as_float(row.x), z1 = __uint_as_float(row.y), z2 = __uint_as_float(row.z);
    const float m = fmaxf(z0, fmaxf(z1, z2));
    const float e0 = __expf(z0 - m), e1 = __expf(z1 - m), e2 = __expf(z2 - m);
    return __fdividef(fmaf(e0, d0, fmaf(e1, d1, e2 * d2)), e0 + e1 + e2);
}

// Edge values of one variable of one cell: WENO5-JS (eRjs, eLjs) and the
// learned form (eR, eL; equal to the JS values where the sensor trips).  vc is
// the cell value and d the four differences across cells c-2..c+2.  Returns
// the number of network rows (edges) the warp evaluated (warp-uniform).
__device__ __forceinline__ int learned_var_edges(float vc, const float (&d)[4], float eps34, float tau, bool bound,
                                                 const uint4* __restrict__ frag, LearnRows& sm, int lane,
                                                 float& eRjs, float& eLjs, float& eR, float& eL) {
    float b0, b1, b2;   // the JS smoothness indicators, reused by the sensor
    weno5_edges(vc, d, eps34, eRjs, eLjs, b0, b1, b2);
    eR = eRjs;
    eL = eLjs;
    const float xm2 = -(d[0] + d[1]), xm1 = -d[1], xp1 = d[2], xp2 = d[2] + d[3];
    const float sc = fmaxf(fmaxf(fabsf(xm2), fabsf(xm1)), fmaxf(fabsf(xp1), fabsf(xp2)));
    const float bmax = fmaxf(b0, fmaxf(b1, b2)), bmin = fminf(b0, fminf(b1, b2));
    const bool usejs = !(sc > 1e-7f * fabsf(vc)) || (bmax > tau * fmaf(1e-6f * sc, sc, bmin));
    const unsigned need = __ballot_sync(0xffffffffu, !usejs);
    if (need == 0u) return 0;
    const int nrows = 2 * __popc(need);
    const int r = 2 * __popc(need & ((1u << lane) - 1u));
    __syncwarp();   // the previous evaluation's logits are read before rows are rewritten
    if (!usejs) {
        const float is = __fdividef(1.0f, sc + 1e-30f);
        // edge at c+1/2: stencil c-2..c+2; edge at c-1/2: the mirrored stencil
        sm.row[r] = make_uint4(pack_bf16(xm2 * is, xm1 * is), pack_bf16(0.f, xp1 * is), pack_bf16(xp2 * is, 0.f), 0u);
        sm.row[r + 1] =
            make_uint4(pack_bf16(xp2 * is, xp1 * is), pack_bf16(0.f, xm1 * is), pack_bf16(xm2 * is, 0.f), 0u);
    }
    learned_logits(frag, sm, nrows, lane);
    if (!usejs) {
        // increments at c+1/2 of the stencils c-2..c, c-1..c+1, c..c+2
        const float p0 = fmaf(5.f / 6.f, d[1], (-1.f / 3.f) * d[0]);
        const float p1 = fmaf(1.f / 6.f, d[1], (1.f / 3.f) * d[2]);
        const float p2 = fmaf(2.f / 3.f, d[2], (-1.f / 6.f) * d[3]);
        // increments at c-1/2 of the stencils c..c+2, c-1..c+1, c-2..c
        const float m0 = fmaf(-5.f / 6.f, d[2], (1.f / 3.f) * d[3]);
        const float m1 = fmaf(-1.f / 6.f, d[2], (-1.f / 3.f) * d[1]);
        const float m2 = fmaf(-2.f / 3.f, d[1], (1.f / 6.f) * d[0]);
        const float il = learned_increment(sm.row[r], p0, p1, p2);
        const float ir = learned_increment(sm.row[r + 1], m0, m1, m2);
        // accept a learned value only inside the range of cells c-1, c, c+1
        const float lo = fminf(0.f, fminf(-d[1], d[2])), hi = fmaxf(0.f, fmaxf(-d[1], d[2]));
        if (!(bound && (il < lo || il > hi))) eL = vc + il;
        if (!(bound && (ir < lo || ir > hi))) eR = vc + ir;
    }
    return nrows;
}

// The same for all NS variables of a cell, unrolled over the variables (the
// pencil-marching sweep, which keeps its stencils in registers): stencil(v, d)
// returns the cell value of variable v and fills d with its four differences.
template <int NS, typename Stencil>
__device__ __forceinline__ int learned_cell_edges(const Stencil& stencil, float eps34, float tau, bool bound,
                                                   const uint4* __restrict__ frag, LearnRows& sm, int lane,
                                                   float (&eRjs)[NS], float (&eLjs)[NS], float (&eR)[NS],
                                                   float (&eL)[NS]) {
    int nrows = 0;
#pragma unroll
    for (int v = 0; v < NS; ++v) {
        float d[4];
        const float vc = stencil(v, d);
        nrows += learned_var_edges(vc, d, eps34, tau, bound, frag, sm, lane, eRjs[v], eLjs[v], eR[v], eL[v]);
    }
    return nrows;
}

// Face flux of the learned form: the learned face states, else (non-physical)
// the WENO5-JS states, else the first-order cell values.  loadJ(Lj, Rj) fills
// the JS states; it is called only where the learned ones fail, so that they
// need not be held beside them.
template <int NF, int NDIM, int DIR, typename LoadJ>
__device__ __forceinline__ void face_flux_learned(const SweepArgs& a, const EosR<float>& e, const float* Ll,
                                                  const float* Rl, const LoadJ& loadJ, const float* cl,
                                                  const float* cr, float* F, float& ut) {
    constexpr int NS = Layout<NF, NDIM>::NS;
    float fl[NS], fr[NS];
#pragma unroll
    for (int v = 0; v < NS; ++v) {
        fl[v] = Ll[v];
        fr[v] = Rl[v];
    }
    Mix<float> mL = mixture<float, NF, NDIM>(fl, e);
    Mix<float> mR = mixture<float, NF, NDIM>(fr, e);
    if (a.fallback) {
        if (!(face_state_ok<float, NF, NDIM>(fl, mL) && face_state_ok<float, NF, NDIM>(fr, mR))) {
            loadJ(fl, fr);
            mL = mixture<float, NF, NDIM>(fl, e);
            mR = mixture<float, NF, NDIM>(fr, e);
            if (!(face_state_ok<float, NF, NDIM>(fl, mL) && face_state_ok<float, NF, NDIM>(fr, mR))) {
#pragma unroll
                for (int v = 0; v < NS; ++v) {
                    fl[v] = cl[v];
                    fr[v] = cr[v];
                }
                mL = mixture<float, NF, NDIM>(fl, e);
                mR = mixture<float, NF, NDIM>(fr, e);
                count_fallback(a.fallback_count);
            }
        }
    }
    hllc<float, NF, NDIM, DIR>(fl, fr, mL, mR, F, ut);
}

}  // namespace mfc
