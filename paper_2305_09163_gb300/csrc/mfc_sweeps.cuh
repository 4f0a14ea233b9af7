// The directional sweeps: pencil-marching y/z kernel, x stream kernel, y/z
// stream kernels, and their bounded entries.
#pragma once
#include "mfc_cell.cuh"

namespace mfc {

// ---------------------------------------------------------------------------
// Directional sweep for y and z.  One thread marches along one pencil segment
// of `seg` cells in direction DIR: it reconstructs the edges of cells
// s0-1..s1, forms faces s0-1/2..s1-1/2 and finishes cells s0..s1-1.  A warp
// covers 32 consecutive x of one segment (lanes past the end of a row work on
// a clamped copy and store nothing), so loads and stores are coalesced and all
// lanes of a warp run the same number of iterations, which the tensor-core
// network of the learned form (LEARNED) requires.
// ---------------------------------------------------------------------------
template <typename Real, int NF, int NDIM, int DIR, bool LEARNED = false, int ORDER = 5>
__global__ void __launch_bounds__(128) sweep_kernel(const SweepArgs a) {
    static_assert(!LEARNED || sizeof(Real) == 4, "the learned form runs in FP32");
    static_assert(!LEARNED || ORDER == 5, "the learned form replaces the WENO5 weights");
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM;
    constexpr int T1 = (DIR == 0) ? 1 : 0;
    constexpr int T2 = (DIR == 2) ? 1 : 2;
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n1 = a.g.n[T1], n2 = a.g.n[T2], nd = a.g.n[DIR];
    const int nxc = (n1 + 31) >> 5;
    if (wid >= (long long)nxc * a.nseg * n2) return;  // whole warps only
    const int xc = (int)(wid % nxc);
    const long long rest = wid / nxc;
    const int sg = (int)(rest % a.nseg);
    const int t2 = (int)(rest / a.nseg);
    const bool active = xc * 32 + lane < n1;
    if (!LEARNED && !active) return;
    const int t1 = active ? xc * 32 + lane : n1 - 1;
    const long long sd = stride_of(a.g, DIR);
    const long long base = (long long)t1 * stride_of(a.g, T1) + (long long)t2 * stride_of(a.g, T2);
    const long long nc = a.g.ncell;
    const int s0 = sg * a.seg;
    const int s1 = min(s0 + a.seg, nd);
    const int bclo = a.g.bc_lo[DIR], bchi = a.g.bc_hi[DIR];
    const Real eps34 = sweep_epsw<Real, ORDER>(a);  // 3/4 eps (WENO5) or eps (WENO3)
    const EosR<Real> e = sweep_eos<Real>(a);
    const Real inv_dx = sweep_inv_dx<Real>(a, DIR);
    LearnRows* lsm = nullptr;
    if constexpr (LEARNED) {
        __shared__ LearnRows lbuf[4];
        lsm = &lbuf[threadIdx.x >> 5];
    }
    unsigned long long net_rows = 0;  // learned form: network rows of this warp
    RateAcc racc;                     // fused RK epilogue: CFL rate of the finished cells

    auto load = [&](int i, Real* out) {
        bool flip = false;
        const int m = ghost_map(i, nd, bclo, bchi, &flip);
        const long long idx = base + (long long)m * sd;
#pragma unroll
        for (int v = 0; v < NS; ++v) out[v] = __ldg(w + v * nc + idx);
        if (flip) out[IM + DIR] = -out[IM + DIR];
    };

    // Window around the cell c being reconstructed: vc = c, vp1 = c+1,
    // vp2 = c+2, the four differences across c-2..c+2, and cm1 = c-1.
    Real vc[NS], vp1[NS], vp2[NS], D[NS][4], cm1[NS];
    {
        Real t[NS];
        load(s0 - 3, t);
        load(s0 - 2, cm1);
        load(s0 - 1, vc);
        load(s0, vp1);
        load(s0 + 1, vp2);
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            D[v][0] = cm1[v] - t[v];
            D[v][1] = vc[v] - cm1[v];
            D[v][2] = vp1[v] - vc[v];
            D[v][3] = vp2[v] - vp1[v];
        }
    }
    Real eLprev[NS], eLprevJ[NS], Fprev[NS], utprev = 0;
#pragma unroll
    for (int v = 0; v < NS; ++v) { eLprev[v] = 0; eLprevJ[v] = 0; Fprev[v] = 0; }

    for (int c = s0 - 1; c <= s1; ++c) {
        Real eR[NS], eL[NS], eRJ[NS], eLJ[NS];
        if constexpr (LEARNED) {
            auto stencil = [&](int v, float (&dd)[4]) -> float {
                dd[0] = D[v][0];
                dd[1] = D[v][1];
                dd[2] = D[v][2];
                dd[3] = D[v][3];
                return vc[v];
            };
            net_rows += learned_cell_edges<NS>(stencil, eps34, a.tau, a.bound != 0, a.mlp_frag, *lsm, lane, eRJ, eLJ, eR,
                                                  eL);
        } else {
#pragma unroll
            for (int v = 0; v < NS; ++v) weno_edges<ORDER>(vc[v], D[v], eps34, eR[v], eL[v]);
        }
        if (c >= s0) {
            Real F[NS], ut;
            if constexpr (LEARNED)
                face_flux_learned<NF, NDIM, DIR>(
                    a, e, eLprev, eR,
                    [&](float* Lj, float* Rj) {
#pragma unroll
                        for (int v = 0; v < NS; ++v) {
                            Lj[v] = eLprevJ[v];
                            Rj[v] = eRJ[v];
                        }
                    },
                    cm1, vc, F, ut);
            else
                face_flux<Real, NF, NDIM, DIR>(a, e, eLprev, eR, cm1, vc, F, ut);
            if (c >= s0 + 1 && active)
                racc.add(finish_cell<Real, NF, NDIM, DIR>(a, base + (long long)(c - 1) * sd, Fprev, F, utprev, ut, cm1,
                                                          inv_dx, c - 1, sd));
#pragma unroll
            for (int v = 0; v < NS; ++v) Fprev[v] = F[v];
            utprev = ut;
        }
        // advance the window by one cell
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            eLprev[v] = eL[v];
            if constexpr (LEARNED) eLprevJ[v] = eLJ[v];
            cm1[v] = vc[v];
        }
        if (c < s1) {
            Real nw[NS];
            load(c + 3, nw);
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                D[v][0] = D[v][1];
                D[v][1] = D[v][2];
                D[v][2] = D[v][3];
                D[v][3] = nw[v] - vp2[v];
                vc[v] = vp1[v];
                vp1[v] = vp2[v];
                vp2[v] = nw[v];
            }
        }
    }
    if constexpr (LEARNED) {
        if ((threadIdx.x & 31) == 0 && net_rows && a.net_rows) atomicAdd(a.net_rows, net_rows);
    }
    publish_rate(a, racc);
}

// ---------------------------------------------------------------------------
// x sweep as a coalesced stream.  Every x-row of n cells is laid out as n+2
// "slots" for edge cells c = -1..n; the rows are concatenated and each CTA
// owns `slots_per_block` consecutive slots.  A chunk of 128 slots is one slot
// per lane: lane s reconstructs the edges of its cell c (five-cell stencil read
// straight from global memory, consecutive lanes = consecutive x), forms the
// face c-1/2 from its own right-side value and the left-side value of slot s-1
// (shared memory), and finishes cell c-1 from faces c-3/2 and c-1/2.  The
// left-side values and fluxes sit in rings indexed by slot, so the next chunk
// reads the last slot's ones where this chunk wrote them; each CTA starts two
// slots early so that its first cell has both faces.  Every lane takes part in
// every chunk, as the learned form's warp-level network needs.
// ---------------------------------------------------------------------------
// The FP64 path's edge values of variable q of cell c along direction dir in
// float-float (DFS): the increment pair of the reconstruction (WENO5 or WENO3
// on uniform grids, WENO5 from the cell's tables on stretched ones) added to
// the split cell value with the accurate float-float addition (the face state
// carries ~2^-48 of its magnitude).  In the six-equation model the volume
// fractions keep
// FP64 edges instead (vc + the widened increment, carried in the same 8 bytes
// by df_pack), since their complement alpha_N enters a flux (face_flux_df).
// VALUE_MAJOR: the grid-table layout of the direction (x sweep: true).
// ---------------------------------------------------------------------------
template <typename Real, int NF, int NDIM, int ORDER, bool NONUNIF, bool SIX, bool VALUE_MAJOR>
__device__ __forceinline__ void dfs_edges(const SweepArgs& a, int dir, int c, int q, double vc, const double (&D)[4],
                                          double eps34, df& eR, df& eL) {
    df2 I;
    if constexpr (NONUNIF) {
        const GridCol<VALUE_MAJOR> grow(a.grid[dir], a.grid_stride[dir], c);
        I = weno5_increments_nu_pair(D, sweep_epsw<double, 3>(a), grow);
    } else if constexpr (ORDER == 5) {
        const df d[4] = {df_from_double(D[0]), df_from_double(D[1]), df_from_double(D[2]), df_from_double(D[3])};
        I = weno5_increments_pair(d, eps34);
    } else {
        I = weno3_increments_pair(D[1], D[2], eps34);
    }
    if (SIX && q >= Layout<NF, NDIM>::IA && q < Layout<NF, NDIM>::IA + NF - 1) {
        eL = df_pack(vc + df_to_double(df2_x(I)));
        eR = df_pack(vc + df_to_double(df2_y(I)));
    } else {
        const df cc = df_from_double(vc);
        const df2 E = df2_add(df2_make(cc, cc), I);
        eL = df2_x(E);
        eR = df2_y(E);
    }
}

// ---------------------------------------------------------------------------
constexpr int kStreamThreads = 128;

template <typename Real, int NF, int NDIM, bool LEARNED = false, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__device__ __forceinline__ void sweep_x_stream_body(const SweepArgs& a) {
    static_assert(!SIX || !LEARNED, "six-equation model: FP64 and mixed forms");
    static_assert(!NONUNIF || (!LEARNED && ORDER == 5), "non-uniform grids: WENO5, FP64 and mixed forms");
    static_assert(!LEARNED || sizeof(Real) == 4, "the learned form runs in FP32");
    static_assert(!LEARNED || ORDER == 5, "the learned form replaces the WENO5 weights");
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM;
    constexpr int NQ = Layout<NF, NDIM, SIX>::NQ;   // flux rows
    constexpr int NJ = LEARNED ? NS : 1;
    // Edge values and face fluxes of slot s sit at position s mod ER of a ring
    // of ER = kStreamThreads + 1: a chunk writes its 128 slots and reads their
    // left neighbours, the first of which the previous chunk wrote; the next
    // chunk overwrites it (s + 128 = s - 1 mod ER) only after the barriers that
    // order it.
    constexpr int ER = kStreamThreads + 1;
    // ROLL (FP64): the reconstruction runs as one copy looped over the
    // variables, stencils loaded per variable, edges to shared memory.  Unrolled
    // over the variables the float-float code overflowed the instruction cache
    // (ncu: "no instruction" the largest stall, 1.0-1.5 warps per issue).
    constexpr bool ROLL = sizeof(Real) == 8 && !LEARNED;
    // DFS (FP64 WENO5 and WENO3, uniform and stretched grids, five- and
    // six-equation models): the edge values stay
    // float-float (cell value + increment, in the same 8 bytes) from the
    // reconstruction into the Riemann solver: no FP64 edge sums and mixtures
    // (256^3 step: WENO5 44.3 -> 39.0 ms, WENO3 33.4 -> 24.7 ms)
    constexpr bool DFS = ROLL;
    __shared__ Real sh_eL[NS][ER];
    __shared__ Real sh_eR[(ROLL || LEARNED) ? NS : 1][kStreamThreads];
    df(*dsh_eL)[ER] = reinterpret_cast<df(*)[ER]>(sh_eL);
    df(*dsh_eR)[kStreamThreads] = reinterpret_cast<df(*)[kStreamThreads]>(sh_eR);
    __shared__ Real sh_eLJ[NJ][ER];
    __shared__ Real sh_eRJ[NJ][kStreamThreads];
    __shared__ Real sh_F[NQ + 1][ER];
    df(*dsh_F)[ER] = reinterpret_cast<df(*)[ER]>(sh_F);   // DFS: float-float fluxes
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const int n = a.g.n[0];
    const long long rowlen = (long long)n + 2;
    const long long nrows = a.g.ncell / n;
    const long long total = rowlen * nrows;
    const long long own0 = (long long)blockIdx.x * a.slots_per_block;
    const long long own1 = min(own0 + a.slots_per_block, total);
    const long long nc = a.g.ncell;
    const int bclo = a.g.bc_lo[0], bchi = a.g.bc_hi[0];
    const Real eps34 = sweep_epsw<Real, ORDER>(a);  // 3/4 eps (WENO5) or eps (WENO3)
    const EosR<Real> e = sweep_eos<Real>(a);
    [[maybe_unused]] const EosDf edf(e);   // DFS: the EOS constants as float-float
    const Real inv_dx = sweep_inv_dx<Real>(a, 0);
    [[maybe_unused]] const df inv_df = df_from_double((double)inv_dx);
    const int t = threadIdx.x;
    LearnRows* lsm = nullptr;
    if constexpr (LEARNED) {
        __shared__ LearnRows lbuf[kStreamThreads / 32];
        lsm = &lbuf[t >> 5];
    }
    unsigned long long net_rows = 0;  // learned form: network rows of this warp
    RateAcc racc;                     // fused RK epilogue: CFL rate of the finished cells

    // (row, column) of this lane's slot: one 64-bit division when the slot first
    // becomes valid, then advanced by 128 slots per chunk with additions (a
    // 64-bit division per chunk would run on the FP64 pipe)
    long long srow = 0;
    int scol = 0;  // slot index within its row, 0..n+1
    bool placed = false;
    // ring position of this lane's slot (own0 - 2 + t) mod ER, then one step
    // back per chunk
    int pos = (int)(((own0 - 2 + t) % ER + ER) % ER);
    for (long long base = own0 - 2; base < own1; base += kStreamThreads) {
        const int pl = pos == 0 ? ER - 1 : pos - 1;   // left neighbour's position
        const long long s = base + t;
        if (s >= 0 && !placed) {
            srow = s / rowlen;
            scol = (int)(s - srow * rowlen);
            placed = true;
        }
        const bool live = (s >= 0) && (s < own1);
        const long long row = srow;
        const int c = live ? scol - 1 : -1;
        const long long rowoff = row * n;
        if (placed) {
            scol += kStreamThreads;
            while (scol >= rowlen) {
                scol -= (int)rowlen;
                ++srow;
            }
        }
        if constexpr (LEARNED) {
            // the learned sweep keeps 16 warps per SM: pull the next chunk's
            // cells into L1 while this chunk computes
            if (placed && base + kStreamThreads + t < own1 && srow < nrows) {
                const float* nx = w + srow * n + min(max(scol - 1, 0), n - 1);
#pragma unroll
                for (int q = 0; q < NS; ++q) asm volatile("prefetch.global.L1 [%0];" ::"l"(nx + q * nc));
            }
        }
        Real cell[NS], cm1[NS], eL[NS], eR[NS];
        if constexpr (LEARNED) {
            // one copy of the reconstruction looped over the variables (the
            // network's code once), the next variable's stencil loaded while
            // this one computes, edge values to shared memory
            int mk[5];
            bool fk[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                fk[k] = false;
                mk[k] = live ? ghost_map(c + k - 2, n, bclo, bchi, &fk[k]) : 0;
            }
            const Real* wr = w + rowoff;
            float vn[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) vn[k] = live ? __ldg(wr + mk[k]) : 0.f;
#pragma unroll 1
            for (int q = 0; q < NS; ++q) {
                float v[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) v[k] = (q == IM && fk[k]) ? -vn[k] : vn[k];
                if (q + 1 < NS) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) vn[k] = live ? __ldg(wr + (q + 1) * nc + mk[k]) : 0.f;
                }
                const float dq[4] = {v[1] - v[0], v[2] - v[1], v[3] - v[2], v[4] - v[3]};
                float ejR, ejL, elR, elL;
                net_rows += learned_var_edges(v[2], dq, eps34, a.tau, a.bound != 0, a.mlp_frag, *lsm, t & 31, ejR,
                                              ejL, elR, elL);
                if (live) {
                    sh_eL[q][pos] = elL;
                    sh_eLJ[q][pos] = ejL;
                    sh_eR[q][t] = elR;
                    sh_eRJ[q][t] = ejR;
                }
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                float x1 = live ? __ldg(wr + q * nc + mk[1]) : 0.f;
                float x2 = live ? __ldg(wr + q * nc + mk[2]) : 0.f;
                if (q == IM && fk[1]) x1 = -x1;
                if (q == IM && fk[2]) x2 = -x2;
                cm1[q] = x1;
                cell[q] = x2;
            }
        }
        Real vcv[NS], Dv[NS][4];
        if constexpr (!LEARNED) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                vcv[q] = 0;
                cm1[q] = 0;
                Dv[q][0] = Dv[q][1] = Dv[q][2] = Dv[q][3] = 0;
            }
        }
        if (ROLL && live) {
            int mk[5];
            bool fk[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                fk[k] = false;
                mk[k] = ghost_map(c + k - 2, n, bclo, bchi, &fk[k]);
            }
            const Real* wr = w + rowoff;
            // the next variable's stencil is loaded while this one computes
            // (x sweep at 256^3: 5.68 -> 4.81 ms per launch)
            Real vn[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) vn[k] = __ldg(wr + mk[k]);
#pragma unroll 1
            for (int q = 0; q < NS; ++q) {
                Real v[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) v[k] = (q == IM && fk[k]) ? -vn[k] : vn[k];
                if (q + 1 < NS) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) vn[k] = __ldg(wr + (q + 1) * nc + mk[k]);
                }
                Real Dq[4] = {v[1] - v[0], v[2] - v[1], v[3] - v[2], v[4] - v[3]};
                if constexpr (DFS) {
                    df er, el;
                    dfs_edges<Real, NF, NDIM, ORDER, NONUNIF, SIX, true>(a, 0, c, q, v[2], Dq, eps34, er, el);
                    dsh_eL[q][pos] = el;
                    dsh_eR[q][t] = er;
                } else {
                    Real er, el;
                    if constexpr (NONUNIF) {
                        const GridCol<true> grow(a.grid[0], a.grid_stride[0], c);
                        weno5_edges_nu(v[2], Dq, sweep_epsw<Real, 3>(a), grow, er, el);
                    } else {
                        weno_edges<ORDER>(v[2], Dq, eps34, er, el);
                    }
                    sh_eL[q][pos] = el;
                    sh_eR[q][t] = er;
                }
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const Real x1 = __ldg(wr + q * nc + mk[1]), x2 = __ldg(wr + q * nc + mk[2]);
                cm1[q] = (q == IM && fk[1]) ? -x1 : x1;
                vcv[q] = (q == IM && fk[2]) ? -x2 : x2;
            }
        }
        if (!ROLL && !LEARNED && live) {
            Real v[5][NS];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                bool flip = false;
                const int m = ghost_map(c + k - 2, n, bclo, bchi, &flip);
#pragma unroll
                for (int q = 0; q < NS; ++q) v[k][q] = __ldg(w + q * nc + rowoff + m);
                if (flip) v[k][IM] = -v[k][IM];
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                Dv[q][0] = v[1][q] - v[0][q];
                Dv[q][1] = v[2][q] - v[1][q];
                Dv[q][2] = v[3][q] - v[2][q];
                Dv[q][3] = v[4][q] - v[3][q];
                vcv[q] = v[2][q];
                cm1[q] = v[1][q];
            }
        }
        if (!ROLL && !LEARNED && live) {
            if constexpr (NONUNIF) {
                const GridCol<true> row(a.grid[0], a.grid_stride[0], c);
                const Real epsn = sweep_epsw<Real, 3>(a);   // unscaled eps
#pragma unroll
                for (int q = 0; q < NS; ++q) weno5_edges_nu(vcv[q], Dv[q], epsn, row, eR[q], eL[q]);
            } else {
#pragma unroll
                for (int q = 0; q < NS; ++q) weno_edges<ORDER>(vcv[q], Dv[q], eps34, eR[q], eL[q]);
            }
        }
        if constexpr (!LEARNED) {
#pragma unroll
            for (int q = 0; q < NS; ++q) cell[q] = vcv[q];
        }
        // left-side values of this chunk (the last chunk's last slot stays at
        // the position before this chunk's first)
        if (!ROLL && !LEARNED && live) {
#pragma unroll
            for (int q = 0; q < NS; ++q) sh_eL[q][pos] = eL[q];
        }
        __syncthreads();
        Real F[NQ], ut = 0;
        [[maybe_unused]] df Fd[DFS ? NQ : 1], utd = {0.f, 0.f};
        const bool has_face = live && c >= 0 && s >= own0 - 1;
        if constexpr (DFS) {
          if (has_face) {
            df lftd[NS], erd[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                lftd[q] = dsh_eL[q][pl];
                erd[q] = dsh_eR[q][t];
            }
            face_flux_df<NF, NDIM, 0, SIX>(a, edf, lftd, erd, cm1, cell, Fd, utd);
#pragma unroll
            for (int q = 0; q < NQ; ++q) dsh_F[q][pos] = Fd[q];
            dsh_F[NQ][pos] = utd;
          }
        } else if (has_face) {
            Real lft[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) lft[q] = sh_eL[q][pl];
            if constexpr (ROLL || LEARNED) {
#pragma unroll
                for (int q = 0; q < NS; ++q) eR[q] = sh_eR[q][t];
            }
            if constexpr (LEARNED) {
                face_flux_learned<NF, NDIM, 0>(
                    a, e, lft, eR,
                    [&](float* Lj, float* Rj) {
#pragma unroll
                        for (int q = 0; q < NS; ++q) {
                            Lj[q] = sh_eLJ[q][pl];
                            Rj[q] = sh_eRJ[q][t];
                        }
                    },
                    cm1, cell, F, ut);
            } else {
                face_flux<Real, NF, NDIM, 0, SIX>(a, e, lft, eR, cm1, cell, F, ut);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) sh_F[q][pos] = F[q];
            sh_F[NQ][pos] = ut;
        }
        __syncthreads();
        if (DFS && has_face && s >= own0 && c >= 1) {
            if constexpr (DFS) {
                df Fm[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) Fm[q] = dsh_F[q][pl];
                double idx_d = inv_dx;
                df idx_df = inv_df;
                if constexpr (NONUNIF) {   // this cell's width
                    idx_df = grid_df(GridCol<true>(a.grid[0], a.grid_stride[0], c - 1), kGridInvDx);
                    idx_d = df_to_double(idx_df);
                }
                racc.add(finish_cell_df<NF, NDIM, 0, SIX>(a, rowoff + (c - 1), Fm, Fd, dsh_F[NQ][pl], utd, cm1, idx_d,
                                                     idx_df, c - 1, 1, row));
            }
        } else if (has_face && s >= own0 && c >= 1) {
            Real Fm[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) Fm[q] = sh_F[q][pl];
            racc.add(finish_cell<Real, NF, NDIM, 0, SIX>(
                a, rowoff + (c - 1), Fm, F, sh_F[NQ][pl], ut, cm1,
                NONUNIF ? grid_inv_dx<true>(a.grid[0], a.grid_stride[0], c - 1, Real(0)) : inv_dx, c - 1, 1, row));
        }
        // No barrier is needed here: the next chunk writes edge values
        // (position pl of this chunk) after this chunk's second barrier, which
        // follows every read of them, and fluxes after its own first barrier,
        // which follows every finish of this chunk.  (The FP64 kernels kept one
        // while their unrolled reconstruction was instruction-cache bound; with
        // the looped one, dropping it took the 256^3 step 48.9 -> 48.5 ms.)
        pos = pl;
    }
    if constexpr (LEARNED) {
        if ((threadIdx.x & 31) == 0 && net_rows && a.net_rows) atomicAdd(a.net_rows, net_rows);
    }
    publish_rate(a, racc);
}

template <typename Real, int NF, int NDIM, bool LEARNED = false, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(kStreamThreads) sweep_x_stream_kernel(const SweepArgs a) {
    sweep_x_stream_body<Real, NF, NDIM, LEARNED, ORDER, NONUNIF, SIX>(a);
}

// The mixed form's five-equation x stream kernel on uniform grids, bounded to
// 7 CTAs per SM for up to two fluids (72 registers), 5 for three.
template <int NF, int NDIM, int ORDER = 5>
__global__ void __launch_bounds__(kStreamThreads, NF <= 2 ? 7 : 5) sweep_x_stream_f32_kernel(const SweepArgs a) {
    sweep_x_stream_body<float, NF, NDIM, false, ORDER, false, false>(a);
}

// The learned form's sweeps bounded to 4 CTAs per SM (128 registers, at most
// 12 bytes of spills; unbounded the x sweep took 168 and kept 12 warps per
// SM).  At 5 CTAs (96 registers, ~300 bytes of spills in x) the 256^3 step
// took 14.2 instead of 13.8 ms; y/z at 6 CTAs (80 registers), 15.2.
#ifndef MFC_LEARN_X_CTAS
#define MFC_LEARN_X_CTAS 4
#endif
#ifndef MFC_LEARN_YZ_CTAS
#define MFC_LEARN_YZ_CTAS 4
#endif
template <int NF, int NDIM>
__global__ void __launch_bounds__(kStreamThreads, MFC_LEARN_X_CTAS) sweep_x_stream_learned_kernel(const SweepArgs a) {
    sweep_x_stream_body<float, NF, NDIM, true, 5, false, false>(a);
}

// FP64 sweeps bounded to 4 CTAs (16 warps) per SM, for the variants where
// the extra warps outweigh the spills (launch_sweep chooses).
template <int NF, int NDIM, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(kStreamThreads, 4) sweep_x_stream_f64_kernel(const SweepArgs a) {
    sweep_x_stream_body<double, NF, NDIM, false, ORDER, NONUNIF, SIX>(a);
}

// ---------------------------------------------------------------------------
// y or z sweep as a coalesced stream.  A CTA of 4 warps covers 32
// consecutive x (lanes) of one pencil segment s0..s1-1 along DIR and walks it
// in chunks of 4 edge cells, one per warp: warp r of a chunk reconstructs the
// edges of cell c = base + r from its five-cell stencil, read from a shared
// ring of the 8 rows base-2..base+5 (each warp loads one new row per chunk,
// prefetched into registers during the previous chunk's arithmetic), forms the
// face c-1/2 with the left-side value of the previous row (a shared ring of
// 5 rows, which holds the previous chunk's last row too) and finishes cell
// c-1 (its operands staged or prefetched when the chunk starts).  Unlike the
// marching kernel no per-thread window is kept, so more warps stay resident to
// hide load and tensor-core latency.
// ---------------------------------------------------------------------------
constexpr int kRowsPerChunk = 4;

// STAGE: the kernel stages its finish operands (a.stage) in dynamic shared
// memory; entries without it keep the plain loads (and their registers).
template <typename Real, int NF, int NDIM, int DIR, bool LEARNED, int ORDER, bool NONUNIF = false, bool SIX = false,
          bool STAGE = false>
__device__ __forceinline__ void sweep_yz_stream_body(const SweepArgs& a) {
    static_assert(!SIX || !LEARNED, "six-equation model: FP64 and mixed forms");
    static_assert(!NONUNIF || (!LEARNED && ORDER == 5), "non-uniform grids: WENO5, FP64 and mixed forms");
    static_assert(!LEARNED || ORDER == 5, "the learned form replaces the WENO5 weights");
    static_assert(DIR == 1 || DIR == 2, "y or z");
    static_assert(!LEARNED || sizeof(Real) == 4, "the learned form runs in FP32");
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM;
    constexpr int NQ = Layout<NF, NDIM, SIX>::NQ;   // flux rows
    constexpr int NJ = LEARNED ? NS : 1;
    constexpr int T1 = 0;
    constexpr int T2 = (DIR == 2) ? 1 : 2;
    constexpr int RING = 2 * kRowsPerChunk;  // rows base-2 .. base+5 of a chunk
    // Edge values and face fluxes of cell c sit in row c mod ER of a ring of
    // ER = kRowsPerChunk + 1 rows: a chunk writes its four cells and reads
    // their left neighbours, the last of which the previous chunk wrote, and the
    // next chunk overwrites that row only after the barriers that order it.
    constexpr int ER = kRowsPerChunk + 1;
    // ROLL (FP64): one copy of the reconstruction looped over the variables
    // (stencils from the ring, edges to shared memory); see the x stream body.
    constexpr bool ROLL = sizeof(Real) == 8 && !LEARNED;
    __shared__ Real ring[RING][NS][32];
    __shared__ Real sh_eL[NS][ER][32];
    __shared__ Real sh_eR[(ROLL || LEARNED) ? NS : 1][kRowsPerChunk][32];
    // DFS: edge values kept in float-float into the Riemann solver (x stream body)
    constexpr bool DFS = ROLL;
    df(*dsh_eL)[ER][32] = reinterpret_cast<df(*)[ER][32]>(sh_eL);
    df(*dsh_eR)[kRowsPerChunk][32] = reinterpret_cast<df(*)[kRowsPerChunk][32]>(sh_eR);
    __shared__ Real sh_eLJ[NJ][ER][32];
    __shared__ Real sh_eRJ[NJ][kRowsPerChunk][32];
    __shared__ Real sh_F[NQ + 1][ER][32];
    df(*dsh_F)[ER][32] = reinterpret_cast<df(*)[ER][32]>(sh_F);   // DFS: float-float fluxes
    extern __shared__ __align__(16) unsigned char stage_smem[];   // a.stage operands
    static_assert(32 * kRowsPerChunk == kStageSlots, "one staging slot per thread");
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int n1 = a.g.n[T1], n2 = a.g.n[T2], nd = a.g.n[DIR];
    const int nxc = (n1 + 31) >> 5;
    const long long bid = blockIdx.x;
    const int xc = (int)(bid % nxc);
    const long long rest = bid / nxc;
    const int sg = (int)(rest % a.nseg);
    const int t2 = (int)(rest / a.nseg);
    if (t2 >= n2) return;  // whole CTA
    const bool active = xc * 32 + lane < n1;
    const int t1 = active ? xc * 32 + lane : n1 - 1;
    const long long sd = stride_of(a.g, DIR);
    const long long basei = (long long)t1 * stride_of(a.g, T1) + (long long)t2 * stride_of(a.g, T2);
    const long long nc = a.g.ncell;
    const int s0 = sg * a.seg;
    const int s1 = min(s0 + a.seg, nd);
    const int bclo = a.g.bc_lo[DIR], bchi = a.g.bc_hi[DIR];
    const Real eps34 = sweep_epsw<Real, ORDER>(a);  // 3/4 eps (WENO5) or eps (WENO3)
    const EosR<Real> e = sweep_eos<Real>(a);
    [[maybe_unused]] const EosDf edf(e);   // DFS: the EOS constants as float-float
    const Real inv_dx = sweep_inv_dx<Real>(a, DIR);
    [[maybe_unused]] const df inv_df = df_from_double((double)inv_dx);
    LearnRows* lsm = nullptr;
    if constexpr (LEARNED) {
        __shared__ LearnRows lbuf[kRowsPerChunk];
        lsm = &lbuf[row];
    }
    unsigned long long net_rows = 0;  // learned form: network rows of this warp
    RateAcc racc;                     // fused RK epilogue: CFL rate of the finished cells
    // cell i along DIR (ghost-mapped) of this lane's column
    auto load = [&](int i, Real* out) {
        bool flip = false;
        const int m = ghost_map(i, nd, bclo, bchi, &flip);
        const long long idx = basei + (long long)m * sd;
#pragma unroll
        for (int q = 0; q < NS; ++q) out[q] = __ldg(w + q * nc + idx);
        if (flip) out[IM + DIR] = -out[IM + DIR];
    };
    auto slot = [](int i) { return ((i % RING) + RING) % RING; };
    auto eslot = [](int i) { return (i + 2 * ER) % ER; };   // i >= -2
    // prologue: rows s0-3 .. s0+4 (cells base-2 .. base+5 of the first chunk)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = s0 - 3 + row + kRowsPerChunk * h;
        if (i <= s1 + 2) {
            Real v[NS];
            load(i, v);
#pragma unroll
            for (int q = 0; q < NS; ++q) ring[slot(i)][q][lane] = v[q];
        }
    }
    __syncthreads();

    for (int base = s0 - 1; base <= s1; base += kRowsPerChunk) {
        // prefetch the row the next chunk adds (cell base+6+row) while this one computes
        const int inext = base + RING - 2 + row;
        const bool pf = inext <= s1 + 2;
        Real nxt[NS];
        if (pf) load(inext, nxt);
        const int c = base + row;       // edge cell of this warp (warp-uniform)
        const bool live = c <= s1;
        const bool fin = live && c >= s0 + 1 && active;   // this lane finishes cell c-1 in this chunk
        if (fin) {
            const long long fidx = basei + (long long)(c - 1) * sd;
            int staged = 0;
            if constexpr (STAGE) {
                staged = a.stage;
                if (staged) stage_finish_operands<Real, NQ>(a, fidx, stage_smem, threadIdx.x);
            }
            // FP32 five-equation forms only: measured faster there (mixed 6.46 ->
            // 6.27, learned 14.2 -> 12.8, mixed stretched 10.3 -> 8.7 ms per step
            // at 256^3), not for the FP64 stretched-grid (70.3 -> 70.6) or the
            // six-equation sweeps (mixed 16.9 -> 17.2)
            if constexpr (sizeof(Real) == 4 && !SIX)
                prefetch_finish_operands<Real, NQ>(a, fidx, stage_mask(a) & ~staged);
        }
        Real cell[NS], cm1[NS], eL[NS], eR[NS];
        if (live) {
            if constexpr (LEARNED) {
                // one copy of the reconstruction looped over the variables
                // (stencils from the ring, edge values to shared memory)
                const int s0r = slot(c - 2), s1r = slot(c - 1), s2r = slot(c), s3r = slot(c + 1), s4r = slot(c + 2);
#pragma unroll 1
                for (int q = 0; q < NS; ++q) {
                    const float v0 = ring[s0r][q][lane], v1 = ring[s1r][q][lane], v2 = ring[s2r][q][lane];
                    const float v3 = ring[s3r][q][lane], v4 = ring[s4r][q][lane];
                    const float dq[4] = {v1 - v0, v2 - v1, v3 - v2, v4 - v3};
                    float ejR, ejL, elR, elL;
                    net_rows += learned_var_edges(v2, dq, eps34, a.tau, a.bound != 0, a.mlp_frag, *lsm, lane, ejR,
                                                  ejL, elR, elL);
                    sh_eL[q][eslot(c)][lane] = elL;
                    sh_eLJ[q][eslot(c)][lane] = ejL;
                    sh_eR[q][row][lane] = elR;
                    sh_eRJ[q][row][lane] = ejR;
                }
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    cell[q] = ring[s2r][q][lane];
                    cm1[q] = ring[s1r][q][lane];
                }
            } else if constexpr (ROLL) {
                const int s0r = slot(c - 2), s1r = slot(c - 1), s2r = slot(c), s3r = slot(c + 1), s4r = slot(c + 2);
#pragma unroll 1
                for (int q = 0; q < NS; ++q) {
                    const Real v0 = ring[s0r][q][lane], v1 = ring[s1r][q][lane], v2 = ring[s2r][q][lane];
                    const Real v3 = ring[s3r][q][lane], v4 = ring[s4r][q][lane];
                    Real Dq[4] = {v1 - v0, v2 - v1, v3 - v2, v4 - v3};
                    if constexpr (DFS) {
                        df er, el;
                        dfs_edges<Real, NF, NDIM, ORDER, NONUNIF, SIX, false>(a, DIR, c, q, v2, Dq, eps34, er, el);
                        dsh_eL[q][eslot(c)][lane] = el;
                        dsh_eR[q][row][lane] = er;
                    } else {
                        Real er, el;
                        if constexpr (NONUNIF) {
                            const GridCol<false> grow(a.grid[DIR], a.grid_stride[DIR], c);
                            weno5_edges_nu(v2, Dq, sweep_epsw<Real, 3>(a), grow, er, el);
                        } else {
                            weno_edges<ORDER>(v2, Dq, eps34, er, el);
                        }
                        sh_eL[q][eslot(c)][lane] = el;
                        sh_eR[q][row][lane] = er;
                    }
                }
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    cell[q] = ring[s2r][q][lane];
                    cm1[q] = ring[s1r][q][lane];
                }
            } else {
                Real Dv[NS][4];
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const Real v0 = ring[slot(c - 2)][q][lane], v1 = ring[slot(c - 1)][q][lane];
                    const Real v2 = ring[slot(c)][q][lane], v3 = ring[slot(c + 1)][q][lane];
                    const Real v4 = ring[slot(c + 2)][q][lane];
                    Dv[q][0] = v1 - v0;
                    Dv[q][1] = v2 - v1;
                    Dv[q][2] = v3 - v2;
                    Dv[q][3] = v4 - v3;
                    cell[q] = v2;
                    cm1[q] = v1;
                }
                if constexpr (NONUNIF) {
                    const GridCol<false> grow(a.grid[DIR], a.grid_stride[DIR], c);
                    const Real epsn = sweep_epsw<Real, 3>(a);   // unscaled eps
#pragma unroll
                    for (int q = 0; q < NS; ++q) weno5_edges_nu(cell[q], Dv[q], epsn, grow, eR[q], eL[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < NS; ++q) weno_edges<ORDER>(cell[q], Dv[q], eps34, eR[q], eL[q]);
                }
            }
            if constexpr (!ROLL && !LEARNED) {
#pragma unroll
                for (int q = 0; q < NS; ++q) sh_eL[q][eslot(c)][lane] = eL[q];
            }
        }
        __syncthreads();
        // rows base-2 .. base+1 are no longer needed: the prefetched rows replace them
        if (pf) {
#pragma unroll
            for (int q = 0; q < NS; ++q) ring[slot(inext)][q][lane] = nxt[q];
        }
        Real F[NQ], ut = 0;
        [[maybe_unused]] df Fd[DFS ? NQ : 1], utd = {0.f, 0.f};
        const bool has_face = live && c >= s0;
        if constexpr (DFS) {
          if (has_face) {
            df lftd[NS], erd[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                lftd[q] = dsh_eL[q][eslot(c - 1)][lane];
                erd[q] = dsh_eR[q][row][lane];
            }
            face_flux_df<NF, NDIM, DIR, SIX>(a, edf, lftd, erd, cm1, cell, Fd, utd);
#pragma unroll
            for (int q = 0; q < NQ; ++q) dsh_F[q][eslot(c)][lane] = Fd[q];
            dsh_F[NQ][eslot(c)][lane] = utd;
          }
        } else if (has_face) {
            Real lft[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) lft[q] = sh_eL[q][eslot(c - 1)][lane];
            if constexpr (ROLL || LEARNED) {
#pragma unroll
                for (int q = 0; q < NS; ++q) eR[q] = sh_eR[q][row][lane];
            }
            if constexpr (LEARNED) {
                face_flux_learned<NF, NDIM, DIR>(
                    a, e, lft, eR,
                    [&](float* Lj, float* Rj) {
#pragma unroll
                        for (int q = 0; q < NS; ++q) {
                            Lj[q] = sh_eLJ[q][eslot(c - 1)][lane];
                            Rj[q] = sh_eRJ[q][row][lane];
                        }
                    },
                    cm1, cell, F, ut);
            } else {
                face_flux<Real, NF, NDIM, DIR, SIX>(a, e, lft, eR, cm1, cell, F, ut);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) sh_F[q][eslot(c)][lane] = F[q];
            sh_F[NQ][eslot(c)][lane] = ut;
        }
        __syncthreads();
        if (fin) {
            const unsigned char* stg = nullptr;
            if constexpr (STAGE) {
                if (a.stage) {
                    cp_async_wait_all();
                    stg = stage_smem;
                }
            }
            if constexpr (DFS) {
                df Fm[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) Fm[q] = dsh_F[q][eslot(c - 1)][lane];
                double idx_d = inv_dx;
                df idx_df = inv_df;
                if constexpr (NONUNIF) {   // this cell's width
                    idx_df = grid_df(GridCol<false>(a.grid[DIR], a.grid_stride[DIR], c - 1), kGridInvDx);
                    idx_d = df_to_double(idx_df);
                }
                racc.add(finish_cell_df<NF, NDIM, DIR, SIX>(a, basei + (long long)(c - 1) * sd, Fm, Fd,
                                                       dsh_F[NQ][eslot(c - 1)][lane], utd, cm1, idx_d, idx_df, c - 1,
                                                       sd, (long long)t1 + (long long)n1 * t2, stg, threadIdx.x));
            } else {
                Real Fm[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) Fm[q] = sh_F[q][eslot(c - 1)][lane];
                racc.add(finish_cell<Real, NF, NDIM, DIR, SIX>(
                    a, basei + (long long)(c - 1) * sd, Fm, F, sh_F[NQ][eslot(c - 1)][lane], ut, cm1,
                    NONUNIF ? grid_inv_dx<false>(a.grid[DIR], a.grid_stride[DIR], c - 1, Real(0)) : inv_dx, c - 1, sd,
                    (long long)t1 + (long long)n1 * t2, stg, threadIdx.x));
            }
        }
        // No barrier is needed here: the next chunk writes edge values (row
        // c+4 = c-1 mod ER) after this chunk's second barrier, which follows
        // every read of them, and fluxes after its own first barrier, which
        // follows every finish of this chunk.
    }
    if constexpr (LEARNED) {
        if ((threadIdx.x & 31) == 0 && net_rows && a.net_rows) atomicAdd(a.net_rows, net_rows);
    }
    publish_rate(a, racc);
}

// The y/z stream kernel (FP64 uniform WENO5 forms, with staged finish
// operands, and the mixed form on non-uniform grids, without: staging took
// it from 96 to 123 registers): the compiler's own register allocation.
template <typename Real, int NF, int NDIM, int DIR, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(32 * kRowsPerChunk) sweep_yz_stream_kernel(const SweepArgs a) {
    sweep_yz_stream_body<Real, NF, NDIM, DIR, false, ORDER, NONUNIF, SIX, sizeof(Real) == 8>(a);
}

// The mixed form's five-equation y/z stream kernel on uniform grids, with
// staged finish operands: bounded to 8 CTAs per SM for up to two fluids (64
// registers, no spills), 5 for three, so that the registers allow the
// residency the staging's shared memory does.  The learned form gets its own
// entry below.
template <int NF, int NDIM, int DIR, int ORDER = 5>
__global__ void __launch_bounds__(32 * kRowsPerChunk, NF <= 2 ? 8 : 5) sweep_yz_stream_f32_kernel(const SweepArgs a) {
    sweep_yz_stream_body<float, NF, NDIM, DIR, false, ORDER, false, false, true>(a);
}

// The mixed form's six-equation y/z sweep: bounded to 5 CTAs per SM (96
// registers; unbounded it took 107 and ran 45 instead of 37 ms over the 256^3
// bench).  A bound of one CTA per SM is not the same as none: it slowed the
// five-equation kernels by half, hence a separate entry.
template <int NF, int NDIM, int DIR, int ORDER = 5, bool NONUNIF = false>
__global__ void __launch_bounds__(32 * kRowsPerChunk, 5) sweep_yz_stream_six32_kernel(const SweepArgs a) {
    sweep_yz_stream_body<float, NF, NDIM, DIR, false, ORDER, NONUNIF, true, true>(a);
}

// The bounded FP64 y/z stream kernel (stretched-grid, six-equation and WENO3
// forms, 4 CTAs per SM).  Staging pays for WENO3 (40.7 -> 39.2 ms per step at
// 256^3), not on stretched grids (70.0 -> 71.8 ms, more spills at the bound).
template <int NF, int NDIM, int DIR, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(32 * kRowsPerChunk, 4) sweep_yz_stream_f64_kernel(const SweepArgs a) {
    sweep_yz_stream_body<double, NF, NDIM, DIR, false, ORDER, NONUNIF, SIX, !NONUNIF>(a);
}

// The FP64 uniform WENO5 y/z stream kernel for three fluids, bounded to 3
// CTAs per SM (168 registers; unbounded it takes 187-192 and keeps 2), the z
// sweep (RK epilogue) to 4 (128 registers, 76 bytes of spills): 512^3 step
// 356.2 -> 346.7 ms with both at 4, the y sweep alone slower at 4.
template <int NF, int NDIM, int DIR>
__global__ void __launch_bounds__(32 * kRowsPerChunk, DIR == 2 ? 4 : 3) sweep_yz_stream_f64b3_kernel(const SweepArgs a) {
    sweep_yz_stream_body<double, NF, NDIM, DIR, false, 5, false, false, true>(a);
}

template <int NF, int NDIM, int DIR>
__global__ void __launch_bounds__(32 * kRowsPerChunk, NF <= 2 ? MFC_LEARN_YZ_CTAS : 3)
    sweep_yz_stream_learned_kernel(const SweepArgs a) {
    sweep_yz_stream_body<float, NF, NDIM, DIR, true, 5, false, false, true>(a);
}

}  // namespace mfc
