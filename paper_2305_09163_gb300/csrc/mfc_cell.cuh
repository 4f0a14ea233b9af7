// Finishing a cell (Sec. 3.1, 3.3, 3.4, 2.1, 2.3): characteristic boundary
// rates, the Kapila coefficients, the six-equation pressure relaxation, and
// finish_cell (flux difference, sources, RK stage update).
#pragma once
#include "mfc_learned.cuh"

namespace mfc {

// Characteristic (non-reflecting) boundary (Sec. 3.3: characteristic-based
// conditions after Thompson).  Normal part of dq/dt of a boundary cell from
// the quasi-linear primitive equations along DIR, written with the wave
// amplitudes L1 = (u - c)(p_x - r c u_x), L5 = (u + c)(p_x + r c u_x),
// Lk = u ((a_k r_k)_x - a_k r_k p_x/(r c^2)) and u (.)_x for the tangential
// velocities and volume fractions; the amplitudes of waves entering the domain
// (speed > 0 at the low boundary, < 0 at the high one) are zero.  wb: the
// cell's primitives, wx: their one-sided derivative towards the interior
// neighbour.  Rates: p_t = -(L5 + L1)/2, u_t = -(L5 - L1)/(2 r c),
// (a_k r_k)_t = -Lk - a_k r_k (L5 + L1)/(2 r c^2), others -L; then conserved.
// Not inlined: only boundary cells run it.
template <typename Real, int NF, int NDIM, int DIR>
__device__ __noinline__ void cbc_rate(const EosR<Real>& e, const Real* wb, const Real* wx, bool high, Real* out) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    Real r = 0, G = e.G_N, P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF; ++k) r += wb[k];
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        G = fma(e.dG[k], wb[IA + k], G);
        P = fma(e.dP[k], wb[IA + k], P);
    }
    const Real p = wb[IE], u = wb[IM + DIR];
    const Real rc2 = ((G + (Real)1) * p + P) / G;          // r c^2
    const Real c = sqrt(rc2 / r);
    const Real ux = wx[IM + DIR], px = wx[IE];
    const Real lam1 = u - c, lam5 = u + c;
    const bool in1 = high ? lam1 < (Real)0 : lam1 > (Real)0;
    const bool in5 = high ? lam5 < (Real)0 : lam5 > (Real)0;
    const bool inu = high ? u < (Real)0 : u > (Real)0;
    const Real L1 = in1 ? (Real)0 : lam1 * (px - r * c * ux);
    const Real L5 = in5 ? (Real)0 : lam5 * (px + r * c * ux);
    const Real ac = (L5 + L1) / (2 * rc2);
    Real wt[NS];
#pragma unroll
    for (int k = 0; k < NF; ++k) wt[k] = -(inu ? (Real)0 : u * (wx[k] - wb[k] * px / rc2)) - wb[k] * ac;
#pragma unroll
    for (int m = 0; m < NDIM; ++m) wt[IM + m] = m == DIR ? -(L5 - L1) / (2 * r * c) : (inu ? (Real)0 : -u * wx[IM + m]);
    wt[IE] = -(L5 + L1) / 2;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) wt[IA + k] = inu ? (Real)0 : -u * wx[IA + k];
    Real rt = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        out[k] = wt[k];
        rt += wt[k];
    }
    Real ke = 0, kt = 0;
#pragma unroll
    for (int m = 0; m < NDIM; ++m) {
        const Real um = wb[IM + m];
        out[IM + m] = fma(um, rt, r * wt[IM + m]);
        ke = fma((Real)0.5 * um, um, ke);
        kt = fma(um, wt[IM + m], kt);
    }
    Real Gt = 0, Pt = 0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        Gt = fma(e.dG[k], wt[IA + k], Gt);
        Pt = fma(e.dP[k], wt[IA + k], Pt);
        out[IA + k] = wt[IA + k];
    }
    out[IE] = G * wt[IE] + p * Gt + Pt + ke * rt + r * kt;
}

// Kapila coefficients (Sec. 2.1, 5-equation models): the volume-fraction rows
// carry (alpha_k + K_k) div(u) instead of alpha_k div(u), with
//   K_k = alpha_k (rho c_W^2 / Z_k - 1),  1/(rho c_W^2) = sum_j alpha_j / Z_j,
// Z_k = rho_k c_k^2 = gamma_k (p + pi_inf_k) for a stiffened gas (Kapila's
// N-phase form; for two phases the formula the section prints).  Written
// with one reciprocal: rho c_W^2 / Z_k = prod_{j != k} Z_j / sum_j alpha_j
// prod_{i != j} Z_i.  w is the primitive state of the cell.  Not inlined:
// the Allaire path of the sweeps keeps its instruction schedule.
template <typename Real, int NF, int NDIM>
__device__ __noinline__ void kapila_K(const SweepArgs& a, const Real* w, Real* K) {
    using Lay = Layout<NF, NDIM>;
    const Real p = w[Lay::IE];
    Real al[NF], Z[NF];
    Real last = (Real)1;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        al[k] = w[Lay::IA + k];
        last -= al[k];
    }
    al[NF - 1] = last;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        if constexpr (sizeof(Real) == 4) Z[k] = a.kgamf[k] * (p + a.kpinff[k]);
        else Z[k] = a.kgam[k] * (p + a.kpinf[k]);
    }
    Real pe[NF];   // product of the other phases' Z
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        Real t = (Real)1;
#pragma unroll
        for (int j = 0; j < NF; ++j)
            if (j != k) t *= Z[j];
        pe[k] = t;
    }
    Real D = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) D = fma(al[k], pe[k], D);
    const Real rD = real_rcp(D);
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) K[k] = al[k] * fma(pe[k], rD, (Real)-1);
}

// The same coefficients for the FP64 path, in float-float arithmetic
// (mfc_df.cuh) and inlined: the FP64 instructions of a reciprocal and the
// call would cost more than the rest of the source term.
template <int NF, int NDIM>
__device__ __forceinline__ void kapila_K_df(const SweepArgs& a, const double* w, double* K) {
    using Lay = Layout<NF, NDIM>;
    const df p = df_from_double(w[Lay::IE]);
    df al[NF], Z[NF];
    double last = 1.0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        al[k] = df_from_double(w[Lay::IA + k]);
        last -= w[Lay::IA + k];
    }
    al[NF - 1] = df_from_double(last);
#pragma unroll
    for (int k = 0; k < NF; ++k)   // gamma_k as float-float: its FP32 rounding would show in K
        Z[k] = df_mul(df_add(p, df_from_double(a.kpinf[k])), df_from_double(a.kgam[k]));
    df pe[NF];   // product of the other phases' Z
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        df t = {1.f, 0.f};
        bool first = true;
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            if (j == k) continue;
            t = first ? Z[j] : df_mul(t, Z[j]);
            first = false;
        }
        pe[k] = t;
    }
    df D = df_mul(al[0], pe[0]);
#pragma unroll
    for (int k = 1; k < NF; ++k) D = df_add(D, df_mul(al[k], pe[k]));
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) K[k] = df_to_double(df_mul(al[k], df_add(df_div(pe[k], D), {-1.f, 0.f})));
}

// Six-equation model (Sec. 2.3): pressure relaxation of one cell's conserved
// state q[NQ] with infinite stiffness, in place, after a Runge-Kutta stage
// (Saurel, Petitpas & Berry 2009; Schmidmayer et al. 2020).  At fixed mass
// each phase's energy follows de_k = -p dv_k at the final pressure p, which for
// a stiffened gas gives the relaxed volume fraction
//     a_k(p) = (g_k - 1)(E_k0 + a_k0 p) / (g_k (p + pinf_k)),  E_k0 = a_k r_k e_k.
// The phases taking part are those with a_k0 > 0 and p_k0 + pinf_k > 0
// (E_k0 > a_k0 pinf_k); the others keep a_k0.  The relaxed pressure solves
// f(p) = sum_{taking part} a_k(p) - (1 - sum_{others} a_k0) = 0; on
// p > lo = -min pinf (over the phases taking part) f is convex and falls
// strictly from +inf to below zero, so the root is unique.
//  1. FP32 Newton from the pressure the mixture law gives for the total energy
//     with the old fractions (the root itself for a relaxed state): from the
//     left of the root Newton rises monotonically to it, from the right it
//     lands left of it unless it would leave the domain, when the step bisects
//     [lo, p] instead; at most 60 iterations, ending at a relative step of 2^-20;
//  2. two Newton steps with f in float-float arithmetic (f' in FP32 suffices:
//     its error only slows the quadratic convergence to a linear one with
//     factor ~1e-7), which bring p to ~1e-14 relative;
//  3. one FP64 Newton step, p1 = p0 - f(p0)/f'(p0), and the new fractions
//     a_k(p1) = a_k(p0) + a_k'(p0)(p1 - p0) (the second-order remainder is
//     below FP64 rounding): a fraction near 1 must be right to ~1e-16
//     absolute, since a trace phase's fraction is 1 minus it;
//  4. in FP64 the pressure of the total energy with the mixture law of the
//     new fractions and every phase's energy reset to it.
// On GB300 an FP64 instruction costs the issue time of ~60 FP32 ones; the
// iteration is the costly part, hence steps 1-2 (see mfc_df.cuh).
template <int NF, int NDIM>
__device__ __noinline__ void relax6(const SweepArgs& a, double* q) {
    using Lay = Layout<NF, NDIM, true>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA, II = Lay::II;
    double a0[NF], E0[NF];
    bool in[NF];
    double asum = 0.0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        a0[k] = q[IA + k];
        asum += a0[k];
    }
    a0[NF - 1] = 1.0 - asum;
    double target = 1.0;
    float lo = 0.f;
    bool any = false;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        E0[k] = q[II + k];
        in[k] = a0[k] > 0.0 && E0[k] > a0[k] * a.kpinf[k];
        if (!in[k]) {
            target -= a0[k];
            continue;
        }
        lo = any ? fmaxf(lo, -a.kpinff[k]) : -a.kpinff[k];
        any = true;
    }
    if (!any) return;   // no phase can relax: left as is (the CFL check flags it)
    // mixture-law pressure of the total energy (old fractions, then new ones)
    double r = q[0], m2 = 0.0;
#pragma unroll
    for (int k = 1; k < NF; ++k) r += q[k];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) m2 = fma(q[IM + d], q[IM + d], m2);
    const double eint = q[IE] - 0.5 * m2 * rcp_nr(r);
    auto mixture_p = [&]() {
        double G = a.e.G_N, P = a.e.P_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            G = fma(q[IA + k], a.e.dG[k], G);
            P = fma(q[IA + k], a.e.dP[k], P);
        }
        return (eint - P) * rcp_nr(G);
    };
    // the phases in float-float (integer splits) and FP32
    df a0d[NF], E0d[NF], pid[NF], c1d[NF];
    float a0f[NF], E0f[NF], pif[NF], c1f[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        a0d[k] = df_from_double(a0[k]);
        E0d[k] = df_from_double(E0[k]);
        pid[k] = df_from_double(a.kpinf[k]);
        c1d[k] = df_from_double(a.rc1[k]);
        a0f[k] = a0d[k].hi;
        E0f[k] = E0d[k].hi;
        pif[k] = a.kpinff[k];
        c1f[k] = c1d[k].hi;
    }
    const df targetd = df_from_double(target);
    // 1. FP32 Newton
    float p = (float)mixture_p();
    if (!(p > lo)) p = lo + fmaxf(fabsf(lo), 1.f);
    float hi = INFINITY;
    for (int it = 0; it < 60; ++it) {
        float f = -targetd.hi, fp = 0.f;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (!in[k]) continue;
            const float t = rcp_approx(p + pif[k]);
            f = fmaf(c1f[k] * fmaf(a0f[k], p, E0f[k]), t, f);
            fp = fmaf(c1f[k] * fmaf(a0f[k], pif[k], -E0f[k]), t * t, fp);
        }
        if (f > 0.f) lo = p;
        else hi = p;
        float pn = p - f * rcp_approx(fp);
        if (!(pn > lo && pn < hi)) pn = 0.5f * (lo + (hi < INFINITY ? hi : p));
        const bool done = fabsf(pn - p) <= 0x1p-20f * fabsf(pn) || !(pn > lo && pn < hi);
        p = pn;
        if (done) break;
    }
    // 2. float-float Newton steps
    df pd = {p, 0.f};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        df f = df_neg(targetd);
        float fp = 0.f;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (!in[k]) continue;
            const df num = df_add(E0d[k], df_mul(a0d[k], pd));
            const df den = df_add(pd, pid[k]);
            f = df_add(f, df_mul(c1d[k], df_div(num, den)));
            const float t = rcp_approx(den.hi);
            fp = fmaf(c1f[k] * fmaf(a0f[k], pif[k], -E0f[k]), t * t, fp);
        }
        pd = df_add(pd, {-(f.hi + f.lo) * rcp_approx(fp), 0.f});
    }
    // 3. one FP64 Newton step and the fractions at its end (first order)
    const double p0 = df_to_double(pd);
    double ak[NF], dak[NF], f64 = -target, fp64 = 0.0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        ak[k] = a0[k];
        dak[k] = 0.0;
        if (!in[k]) continue;
        const double pi = a.kpinf[k];
        const double t = rcp_nr(p0 + pi);
        ak[k] = a.rc1[k] * fma(a0[k], p0, E0[k]) * t;
        dak[k] = a.rc1[k] * fma(a0[k], pi, -E0[k]) * t * t;
        f64 += ak[k];
        fp64 += dak[k];
    }
    const double dp = df_widen(-(float)f64 * rcp_approx((float)fp64));
    // 4. new fractions, the pressure of the total energy, the phase energies
    double an = 1.0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        if (in[k]) q[IA + k] = fma(dak[k], dp, ak[k]);
        an -= q[IA + k];
    }
    const double pe = mixture_p();
#pragma unroll
    for (int k = 0; k < NF - 1; ++k)
        q[II + k] = q[IA + k] * fma(a.e.G_N + a.e.dG[k], pe, a.e.P_N + a.e.dP[k]);
    q[II + NF - 1] = an * fma(a.e.G_N, pe, a.e.P_N);
}

// Normal rate of a characteristic boundary cell (flat index idx, neighbours
// sd apart along DIR; n cells along DIR) from its primitives and those of its
// interior neighbour.
template <typename Real, int NF, int NDIM, int DIR>
__device__ __noinline__ void cbc_cell_rate(const SweepArgs& a, long long idx, long long sd, int n, bool high,
                                           Real inv_dx, Real* out) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS;
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const long long nc = a.g.ncell;
    const long long nb = n > 1 ? (high ? idx - sd : idx + sd) : idx;   // one cell: no gradient
    Real wb[NS], wx[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        wb[q] = w[q * nc + idx];
        const Real wn = w[q * nc + nb];
        wx[q] = (high ? wb[q] - wn : wn - wb[q]) * inv_dx;
    }
    cbc_rate<Real, NF, NDIM, DIR>(sweep_eos<Real>(a), wb, wx, high, out);
}

// Characteristic boundary rates of every boundary cell, ahead of the sweeps:
// one lane per cell, so no sweep warp waits on the FP64 boundary arithmetic.
// cbc_rates holds, for direction d and side s (0 low, 1 high) from
// cbc_off[d][s], NS rows of the plane's cells, indexed by the transverse flat
// index tr (x fastest among the two other directions).
template <typename Real, int NF, int NDIM>
__global__ void __launch_bounds__(256) cbc_rates_kernel(const SweepArgs a, long long total) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS;
    Real* out = static_cast<Real*>(const_cast<void*>(a.cbc_rates));
    const int nx = a.g.n[0], ny = a.g.n[1];
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        int dir = -1, side = 0;
        long long tr = 0, nt = 0, base = 0;
        for (int dd = 0; dd < NDIM && dir < 0; ++dd)
            for (int s = 0; s < 2 && dir < 0; ++s) {
                const long long o = a.cbc_off[dd][s];
                if (o < 0) continue;
                const long long cnt = a.g.ncell / a.g.n[dd];
                const long long first = o / NS;   // cells before this plane
                if (g < first + cnt) {
                    dir = dd;
                    side = s;
                    tr = g - first;
                    nt = cnt;
                    base = o;
                }
            }
        if (dir < 0) continue;
        const int n = a.g.n[dir];
        const int b = side ? n - 1 : 0;
        long long idx;
        if (dir == 0) idx = (long long)b + (long long)nx * tr;
        else if (dir == 1) idx = (tr % nx) + (long long)nx * (b + (long long)ny * (tr / nx));
        else idx = tr + (long long)nx * ny * b;
        const long long sd = stride_of(a.g, dir);
        Real inv = (Real)a.g.inv_dx[dir];
        if (a.grid[dir])
            inv = dir == 0 ? grid_inv_dx<true>(a.grid[0], a.grid_stride[0], b, Real(0))
                           : grid_inv_dx<false>(a.grid[dir], a.grid_stride[dir], b, Real(0));
        Real r[NS];
        if (dir == 0) cbc_cell_rate<Real, NF, NDIM, 0>(a, idx, sd, n, side == 1, inv, r);
        else if (dir == 1) {
            if constexpr (NDIM > 1) cbc_cell_rate<Real, NF, NDIM, 1>(a, idx, sd, n, side == 1, inv, r);
        } else {
            if constexpr (NDIM > 2) cbc_cell_rate<Real, NF, NDIM, 2>(a, idx, sd, n, side == 1, inv, r);
        }
#pragma unroll
        for (int v = 0; v < NS; ++v) out[base + v * nt + tr] = r[v];
    }
}

// Finish-operand staging of the y/z stream kernels.  The R accumulator, qs and
// q0 values of the cell a lane finishes in a chunk are copied to shared memory
// by cp.async when the chunk starts, so their DRAM latency overlaps the
// chunk's reconstruction and Riemann arithmetic instead of stalling the
// finish.  Layout: [R: NQ x kStageSlots Real][qs: NQ x kStageSlots double]
// [q0: NQ x kStageSlots double], only the parts a.stage selects, slot = the
// thread's index in its CTA.  Each lane reads back only what it staged itself.
constexpr int kStageSlots = 128;

template <int B>
__device__ __forceinline__ void cp_async_ca(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename Real, int NQ>
__host__ __device__ constexpr size_t stage_offset_qs(int mask) {
    return (mask & 1) ? (size_t)NQ * kStageSlots * sizeof(Real) : 0;
}
template <typename Real, int NQ>
__host__ __device__ constexpr size_t stage_offset_q0(int mask) {
    return stage_offset_qs<Real, NQ>(mask) + ((mask & 2) ? (size_t)NQ * kStageSlots * sizeof(double) : 0);
}
template <typename Real, int NQ>
__host__ __device__ constexpr size_t stage_bytes(int mask) {
    return stage_offset_q0<Real, NQ>(mask) + ((mask & 4) ? (size_t)NQ * kStageSlots * sizeof(double) : 0);
}

// Finish operands of a sweep launch, as a staging mask: the R accumulator
// where the finish reads it, qs in an RK stage, q0 where the stage has a q0
// term.
__host__ __device__ inline int stage_mask(const SweepArgs& a) {
    switch (a.mode) {
        case 1: return 1;
        case 2: return (a.acc_in ? 1 : 0) | 2 | (a.c0 != 0.0 ? 4 : 0);
        case 3: return a.acc_in ? 1 : 0;
        default: return 0;
    }
}

// The finish operands in mask m that are not staged: an L2 prefetch when the
// chunk starts, so that the finish's own loads meet L2 rather than DRAM.
template <typename Real, int NQ>
__device__ __forceinline__ void prefetch_finish_operands(const SweepArgs& a, long long idx, int m) {
    const long long nc = a.g.ncell;
    if (m & 1) {
        const Real* R = static_cast<const Real*>(a.R);
#pragma unroll
        for (int v = 0; v < NQ; ++v) asm volatile("prefetch.global.L2 [%0];" ::"l"(R + v * nc + idx));
    }
    if (m & 2) {
#pragma unroll
        for (int v = 0; v < NQ; ++v) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.qs + v * nc + idx));
    }
    if (m & 4) {
#pragma unroll
        for (int v = 0; v < NQ; ++v) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.q0 + v * nc + idx));
    }
}

template <typename Real, int NQ>
__device__ __forceinline__ void stage_finish_operands(const SweepArgs& a, long long idx, unsigned char* stg, int slot) {
    const long long nc = a.g.ncell;
    const int m = a.stage;
    if (m & 1) {
        Real* d = reinterpret_cast<Real*>(stg) + slot;
        const Real* R = static_cast<const Real*>(a.R);
#pragma unroll
        for (int v = 0; v < NQ; ++v) cp_async_ca<sizeof(Real)>(d + v * kStageSlots, R + v * nc + idx);
    }
    if (m & 2) {
        double* d = reinterpret_cast<double*>(stg + stage_offset_qs<Real, NQ>(m)) + slot;
#pragma unroll
        for (int v = 0; v < NQ; ++v) cp_async_ca<8>(d + v * kStageSlots, a.qs + v * nc + idx);
    }
    if (m & 4) {
        double* d = reinterpret_cast<double*>(stg + stage_offset_q0<Real, NQ>(m)) + slot;
#pragma unroll
        for (int v = 0; v < NQ; ++v) cp_async_ca<8>(d + v * kStageSlots, a.q0 + v * nc + idx);
    }
    cp_async_commit();
}

// ---------------------------------------------------------------------------
// Conserved -> primitive (Sec. 2.1): rho = sum a_k r_k, u = (rho u)/rho,
// p = (rho E - rho|u|^2/2 - Pi)/Gamma.  FP64 path: all in FP64.  Mixed path:
// rho E - Pi (the water Pi ~ 7.8e8 Pa cancels against rho E) and the kinetic
// energy subtraction stay FP64, the rest is FP32.  Optionally the CFL rate
// max_d (|u_d| + c)/dx_d with c^2 = ((Gamma+1)p + Pi)/(Gamma rho), reduced to one
// max per launch with an order-preserving integer atomic (non-negative
// doubles), so it is exact and independent of scheduling.  Six-equation model
// (SIX): the frozen sound speed, r c^2 = A p + B (Sec. 2.3).
// ---------------------------------------------------------------------------
template <int NF, int NDIM, bool SIX = false>
__device__ __forceinline__ void prims_cell(const double* q, const EosConst& e, double* wv, double& c2) {
    using Lay = Layout<NF, NDIM>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    double rho = q[0];
#pragma unroll
    for (int k = 1; k < NF; ++k) rho += q[k];
    double G = e.G_N, P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        G = fma(q[IA + k], e.dG[k], G);
        P = fma(q[IA + k], e.dP[k], P);
    }
    const double x = rcp_nr(rho * G);   // FP32 seed + cubic Newton step: 3 FP64 instructions
    const double irho = G * x, iG = rho * x;
    double ke = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) { wv[IM + d] = q[IM + d] * irho; ke = fma(q[IM + d], wv[IM + d], ke); }
    const double p = (q[IE] - 0.5 * ke - P) * iG;
#pragma unroll
    for (int k = 0; k < NF; ++k) wv[k] = q[k];
    wv[IE] = p;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) wv[IA + k] = q[IA + k];
    if constexpr (SIX) {
        double A = e.A_N, B = e.B_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            A = fma(q[IA + k], e.dA[k], A);
            B = fma(q[IA + k], e.dB[k], B);
        }
        c2 = fma(A, p, B) * irho;
    } else {
        c2 = fma(G + 1.0, p, P) * iG * irho;
    }
}

// FP32 form: the per-cell FP64 -> FP32 conversions by integer operations
// (narrow_rn, df_widen), since conversion instructions run on the FP64 pipe.
template <int NF, int NDIM, bool SIX = false>
__device__ __forceinline__ void prims_cell(const double* q, const EosConst& e, float* wv, float& c2) {
    using Lay = Layout<NF, NDIM>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    float qf[Lay::NS];
#pragma unroll
    for (int v = 0; v < Lay::NS; ++v) qf[v] = v == IE ? 0.f : narrow_rn(q[v]);
    float rho = qf[0];
#pragma unroll
    for (int k = 1; k < NF; ++k) rho += qf[k];
    float G = (float)e.G_N;
    double P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        G = fmaf(qf[IA + k], (float)e.dG[k], G);
        P = fma(q[IA + k], e.dP[k], P);
    }
    const float irho = __fdividef(1.0f, rho);
    float ke = 0.f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const float m = qf[IM + d];
        wv[IM + d] = m * irho;
        ke = fmaf(m, wv[IM + d], ke);
    }
    const double eint = fma(-0.5, df_widen(ke), q[IE] - P);
    const float p = __fdividef(narrow_rn(eint), G);
#pragma unroll
    for (int k = 0; k < NF; ++k) wv[k] = qf[k];
    wv[IE] = p;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) wv[IA + k] = qf[IA + k];
    if constexpr (SIX) {
        float A = (float)e.A_N, B = (float)e.B_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            A = fmaf(qf[IA + k], (float)e.dA[k], A);
            B = fmaf(qf[IA + k], (float)e.dB[k], B);
        }
        c2 = __fdividef(fmaf(A, p, B), rho);
    } else {
        c2 = __fdividef(fmaf(G + 1.0f, p, narrow_rn(P)), G * rho);
    }
}

// CFL rate of one cell from its primitives (Sec. 1: the CFL restriction),
// max_d (|u_d| + c)/dx_d, in the arithmetic of the path (FP64: the root in
// float-float, ~2^-46 relative, off the FP64 pipe; FP32 forms: FP32), or -1
// for a non-physical cell (c^2 <= 0 or a non-finite value).  i: the cell's
// index (non-uniform grids take its widths from the tables).  Shared by the
// primitive-recovery kernel and the fused RK epilogue, so both give the same
// bits.
template <typename Real, int NF, int NDIM>
__device__ __forceinline__ double cell_cfl_rate(const Real* wv, Real c2, const Geometry& g, const float* const* grid,
                                                const int* grid_stride, long long i) {
    constexpr int IM = Layout<NF, NDIM>::IM;
    Real us = 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) us += wv[IM + d];
    if (!(c2 > (Real)0) || !(c2 - c2 == (Real)0) || !(us - us == (Real)0)) return -1.0;
    Real cs;
    if constexpr (sizeof(Real) == 8) cs = df_to_double(df_sqrt(df_from_double(c2)));
    else cs = real_sqrt(c2);
    Real r = 0;
    int ci[3] = {0, 0, 0};
    if (grid[0] || grid[1] || grid[2]) {   // non-uniform: this cell's widths
        const unsigned ii = (unsigned)i, nx = (unsigned)g.n[0], ny = (unsigned)g.n[1];
        ci[0] = (int)(ii % nx);
        ci[1] = (int)((ii / nx) % ny);
        ci[2] = (int)(ii / (nx * ny));
    }
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const Real inv = !grid[d] ? (Real)g.inv_dx[d]
                         : d == 0 ? grid_inv_dx<true>(grid[d], grid_stride[d], ci[d], Real(0))
                                  : grid_inv_dx<false>(grid[d], grid_stride[d], ci[d], Real(0));
        r = real_max(r, (fabs(wv[IM + d]) + cs) * inv);
    }
    return (double)r;
}

// Running CFL maximum and non-physical count of the cells a thread finished
// (fused RK epilogue), published once per kernel: the converged lanes reduce
// the ordered bits of the non-negative rate (high word, then the low word among
// the lanes holding the largest high word) and one lane does the atomics.
struct RateAcc {
    double rate = 0.0;
    int bad = 0;
    __device__ __forceinline__ void add(double r) {
        if (r < 0.0) bad += 1;
        else rate = fmax(rate, r);
    }
};

__device__ __forceinline__ void publish_rate(const SweepArgs& a, const RateAcc& acc) {
    if (!a.rate_max) return;
    const unsigned mask = __activemask();
    const unsigned long long bits = (unsigned long long)__double_as_longlong(acc.rate);
    const unsigned hi = (unsigned)(bits >> 32);
    const unsigned mhi = __reduce_max_sync(mask, hi);
    const unsigned mlo = __reduce_max_sync(mask, hi == mhi ? (unsigned)bits : 0u);
    const unsigned nbad = __reduce_add_sync(mask, (unsigned)acc.bad);
    if ((int)(threadIdx.x & 31) == __ffs((int)mask) - 1) {
        atomicMax(a.rate_max, ((unsigned long long)mhi << 32) | mlo);
        if (nbad) atomicAdd(a.bad, (int)nbad);
    }
}


// Finish cell idx (coordinate b along DIR, neighbours sd apart, transverse
// flat index tr or -1): flux difference and alpha div(u) source, or, at a
// characteristic boundary, the boundary rate (from cbc_rates when the caller
// gives tr, else computed here); then store, accumulate or apply the RK stage.
//
// Six-equation model (SIX): NQ rows; the phase energies lose a_k p div(u)
// (cell values), and an RK stage update ends with the pressure relaxation
// (relax6) before it is stored.
//
// stg (y/z stream kernels, or null): this lane's operands staged by
// stage_finish_operands, complete (cp_async_wait_all) before the call.
//
// Fused primitive recovery (FP64 form, five-equation models, RK stage update
// with a.w_next set): the new state of the cell is in registers, so its primitives
// are written to a.w_next (the next stage's sweeps read them there instead of
// a separate recovery pass over q) and, with a.rate_max, its CFL rate is
// returned for the caller's RateAcc (-1: non-physical); otherwise 0.
//
// finish_cell takes the two face fluxes and face velocities; finish_cell_df the
// same in float-float (FP64 path: the flux differences are formed before one
// widening each); both call finish_cell_rates with (F_- - F_+)/dx and the
// face-velocity divergence.
template <typename Real, int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ double finish_cell_rates(const SweepArgs& a, long long idx, Real* out, const Real du,
                                                    const Real* cell, Real inv_dx, int b, long long sd, long long tr,
                                                    const unsigned char* stg, int slot) {
    using Lay = Layout<NF, NDIM, SIX>;
    constexpr int NS = Lay::NS, NQ = Lay::NQ, IA = Lay::IA;
    if constexpr (SIX) {
        const Real pdu = cell[Lay::IE] * du;
        Real aN = 1;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            aN -= cell[IA + k];
            out[Lay::II + k] -= cell[IA + k] * pdu;
        }
        out[Lay::II + NF - 1] -= aN * pdu;
    }
    if constexpr (NF > 1) {
        if (a.kapila) {
            Real K[NF - 1];
            if constexpr (sizeof(Real) == 8) kapila_K_df<NF, NDIM>(a, cell, K);
            else kapila_K<Real, NF, NDIM>(a, cell, K);
#pragma unroll
            for (int k = 0; k < NF - 1; ++k) out[IA + k] = fma(cell[IA + k] + K[k], du, out[IA + k]);
        } else {
#pragma unroll
            for (int k = 0; k < NF - 1; ++k) out[IA + k] = fma(cell[IA + k], du, out[IA + k]);
        }
    }
    if (a.cbc) {
        const int n = a.g.n[DIR];
        const bool lo = b == 0 && a.g.bc_lo[DIR] == BC_CHARACTERISTIC;
        const bool hi = b == n - 1 && a.g.bc_hi[DIR] == BC_CHARACTERISTIC;
        if (lo || hi) {   // the boundary rate replaces the flux difference and the source
            if (a.cbc_rates && tr >= 0) {
                const Real* rb = static_cast<const Real*>(a.cbc_rates) + a.cbc_off[DIR][lo ? 0 : 1] + tr;
                const long long nt = a.g.ncell / n;
#pragma unroll
                for (int v = 0; v < NS; ++v) out[v] = rb[v * nt];
            } else {
                Real cb[NS];
                cbc_cell_rate<Real, NF, NDIM, DIR>(a, idx, sd, n, !lo, inv_dx, cb);
#pragma unroll
                for (int v = 0; v < NS; ++v) out[v] = cb[v];
            }
        }
    }
    const long long nc = a.g.ncell;
    Real* R = static_cast<Real*>(a.R);
    // operand rows: staged (stride kStageSlots) or in global memory (stride nc)
    const Real* pR = R + idx;
    const double *pQs = a.qs + idx, *pQ0 = a.q0 + idx;
    long long sRv = nc, sQsv = nc, sQ0v = nc;
    if (stg) {
        const int m = a.stage;
        if (m & 1) { pR = reinterpret_cast<const Real*>(stg) + slot; sRv = kStageSlots; }
        if (m & 2) { pQs = reinterpret_cast<const double*>(stg + stage_offset_qs<Real, NQ>(m)) + slot; sQsv = kStageSlots; }
        if (m & 4) { pQ0 = reinterpret_cast<const double*>(stg + stage_offset_q0<Real, NQ>(m)) + slot; sQ0v = kStageSlots; }
    }
    auto Rv = [&](int v) -> Real { return pR[v * sRv]; };
    auto qsv = [&](int v) -> double { return pQs[v * sQsv]; };
    auto q0v = [&](int v) -> double { return pQ0[v * sQ0v]; };
    if (a.mode == 0) {
#pragma unroll
        for (int v = 0; v < NQ; ++v) R[v * nc + idx] = out[v];
    } else if (a.mode == 1) {
#pragma unroll
        for (int v = 0; v < NQ; ++v) R[v * nc + idx] = Rv(v) + out[v];
    } else if (a.mode == 2) {
        double qn[NQ];
        // FP32 forms: the increment c1 dt R is formed in FP32 (R is an FP32
        // quantity there) and widened by integer operations, so the FP64
        // accumulation takes one FP64 operation per value, two with the q0
        // term.  FP64 form: c1 (qs + dt R), the product skipped when c1 = 1.
        [[maybe_unused]] float c1dt = 0.f;
        if constexpr (sizeof(Real) == 4) c1dt = narrow_rn(a.c1 * a.dt);
        const bool unit = a.c1 == 1.0;
#pragma unroll
        for (int v = 0; v < NQ; ++v) {
            const Real rv = a.acc_in ? Rv(v) + out[v] : out[v];
            double o;
            if constexpr (sizeof(Real) == 4) {
                o = fma(a.c1, qsv(v), widen_all(c1dt * rv));
            } else {
                o = fma(a.dt, rv, qsv(v));
                if (!unit) o *= a.c1;
            }
            if (a.c0 != 0.0) o = fma(a.c0, q0v(v), o);
            qn[v] = o;
            if constexpr (!SIX) a.qout[v * nc + idx] = o;
        }
        if constexpr (SIX) {
            relax6<NF, NDIM>(a, qn);
#pragma unroll
            for (int v = 0; v < NQ; ++v) a.qout[v * nc + idx] = qn[v];
        } else if constexpr (sizeof(Real) == 8) {
            // FP64 form only: in the FP32 forms' z sweep (memory-bound, 64
            // registers) the fused recovery spilled and cost more than the
            // separate pass it replaced (mixed 6.27 -> 6.52 ms per step at 256^3)
            if (a.w_next) {
                Real wv[NS], c2;
                prims_cell<NF, NDIM>(qn, a.e, wv, c2);
                Real* wn = static_cast<Real*>(a.w_next);
#pragma unroll
                for (int v = 0; v < NS; ++v) wn[v * nc + idx] = wv[v];
                if (a.rate_max) return cell_cfl_rate<Real, NF, NDIM>(wv, c2, a.g, a.grid, a.grid_stride, idx);
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < NQ; ++v) {
            const Real rv = a.acc_in ? Rv(v) + out[v] : out[v];
            a.out[v * nc + idx] = (double)rv;
        }
    }
    return 0.0;
}

template <typename Real, int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ double finish_cell(const SweepArgs& a, long long idx, const Real* Fm, const Real* Fp,
                                              Real um, Real up, const Real* cell, Real inv_dx, int b, long long sd,
                                              long long tr = -1, const unsigned char* stg = nullptr, int slot = 0) {
    constexpr int NQ = Layout<NF, NDIM, SIX>::NQ;
    Real out[NQ];
#pragma unroll
    for (int v = 0; v < NQ; ++v) out[v] = (Fm[v] - Fp[v]) * inv_dx;
    const Real du = (up - um) * inv_dx;
    return finish_cell_rates<Real, NF, NDIM, DIR, SIX>(a, idx, out, du, cell, inv_dx, b, sd, tr, stg, slot);
}

// Five-equation FP64 path with float-float fluxes: the differences and the
// division by dx in float-float (accurate addition: relative error ~2^-47 of
// the difference), one widening per value.
template <int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ double finish_cell_df(const SweepArgs& a, long long idx, const df* Fm, const df* Fp,
                                                 df um, df up, const double* cell, double inv_dx, df inv_df, int b,
                                                 long long sd, long long tr = -1, const unsigned char* stg = nullptr,
                                                 int slot = 0) {
    constexpr int NQ = Layout<NF, NDIM, SIX>::NQ;
    double out[NQ];
#pragma unroll
    for (int v = 0; v < NQ; ++v) out[v] = df_to_double(df_mul(df_add(Fm[v], df_neg(Fp[v])), inv_df));
    const double du = df_to_double(df_mul(df_add(up, df_neg(um)), inv_df));
    return finish_cell_rates<double, NF, NDIM, DIR, SIX>(a, idx, out, du, cell, inv_dx, b, sd, tr, stg, slot);
}

}  // namespace mfc
