/*
 * Plain, slow CPU FP64 oracle for the right-hand side of the five-equation
 * (Allaire) diffuse-interface model with stiffened-gas fluids.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it exists so tests, the smoke check and the CPU baseline can
 * compare the CUDA path against an independent definition.  It shares no code,
 * header, table or constant with the CUDA sources.
 *
 * What it computes (arXiv 2305.09163):
 *   - Model (Sec. 2.1, "5-equation models"): partial densities a_k r_k, mixture
 *     momentum r u, total energy r E and volume fractions a_k, with the Kapila
 *     source K div(u) dropped (the Allaire reduction stated at the end of
 *     Sec. 2.1).  N fluids carry N-1 transported volume fractions; a_N = 1 - sum.
 *   - EOS (Sec. 2.1, Eq. "soe"): stiffened gas.  Mixture closure
 *     r E = Gamma p + Pi + 0.5 r |u|^2, Gamma = sum a_k/(g_k-1),
 *     Pi = sum a_k g_k pinf_k/(g_k-1); sound speed c^2 = ((Gamma+1)p+Pi)/(Gamma r).
 *     With model = 1 the Kapila source is kept instead (the first model of
 *     Sec. 2.1): the volume-fraction rows gain K_k div(u), see oracle_kapila_K.
 *   - Finite volumes (Sec. 3.1, Eqs. "fvm" and "fvmdis"):
 *     dq/dt = sum_d (F_{-1/2} - F_{+1/2})/dx_d - h(q) div(u), with h = -a_k in the
 *     volume-fraction rows and div(u) from face velocities (Sec. 3.1, last eq.).
 *   - Reconstruction (Sec. 3.2): WENO5-JS on the primitive variables
 *     (a_k r_k, u, p, a_k), one variable at a time, textbook Jiang-Shu
 *     candidates, smoothness indicators and ideal weights (0.1, 0.6, 0.3);
 *     or, with weno_order = 3, the third-order variant the section also
 *     names (k = 2 candidates of two cells, ideal weights (1/3, 2/3),
 *     smoothness indicators the squared one-sided differences).
 *   - Riemann solver (Sec. 3.2.1): HLLC, Davis wave-speed estimates, star states
 *     with continuity of normal velocity and pressure, four-branch flux.
 *     Face velocity = HLLC flux of a volume fraction divided by that fraction.
 *   - Grid (Sec. 4.1): uniform, or non-uniform per direction with WENO5
 *     coefficient tables (candidates, ideal weights, smoothness-indicator
 *     quadratic forms per cell, as Listing 1's per-index tables) built by
 *     oracle/nonuniform.py from the definitions.
 *   - Boundaries (Sec. 3.3): ghost cells three deep (WENO5 order); periodic,
 *     transmissive (copy of the nearest interior cell) and reflective (mirror,
 *     normal momentum negated); and characteristic (bc 3, Sec. 3.3's
 *     characteristic-based conditions after Thompson): stencils see
 *     transmissive ghosts, and the boundary cell's normal contribution comes
 *     from the characteristic amplitudes with the incoming ones set to zero
 *     (oracle_cbc_normal).
 *
 *   - With model = 2, the six-equation model with pressure relaxation (Sec. 2.3,
 *     after Saurel, Petitpas & Berry 2009 and Schmidmayer et al. 2020): each
 *     phase also carries its internal energy a_k r_k e_k, obeying
 *     d(a_k r_k e_k)/dt + div(a_k r_k e_k u) + a_k p_k div(u) = 0, and waves
 *     travel at the frozen sound speed, r c^2 = sum a_k g_k (p_k + pinf_k).
 *     After every Runge-Kutta stage the state is relaxed to one pressure with
 *     infinite stiffness (oracle_relax6), so the right-hand side always acts
 *     on states with p_k = p: it takes p from the total energy and the mixture
 *     law (as the five-equation model does), the phase energies at the faces
 *     as a_k (p + g_k pinf_k)/(g_k - 1), and the work term as a_k p div(u).
 *     The primitive vector carries, after the five-equation variables, the
 *     phase pressures (g_k - 1) a_k r_k e_k / a_k - g_k pinf_k of the state
 *     (informative; the right-hand side does not read them).
 *
 * Optional first-order fallback (Sec. 3.2, first-order reconstruction): when a
 * reconstructed face state has a negative partial density, a volume fraction
 * outside [0,1] or (Gamma+1)p+Pi <= 0, both sides of that face use the cell
 * values instead.  Off unless params->fallback is set.
 *
 * Built with -O2 -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXF 3             /* fluids */
#define OR_MAXV (3 * OR_MAXF + 3) /* conserved variables (six-equation model) */

typedef struct {
    int n[3];          /* cells per direction; 1 for an inactive direction */
    int ndim;          /* 1, 2 or 3: directions 0..ndim-1 are active */
    int nf;            /* number of fluids, 1..3 */
    double dx[3];      /* uniform cell widths */
    int bc[6];         /* -x,+x,-y,+y,-z,+z: 0 periodic, 1 transmissive, 2 reflective */
    double gamma[OR_MAXF];
    double pi_inf[OR_MAXF];
    double eps;        /* WENO epsilon */
    int fallback;      /* first-order fallback at non-physical faces */
    int weno_order;    /* 5 (default) or 3 */
    int model;         /* 0: Allaire (K = 0); 1: Kapila (K div u in the alpha rows);
                          2: six-equation (phase internal energies; relaxation between stages) */
    const double *tab[3]; /* non-uniform grid: per-direction WENO5 tables (NULL: uniform) */
} oracle_params;

/* Layout of one table row (cell c of a direction, rows for c = -1..n), written
 * by oracle/nonuniform.py from the definitions of the finite-volume WENO5
 * construction: candidate values at c+1/2 and c-1/2 over the five-cell
 * stencil, ideal weights of both edges, the smoothness-indicator quadratic
 * forms over each candidate's three cells, and 1/dx_c. */
#define TAB_CL 0
#define TAB_CR 15
#define TAB_DL 30
#define TAB_DR 33
#define TAB_B 36
#define TAB_IDX 63
#define TAB_ROW 64

static const double *tab_row(const oracle_params *P, int d, int c) { return P->tab[d] + (long)(c + 1) * TAB_ROW; }

/* WENO5-JS value at one edge of cell c from a table row (side 0: c+1/2,
 * side 1: c-1/2); st = the five cell values c-2..c+2.  The candidates'
 * coefficients sum to one and the smoothness indicators vanish on constants
 * (they measure derivatives), so both are evaluated on the values relative to
 * the cell value v_c: the same numbers, without the cancellation a quadratic
 * form of raw values suffers when |v| is large and its variation small. */
static double weno5_table(const double *row, int side, const double *st, double eps) {
    const double *cand = row + (side ? TAB_CR : TAB_CL);
    const double *dd = row + (side ? TAB_DR : TAB_DL);
    double rel[5];
    for (int j = 0; j < 5; ++j) rel[j] = st[j] - st[2];
    double a[3], p[3], s = 0.0;
    for (int r = 0; r < 3; ++r) {
        p[r] = 0.0;
        for (int j = 0; j < 5; ++j) p[r] += cand[5 * r + j] * rel[j];
        const double *B = row + TAB_B + 9 * r;
        double b = 0.0;
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) b += B[3 * j + k] * rel[r + j] * rel[r + k];
        a[r] = dd[r] / ((eps + b) * (eps + b));
        s += a[r];
    }
    return st[2] + (a[0] * p[0] + a[1] * p[1] + a[2] * p[2]) / s;
}

/* ---- variable indexing (conserved and primitive share positions) ----
 * a_k r_k (N), r u or u (ndim), r E or p (1), a_k (N-1); the six-equation model
 * appends a_k r_k e_k or p_k (N). */
static int six(const oracle_params *P) { return P->model == 2; }
static int sys_size(const oracle_params *P) { return (six(P) ? 3 : 2) * P->nf + P->ndim; }
static int i_mom(const oracle_params *P, int d) { return P->nf + d; }
static int i_E(const oracle_params *P) { return P->nf + P->ndim; }
static int i_alpha(const oracle_params *P, int k) { return P->nf + P->ndim + 1 + k; }
static int i_int(const oracle_params *P, int k) { return 2 * P->nf + P->ndim + k; }

int oracle_sys_size(const oracle_params *P) { return sys_size(P); }

/* Volume fractions of all N fluids from the N-1 transported ones. */
static void all_alphas(const oracle_params *P, const double *v, double *a) {
    double s = 0.0;
    for (int k = 0; k < P->nf - 1; ++k) { a[k] = v[i_alpha(P, k)]; s += a[k]; }
    a[P->nf - 1] = 1.0 - s;
}

/* Mixture Gamma = sum a_k/(g_k-1) and Pi = sum a_k g_k pinf_k/(g_k-1). */
static void mixture(const oracle_params *P, const double *v, double *Gam, double *Pi) {
    double a[OR_MAXF];
    all_alphas(P, v, a);
    double G = 0.0, Q = 0.0;
    for (int k = 0; k < P->nf; ++k) {
        G += a[k] / (P->gamma[k] - 1.0);
        Q += a[k] * P->gamma[k] * P->pi_inf[k] / (P->gamma[k] - 1.0);
    }
    *Gam = G; *Pi = Q;
}

/* ---- Kapila source coefficient (Sec. 2.1, 5-equation models) ----
 * d(alpha_k)/dt + u . grad(alpha_k) = K_k div(u).  For two components the
 * section gives K = (r2 c2^2 - r1 c1^2) / (r2 c2^2/a2 + r1 c1^2/a1) (its second
 * term is printed with c2 where c1 belongs).  For N components the model of
 * Kapila et al. (the section's reference) has
 *     K_k = a_k (r c_W^2 / (r_k c_k^2) - 1),  1/(r c_W^2) = sum_j a_j / (r_j c_j^2),
 * c_W the Wood mixture sound speed; for N = 2 this is the printed form.  For a
 * stiffened gas r_k c_k^2 = g_k (p + pinf_k).  w is a primitive cell state;
 * K receives the N-1 coefficients of the transported fractions.
 */
void oracle_kapila_K(const oracle_params *P, const double *w, double *K) {
    double a[OR_MAXF], Z[OR_MAXF];
    all_alphas(P, w, a);
    double p = w[P->nf + P->ndim];
    double s = 0.0;
    for (int k = 0; k < P->nf; ++k) {
        Z[k] = P->gamma[k] * (p + P->pi_inf[k]);
        s += a[k] / Z[k];
    }
    double rcw2 = 1.0 / s;
    for (int k = 0; k < P->nf - 1; ++k) K[k] = a[k] * (rcw2 / Z[k] - 1.0);
}

static double density(const oracle_params *P, const double *v) {
    double r = 0.0;
    for (int k = 0; k < P->nf; ++k) r += v[k];
    return r;
}

/* Conserved -> primitive for one cell (EOS solved for p). */
void oracle_cons_to_prim(const oracle_params *P, const double *q, double *w) {
    int ns = sys_size(P);
    double r = density(P, q);
    double ke = 0.0;
    for (int k = 0; k < ns; ++k) w[k] = q[k];
    for (int d = 0; d < P->ndim; ++d) {
        double u = q[i_mom(P, d)] / r;
        w[i_mom(P, d)] = u;
        ke += 0.5 * r * u * u;
    }
    double G, Q;
    mixture(P, q, &G, &Q);
    w[i_E(P)] = (q[i_E(P)] - ke - Q) / G;
    if (six(P)) {   /* phase pressures from the internal energies */
        double a[OR_MAXF];
        all_alphas(P, q, a);
        for (int k = 0; k < P->nf; ++k)
            w[i_int(P, k)] = (P->gamma[k] - 1.0) * q[i_int(P, k)] / a[k] - P->gamma[k] * P->pi_inf[k];
    }
}

/* Primitive -> conserved for one cell. */
void oracle_prim_to_cons(const oracle_params *P, const double *w, double *q) {
    int ns = sys_size(P);
    double r = density(P, w);
    double ke = 0.0;
    for (int k = 0; k < ns; ++k) q[k] = w[k];
    for (int d = 0; d < P->ndim; ++d) {
        double u = w[i_mom(P, d)];
        q[i_mom(P, d)] = r * u;
        ke += 0.5 * r * u * u;
    }
    if (six(P)) {   /* a_k r_k e_k = a_k (p_k + g_k pinf_k)/(g_k - 1); r E = sum + kinetic */
        double a[OR_MAXF], e = 0.0;
        all_alphas(P, w, a);
        for (int k = 0; k < P->nf; ++k) {
            q[i_int(P, k)] = a[k] * (w[i_int(P, k)] + P->gamma[k] * P->pi_inf[k]) / (P->gamma[k] - 1.0);
            e += q[i_int(P, k)];
        }
        q[i_E(P)] = e + ke;
        return;
    }
    double G, Q;
    mixture(P, w, &G, &Q);
    q[i_E(P)] = G * w[i_E(P)] + Q + ke;
}

void oracle_prim_to_cons_array(const oracle_params *P, const double *w, double *q, long ncell) {
    int ns = sys_size(P);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < ncell; ++c) {
        double wc[OR_MAXV], qc[OR_MAXV];
        for (int v = 0; v < ns; ++v) wc[v] = w[(long)v * ncell + c];
        oracle_prim_to_cons(P, wc, qc);
        for (int v = 0; v < ns; ++v) q[(long)v * ncell + c] = qc[v];
    }
}

void oracle_cons_to_prim_array(const oracle_params *P, const double *q, double *w, long ncell) {
    int ns = sys_size(P);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < ncell; ++c) {
        double wc[OR_MAXV], qc[OR_MAXV];
        for (int v = 0; v < ns; ++v) qc[v] = q[(long)v * ncell + c];
        oracle_cons_to_prim(P, qc, wc);
        for (int v = 0; v < ns; ++v) w[(long)v * ncell + c] = wc[v];
    }
}

/* Squared sound speed ((Gamma+1)p + Pi)/(Gamma rho) of a primitive state;
 * six-equation model: the frozen sound speed sum a_k g_k (p + pinf_k) / rho of
 * the phases at the mixture pressure. */
static double sound_speed_sq(const oracle_params *P, const double *w) {
    if (six(P)) {
        double a[OR_MAXF], s = 0.0;
        all_alphas(P, w, a);
        for (int k = 0; k < P->nf; ++k) s += a[k] * P->gamma[k] * (w[i_E(P)] + P->pi_inf[k]);
        return s / density(P, w);
    }
    double G, Q;
    mixture(P, w, &G, &Q);
    return ((G + 1.0) * w[i_E(P)] + Q) / (G * density(P, w));
}

/* ---- WENO5-JS (Jiang & Shu 1996; Sec. 3.2) ----
 * v[0..4] = values of cells i-2..i+2; returns the left-biased value at i+1/2.
 * The value at i-1/2 seen from cell i is the same call on the reversed stencil.
 */
void oracle_weno5_weights(const double *v, double eps, double *omega, double *cand) {
    double p0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
    double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
    double p2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
    double t;
    double b0, b1, b2;
    t = v[0] - 2.0 * v[1] + v[2];
    b0 = 13.0 / 12.0 * t * t;
    t = v[0] - 4.0 * v[1] + 3.0 * v[2];
    b0 += 0.25 * t * t;
    t = v[1] - 2.0 * v[2] + v[3];
    b1 = 13.0 / 12.0 * t * t;
    t = v[1] - v[3];
    b1 += 0.25 * t * t;
    t = v[2] - 2.0 * v[3] + v[4];
    b2 = 13.0 / 12.0 * t * t;
    t = 3.0 * v[2] - 4.0 * v[3] + v[4];
    b2 += 0.25 * t * t;
    double a0 = 0.1 / ((eps + b0) * (eps + b0));
    double a1 = 0.6 / ((eps + b1) * (eps + b1));
    double a2 = 0.3 / ((eps + b2) * (eps + b2));
    double s = a0 + a1 + a2;
    omega[0] = a0 / s; omega[1] = a1 / s; omega[2] = a2 / s;
    if (cand) { cand[0] = p0; cand[1] = p1; cand[2] = p2; }
}

double oracle_weno5(const double *v, double eps) {
    double om[3], c[3];
    oracle_weno5_weights(v, eps, om, c);
    return om[0] * c[0] + om[1] * c[1] + om[2] * c[2];
}

/* Smoothness indicators alone (for tests against their integral definition). */
void oracle_weno5_beta(const double *v, double *beta) {
    double t;
    t = v[0] - 2.0 * v[1] + v[2]; beta[0] = 13.0 / 12.0 * t * t;
    t = v[0] - 4.0 * v[1] + 3.0 * v[2]; beta[0] += 0.25 * t * t;
    t = v[1] - 2.0 * v[2] + v[3]; beta[1] = 13.0 / 12.0 * t * t;
    t = v[1] - v[3]; beta[1] += 0.25 * t * t;
    t = v[2] - 2.0 * v[3] + v[4]; beta[2] = 13.0 / 12.0 * t * t;
    t = 3.0 * v[2] - 4.0 * v[3] + v[4]; beta[2] += 0.25 * t * t;
}

/* ---- WENO3-JS (Sec. 3.2, the third-order variant: (2k-1)th order with k = 2) ----
 * v[0..2] = values of cells i-1..i+1; returns the left-biased value at i+1/2.
 * Candidates: the linear interpolants of cells (i-1, i) and (i, i+1) at
 * i+1/2; ideal weights 1/3 and 2/3 (their combination is the third-order
 * interpolant of the three cells); smoothness indicators the squares of the
 * candidates' differences.  The value at i-1/2 is the same call on the
 * reversed stencil.
 */
void oracle_weno3_weights(const double *v, double eps, double *omega, double *cand) {
    double p0 = -0.5 * v[0] + 1.5 * v[1];
    double p1 = 0.5 * v[1] + 0.5 * v[2];
    double b0 = (v[1] - v[0]) * (v[1] - v[0]);
    double b1 = (v[2] - v[1]) * (v[2] - v[1]);
    double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
    double a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
    double s = a0 + a1;
    omega[0] = a0 / s; omega[1] = a1 / s;
    if (cand) { cand[0] = p0; cand[1] = p1; }
}

double oracle_weno3(const double *v, double eps) {
    double om[2], c[2];
    oracle_weno3_weights(v, eps, om, c);
    return om[0] * c[0] + om[1] * c[1];
}

/* ---- physical flux in direction d of a primitive state (Sec. 2.1 equations) ---- */
static void physical_flux(const oracle_params *P, int d, const double *w, double *F) {
    int ns = sys_size(P);
    double r = density(P, w);
    double un = w[i_mom(P, d)];
    double p = w[i_E(P)];
    double q[OR_MAXV];
    oracle_prim_to_cons(P, w, q);
    double rE = q[i_E(P)];
    for (int k = 0; k < P->nf; ++k) F[k] = w[k] * un;
    for (int e = 0; e < P->ndim; ++e) F[i_mom(P, e)] = r * w[i_mom(P, e)] * un;
    F[i_mom(P, d)] += p;
    F[i_E(P)] = (rE + p) * un;
    for (int k = 0; k < P->nf - 1; ++k) F[i_alpha(P, k)] = w[i_alpha(P, k)] * un;
    if (six(P))
        for (int k = 0; k < P->nf; ++k) F[i_int(P, k)] = q[i_int(P, k)] * un;
    (void)ns;
}

/* Conserved vector of a primitive state (local helper for the star states). */
static void cons_of(const oracle_params *P, const double *w, double *q) {
    oracle_prim_to_cons(P, w, q);
}

/* HLLC star state q*_K (Sec. 3.2.1): continuity of u_n and p across s*. */
static void star_state(const oracle_params *P, int d, const double *w, double sK, double ss,
                       double *qs) {
    int ns = sys_size(P);
    double q[OR_MAXV];
    cons_of(P, w, q);
    double r = density(P, w);
    double un = w[i_mom(P, d)];
    double p = w[i_E(P)];
    double xi = (sK - un) / (sK - ss);
    for (int k = 0; k < P->nf; ++k) qs[k] = xi * w[k];
    for (int e = 0; e < P->ndim; ++e) qs[i_mom(P, e)] = xi * r * w[i_mom(P, e)];
    qs[i_mom(P, d)] = xi * r * ss;
    qs[i_E(P)] = xi * (q[i_E(P)] + (ss - un) * (r * ss + p / (sK - un)));
    for (int k = 0; k < P->nf - 1; ++k) qs[i_alpha(P, k)] = xi * w[i_alpha(P, k)];
    if (six(P))   /* internal energies: advected with the mass, as the partial densities */
        for (int k = 0; k < P->nf; ++k) qs[i_int(P, k)] = xi * q[i_int(P, k)];
    (void)ns;
}

/* HLLC flux F and face velocity ut between primitive states wL | wR, normal d. */
void oracle_hllc(const oracle_params *P, int d, const double *wL, const double *wR,
                 double *F, double *ut) {
    int ns = sys_size(P);
    double rL = density(P, wL), rR = density(P, wR);
    double uL = wL[i_mom(P, d)], uR = wR[i_mom(P, d)];
    double pL = wL[i_E(P)], pR = wR[i_E(P)];
    double cL = sqrt(sound_speed_sq(P, wL));
    double cR = sqrt(sound_speed_sq(P, wR));
    /* Davis direct wave-speed estimates */
    double sL = fmin(uL - cL, uR - cR);
    double sR = fmax(uL + cL, uR + cR);
    double ss = (pR - pL + rL * uL * (sL - uL) - rR * uR * (sR - uR)) /
                (rL * (sL - uL) - rR * (sR - uR));
    if (0.0 <= sL) {
        physical_flux(P, d, wL, F);
        *ut = uL;
    } else if (0.0 <= ss) {
        double FL[OR_MAXV], qL[OR_MAXV], qs[OR_MAXV];
        physical_flux(P, d, wL, FL);
        cons_of(P, wL, qL);
        star_state(P, d, wL, sL, ss, qs);
        for (int v = 0; v < ns; ++v) F[v] = FL[v] + sL * (qs[v] - qL[v]);
        *ut = uL + sL * ((sL - uL) / (sL - ss) - 1.0);
    } else if (0.0 < sR) {
        double FR[OR_MAXV], qR[OR_MAXV], qs[OR_MAXV];
        physical_flux(P, d, wR, FR);
        cons_of(P, wR, qR);
        star_state(P, d, wR, sR, ss, qs);
        for (int v = 0; v < ns; ++v) F[v] = FR[v] + sR * (qs[v] - qR[v]);
        *ut = uR + sR * ((sR - uR) / (sR - ss) - 1.0);
    } else {
        physical_flux(P, d, wR, F);
        *ut = uR;
    }
}

/* ---- ghost cells by index mapping (Sec. 3.3) ---- */
/* Fetch the conserved vector of cell (i,j,k); indices may lie in the ghost
 * layers of at most one direction. */
static void fetch_cell(const oracle_params *P, const double *q, int idx[3], double *qc) {
    int ns = sys_size(P);
    int flip = -1;
    int ii[3] = {idx[0], idx[1], idx[2]};
    for (int d = 0; d < 3; ++d) {
        int n = P->n[d];
        if (ii[d] < 0) {
            int bc = P->bc[2 * d];
            if (bc == 0) ii[d] += n;
            else if (bc == 1 || bc == 3) ii[d] = 0;
            else { ii[d] = -ii[d] - 1; flip = d; }
        } else if (ii[d] >= n) {
            int bc = P->bc[2 * d + 1];
            if (bc == 0) ii[d] -= n;
            else if (bc == 1 || bc == 3) ii[d] = n - 1;
            else { ii[d] = 2 * n - 1 - ii[d]; flip = d; }
        }
    }
    long ncell = (long)P->n[0] * P->n[1] * P->n[2];
    long c = ((long)ii[2] * P->n[1] + ii[1]) * P->n[0] + ii[0];
    for (int v = 0; v < ns; ++v) qc[v] = q[(long)v * ncell + c];
    if (flip >= 0) qc[i_mom(P, flip)] = -qc[i_mom(P, flip)];
}

static int face_state_ok(const oracle_params *P, const double *w) {
    for (int k = 0; k < P->nf; ++k)
        if (!(w[k] >= 0.0)) return 0;
    double a[OR_MAXF];
    all_alphas(P, w, a);
    for (int k = 0; k < P->nf; ++k)
        if (!(a[k] >= 0.0 && a[k] <= 1.0)) return 0;
    if (!(density(P, w) > 0.0)) return 0;
    if (six(P)) return sound_speed_sq(P, w) > 0.0;
    double G, Q;
    mixture(P, w, &G, &Q);
    if (!((G + 1.0) * w[i_E(P)] + Q > 0.0)) return 0;
    return 1;
}

/* ---- characteristic boundary (Sec. 3.3, Thompson's characteristic-based
 * conditions), non-reflecting ----
 * Normal part of dq/dt at a boundary cell from the quasi-linear form of the
 * model in primitive variables along d (Sec. 2.1, Allaire):
 *   (a_k r_k)_t + u (a_k r_k)_x + a_k r_k u_x = 0,  u_t + u u_x + p_x / r = 0,
 *   (u_tan)_t + u (u_tan)_x = 0,  p_t + u p_x + r c^2 u_x = 0,  a_t + u a_x = 0,
 * c^2 = ((Gamma+1) p + Pi)/(Gamma r), written with the wave amplitudes
 *   L1 = (u - c)(p_x - r c u_x),  L5 = (u + c)(p_x + r c u_x),
 *   Lk = u ((a_k r_k)_x - a_k r_k p_x/(r c^2)),  Lt = u (u_tan)_x,  La = u a_x,
 * as p_t = -(L5 + L1)/2, u_t = -(L5 - L1)/(2 r c), (a_k r_k)_t = -Lk - a_k r_k
 * (L5 + L1)/(2 r c^2), (u_tan)_t = -Lt, a_t = -La.  Amplitudes of waves that
 * enter the domain (speed > 0 at the low boundary, < 0 at the high one) are
 * set to zero; the others use the one-sided difference between the boundary
 * cell (qb) and its interior neighbour (qn), h the boundary cell's width.  The
 * primitive rates are then turned into conserved ones. */
void oracle_cbc_normal(const oracle_params *P, int d, int high, const double *qb, const double *qn, double h,
                       double *out) {
    int ns = sys_size(P), nf = P->nf, nd = P->ndim;
    double wb[OR_MAXV], wn[OR_MAXV], wx[OR_MAXV], wt[OR_MAXV];
    oracle_cons_to_prim(P, qb, wb);
    oracle_cons_to_prim(P, qn, wn);
    for (int v = 0; v < ns; ++v) wx[v] = high ? (wb[v] - wn[v]) / h : (wn[v] - wb[v]) / h;
    double r = density(P, wb), c = sqrt(sound_speed_sq(P, wb));
    double u = wb[i_mom(P, d)], p = wb[i_E(P)];
    double ux = wx[i_mom(P, d)], px = wx[i_E(P)];
    double lam1 = u - c, lam5 = u + c;
    int in1 = high ? lam1 < 0.0 : lam1 > 0.0;
    int in5 = high ? lam5 < 0.0 : lam5 > 0.0;
    int inu = high ? u < 0.0 : u > 0.0;
    double L1 = in1 ? 0.0 : lam1 * (px - r * c * ux);
    double L5 = in5 ? 0.0 : lam5 * (px + r * c * ux);
    for (int k = 0; k < nf; ++k) {
        double Lk = inu ? 0.0 : u * (wx[k] - wb[k] * px / (r * c * c));
        wt[k] = -Lk - wb[k] * (L5 + L1) / (2.0 * r * c * c);
    }
    for (int e = 0; e < nd; ++e) {
        if (e == d) wt[i_mom(P, e)] = -(L5 - L1) / (2.0 * r * c);
        else wt[i_mom(P, e)] = inu ? 0.0 : -u * wx[i_mom(P, e)];
    }
    wt[i_E(P)] = -0.5 * (L5 + L1);
    for (int a = 0; a < nf - 1; ++a) wt[i_alpha(P, a)] = inu ? 0.0 : -u * wx[i_alpha(P, a)];
    /* primitive rates -> conserved rates */
    double rt = 0.0;
    for (int k = 0; k < nf; ++k) { out[k] = wt[k]; rt += wt[k]; }
    double ke = 0.0, kt = 0.0;
    for (int e = 0; e < nd; ++e) {
        double ue = wb[i_mom(P, e)];
        out[i_mom(P, e)] = ue * rt + r * wt[i_mom(P, e)];
        ke += 0.5 * ue * ue;
        kt += ue * wt[i_mom(P, e)];
    }
    double G, Q, Gt = 0.0, Pt = 0.0;
    mixture(P, wb, &G, &Q);
    double GN = 1.0 / (P->gamma[nf - 1] - 1.0), PN = P->gamma[nf - 1] * P->pi_inf[nf - 1] / (P->gamma[nf - 1] - 1.0);
    for (int a = 0; a < nf - 1; ++a) {
        double Ga = 1.0 / (P->gamma[a] - 1.0), Pa = P->gamma[a] * P->pi_inf[a] / (P->gamma[a] - 1.0);
        Gt += (Ga - GN) * wt[i_alpha(P, a)];
        Pt += (Pa - PN) * wt[i_alpha(P, a)];
        out[i_alpha(P, a)] = wt[i_alpha(P, a)];
    }
    out[i_E(P)] = G * wt[i_E(P)] + p * Gt + Pt + ke * rt + r * kt;
}

/* ---- six-equation model (Sec. 2.3) ---- */
/* a_k p of cell c (the coefficient of div(u) in the internal-energy rows). */
static void six_work(const oracle_params *P, const double *q, long ncell, long c, double *src) {
    double qc[OR_MAXV], wc[OR_MAXV], a[OR_MAXF];
    for (int v = 0; v < sys_size(P); ++v) qc[v] = q[(long)v * ncell + c];
    oracle_cons_to_prim(P, qc, wc);
    all_alphas(P, wc, a);
    for (int k = 0; k < P->nf; ++k) src[k] = a[k] * wc[i_E(P)];
}

/* Volume fraction of phase k after relaxing to pressure p with infinite
 * stiffness: at fixed mass the phase energy follows de_k = -p dv_k with the
 * interfacial pressure taken as the final p, which for a stiffened gas,
 * a_k r_k e_k = a_k (p + g_k pinf_k)/(g_k - 1), integrates to
 *   a_k (p + g_k pinf_k)/(g_k - 1) - E_k0 = -p (a_k - a_k0),
 *   a_k(p) = (g_k - 1)(E_k0 + a_k0 p) / (g_k (p + pinf_k)),
 * E_k0 = a_k r_k e_k before the relaxation. */
static double relaxed_alpha(const oracle_params *P, int k, double a0, double E0, double p) {
    double g = P->gamma[k], pi = P->pi_inf[k];
    return (g - 1.0) * (E0 + a0 * p) / (g * (p + pi));
}

/* Pressure relaxation of one conserved cell state, in place (Sec. 2.3: the
 * hyperbolic step is followed by relaxation to pressure equilibrium with
 * infinite stiffness; Saurel, Petitpas & Berry 2009, Schmidmayer et al. 2020).
 *  1. the phases that take part are those with a_k0 > 0 and a positive
 *     p_k0 + pinf_k (E_k0 > a_k0 pinf_k); the others (traces that transport
 *     has driven to or below zero) keep their volume fraction;
 *  2. the relaxed pressure p^ solves sum_{taking part} a_k(p^) = 1 - sum_{others}
 *     a_k0 (relaxed_alpha).  Each a_k(p) of a phase taking part falls strictly
 *     on p > -min pinf (over those phases), so the left side falls from +inf
 *     to below the right side; the root is unique and is found by bisection
 *     to the last bit;
 *  3. the volume fractions of the phases taking part become a_k(p^);
 *  4. the pressure is recomputed from the conserved total energy with the
 *     mixture law of the new fractions, p = (r E - r|u|^2/2 - Pi)/Gamma, and
 *     every phase's internal energy is reset to that pressure.
 * Returns p^ (NaN if no phase can take part). */
double oracle_relax6(const oracle_params *P, double *q) {
    int nf = P->nf;
    double a0[OR_MAXF], E0[OR_MAXF];
    int in[OR_MAXF], nin = 0;
    all_alphas(P, q, a0);
    double pimin = 0.0, pmax = 0.0, target = 1.0;
    for (int k = 0; k < nf; ++k) {
        E0[k] = q[i_int(P, k)];
        in[k] = a0[k] > 0.0 && E0[k] > a0[k] * P->pi_inf[k];
        if (!in[k]) {
            target -= a0[k];
            continue;
        }
        if (nin == 0 || P->pi_inf[k] < pimin) pimin = P->pi_inf[k];
        double pk = (P->gamma[k] - 1.0) * E0[k] / a0[k] - P->gamma[k] * P->pi_inf[k];
        if (pk > pmax) pmax = pk;
        nin += 1;
    }
    if (nin == 0) return NAN;
    double lo = -pimin, hi = pmax + 1.0;
    for (int it = 0; it < 2100; ++it) {   /* upper end of the bracket */
        double s = 0.0;
        for (int k = 0; k < nf; ++k)
            if (in[k]) s += relaxed_alpha(P, k, a0[k], E0[k], hi);
        if (s < target) break;
        hi = 2.0 * hi + 1.0;
    }
    for (int it = 0; it < 2100; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double s = 0.0;
        for (int k = 0; k < nf; ++k)
            if (in[k]) s += relaxed_alpha(P, k, a0[k], E0[k], mid);
        if (s > target) lo = mid;
        else hi = mid;
    }
    double ph = 0.5 * (lo + hi);
    for (int k = 0; k < nf - 1; ++k)
        if (in[k]) q[i_alpha(P, k)] = relaxed_alpha(P, k, a0[k], E0[k], ph);
    double a[OR_MAXF], G = 0.0, Q = 0.0;
    all_alphas(P, q, a);
    for (int k = 0; k < nf; ++k) {
        G += a[k] / (P->gamma[k] - 1.0);
        Q += a[k] * P->gamma[k] * P->pi_inf[k] / (P->gamma[k] - 1.0);
    }
    double r = density(P, q), ke = 0.0;
    for (int d = 0; d < P->ndim; ++d) ke += 0.5 * q[i_mom(P, d)] * q[i_mom(P, d)] / r;
    double p = (q[i_E(P)] - ke - Q) / G;
    for (int k = 0; k < nf; ++k)
        q[i_int(P, k)] = a[k] * (p + P->gamma[k] * P->pi_inf[k]) / (P->gamma[k] - 1.0);
    return ph;
}

/* oracle_relax6 on every cell; returns the number of cells that could not be relaxed. */
long oracle_relax6_array(const oracle_params *P, double *q, long ncell) {
    int ns = sys_size(P);
    long bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long c = 0; c < ncell; ++c) {
        double qc[OR_MAXV];
        for (int v = 0; v < ns; ++v) qc[v] = q[(long)v * ncell + c];
        if (isnan(oracle_relax6(P, qc))) { bad += 1; continue; }
        for (int v = 0; v < ns; ++v) q[(long)v * ncell + c] = qc[v];
    }
    return bad;
}

/* Flux through the face on the low side of cell (i,j,k) in direction d, i.e.
 * between cells idx - e_d and idx.  Returns 1 if the first-order fallback was
 * used at this face. */
int oracle_face(const oracle_params *P, const double *q, int d, int i, int j, int k,
                double *F, double *ut) {
    int ns = sys_size(P);
    double w[6][OR_MAXV];
    for (int s = 0; s < 6; ++s) {
        int idx[3] = {i, j, k};
        idx[d] += s - 3; /* cells -3..+2 relative to the face's high side */
        double qc[OR_MAXV];
        fetch_cell(P, q, idx, qc);
        oracle_cons_to_prim(P, qc, w[s]);
    }
    double wL[OR_MAXV], wR[OR_MAXV];
    for (int v = 0; v < ns; ++v) {
        double st[5];
        if (P->weno_order == 3) {
            for (int s = 0; s < 3; ++s) st[s] = w[1 + s][v];   /* cells -2..0, centre -1 */
            wL[v] = oracle_weno3(st, P->eps);
            for (int s = 0; s < 3; ++s) st[s] = w[4 - s][v];   /* cells +1..-1, centre 0 */
            wR[v] = oracle_weno3(st, P->eps);
        } else if (P->tab[d]) {
            /* non-uniform grid: the tables of the two cells next to the face */
            for (int s = 0; s < 5; ++s) st[s] = w[s][v];       /* cells -3..+1, centre -1 */
            wL[v] = weno5_table(tab_row(P, d, (d == 0 ? i : d == 1 ? j : k) - 1), 0, st, P->eps);
            for (int s = 0; s < 5; ++s) st[s] = w[1 + s][v];   /* cells -2..+2, centre 0 */
            wR[v] = weno5_table(tab_row(P, d, d == 0 ? i : d == 1 ? j : k), 1, st, P->eps);
        } else {
            for (int s = 0; s < 5; ++s) st[s] = w[s][v];       /* cells -3..+1, centre -1 */
            wL[v] = oracle_weno5(st, P->eps);
            for (int s = 0; s < 5; ++s) st[s] = w[5 - s][v];   /* cells +2..-2, centre 0 */
            wR[v] = oracle_weno5(st, P->eps);
        }
    }
    if (six(P))   /* phases at the face pressure: the state is relaxed */
        for (int k = 0; k < P->nf; ++k) {
            wL[i_int(P, k)] = wL[i_E(P)];
            wR[i_int(P, k)] = wR[i_E(P)];
        }
    int fb = 0;
    if (P->fallback && !(face_state_ok(P, wL) && face_state_ok(P, wR))) {
        for (int v = 0; v < ns; ++v) { wL[v] = w[2][v]; wR[v] = w[3][v]; }
        if (six(P))
            for (int k = 0; k < P->nf; ++k) {
                wL[i_int(P, k)] = wL[i_E(P)];
                wR[i_int(P, k)] = wR[i_E(P)];
            }
        fb = 1;
    }
    oracle_hllc(P, d, wL, wR, F, ut);
    return fb;
}

/* Full right-hand side R(q), Eq. "fvmdis".  Also returns, per variable, the
 * largest |F| over all faces (a scale for relative error measures), and the
 * number of faces that used the first-order fallback. */
long oracle_rhs(const oracle_params *P, const double *q, double *rhs, double *fmax) {
    int ns = sys_size(P);
    int nx = P->n[0], ny = P->n[1], nz = P->n[2];
    long ncell = (long)nx * ny * nz;
    long nfb = 0;
    for (int v = 0; v < ns; ++v) fmax[v] = 0.0;
    memset(rhs, 0, sizeof(double) * (size_t)ns * (size_t)ncell);
    for (int d = 0; d < P->ndim; ++d) {
        int m[3] = {nx, ny, nz};
        m[d] += 1; /* faces along d */
        long nface = (long)m[0] * m[1] * m[2];
        double *Ff = (double *)malloc(sizeof(double) * (size_t)(ns + 1) * (size_t)nface);
#pragma omp parallel for schedule(static) reduction(+ : nfb)
        for (long f = 0; f < nface; ++f) {
            int i = (int)(f % m[0]);
            int j = (int)((f / m[0]) % m[1]);
            int k = (int)(f / ((long)m[0] * m[1]));
            double F[OR_MAXV], ut;
            nfb += oracle_face(P, q, d, i, j, k, F, &ut);
            for (int v = 0; v < ns; ++v) Ff[(long)v * nface + f] = F[v];
            Ff[(long)ns * nface + f] = ut;
        }
        for (int v = 0; v < ns; ++v)
            for (long f = 0; f < nface; ++f)
                if (fabs(Ff[(long)v * nface + f]) > fmax[v]) fmax[v] = fabs(Ff[(long)v * nface + f]);
        const double inv_u = 1.0 / P->dx[d];
#pragma omp parallel for schedule(static)
        for (long c = 0; c < ncell; ++c) {
            int ci[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long)nx * ny))};
            const double inv = P->tab[d] ? tab_row(P, d, ci[d])[TAB_IDX] : inv_u;
            int cb_high = (P->bc[2 * d + 1] == 3 && ci[d] == P->n[d] - 1);
            int cb_low = (P->bc[2 * d] == 3 && ci[d] == 0);
            if (cb_low || cb_high) {   /* characteristic boundary cell: normal part from the amplitudes */
                int nb[3] = {ci[0], ci[1], ci[2]};
                nb[d] += cb_low ? 1 : -1;
                double qb[OR_MAXV], qn[OR_MAXV], o[OR_MAXV];
                fetch_cell(P, q, ci, qb);
                fetch_cell(P, q, nb, qn);
                oracle_cbc_normal(P, d, cb_high, qb, qn, 1.0 / inv, o);
                for (int v = 0; v < ns; ++v) rhs[(long)v * ncell + c] += o[v];
                continue;
            }
            int hi[3] = {ci[0], ci[1], ci[2]};
            hi[d] += 1;
            long flo = ((long)ci[2] * m[1] + ci[1]) * m[0] + ci[0];
            long fhi = ((long)hi[2] * m[1] + hi[1]) * m[0] + hi[0];
            for (int v = 0; v < ns; ++v)
                rhs[(long)v * ncell + c] += (Ff[(long)v * nface + flo] - Ff[(long)v * nface + fhi]) * inv;
            double divu = (Ff[(long)ns * nface + fhi] - Ff[(long)ns * nface + flo]) * inv;
            double K[OR_MAXF] = {0.0, 0.0, 0.0};
            if (P->model == 1) {
                double qc[OR_MAXV], wc[OR_MAXV];
                for (int v = 0; v < ns; ++v) qc[v] = q[(long)v * ncell + c];
                oracle_cons_to_prim(P, qc, wc);
                oracle_kapila_K(P, wc, K);
            }
            for (int a = 0; a < P->nf - 1; ++a) {
                long o = (long)i_alpha(P, a) * ncell + c;
                rhs[o] += (q[o] + K[a]) * divu;
            }
            if (six(P)) {
                double src[OR_MAXF];
                six_work(P, q, ncell, c, src);
                for (int a = 0; a < P->nf; ++a) rhs[(long)i_int(P, a) * ncell + c] -= src[a] * divu;
            }
        }
        free(Ff);
    }
    return nfb;
}

/* R at selected cells only (flat cell indices), computed face by face from the
 * same definitions; out is [ncells][sys_size].  If fmax is not NULL it receives,
 * per variable, the largest |F| over the faces visited. */
void oracle_rhs_cells(const oracle_params *P, const double *q, long nsel, const long *cells,
                      double *out, double *fmax) {
    int ns = sys_size(P);
    int nx = P->n[0], ny = P->n[1];
    long ncell = (long)nx * ny * P->n[2];
    double fm[OR_MAXV];
    for (int v = 0; v < ns; ++v) fm[v] = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : fm[:OR_MAXV])
    for (long s = 0; s < nsel; ++s) {
        long c = cells[s];
        int ci[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long)nx * ny))};
        double *o = out + s * ns;
        for (int v = 0; v < ns; ++v) o[v] = 0.0;
        for (int d = 0; d < P->ndim; ++d) {
            double Flo[OR_MAXV], Fhi[OR_MAXV], ulo, uhi;
            int cb_high = (P->bc[2 * d + 1] == 3 && ci[d] == P->n[d] - 1);
            int cb_low = (P->bc[2 * d] == 3 && ci[d] == 0);
            if (cb_low || cb_high) {
                int nb[3] = {ci[0], ci[1], ci[2]};
                nb[d] += cb_low ? 1 : -1;
                double qb[OR_MAXV], qn[OR_MAXV], ob[OR_MAXV];
                fetch_cell(P, q, ci, qb);
                fetch_cell(P, q, nb, qn);
                double h = P->tab[d] ? 1.0 / tab_row(P, d, ci[d])[TAB_IDX] : P->dx[d];
                oracle_cbc_normal(P, d, cb_high, qb, qn, h, ob);
                for (int v = 0; v < ns; ++v) o[v] += ob[v];
                continue;
            }
            oracle_face(P, q, d, ci[0], ci[1], ci[2], Flo, &ulo);
            int hi[3] = {ci[0], ci[1], ci[2]};
            hi[d] += 1;
            oracle_face(P, q, d, hi[0], hi[1], hi[2], Fhi, &uhi);
            double inv = P->tab[d] ? tab_row(P, d, ci[d])[TAB_IDX] : 1.0 / P->dx[d];
            for (int v = 0; v < ns; ++v) {
                o[v] += (Flo[v] - Fhi[v]) * inv;
                if (fabs(Flo[v]) > fm[v]) fm[v] = fabs(Flo[v]);
                if (fabs(Fhi[v]) > fm[v]) fm[v] = fabs(Fhi[v]);
            }
            double divu = (uhi - ulo) * inv;
            double K[OR_MAXF] = {0.0, 0.0, 0.0};
            if (P->model == 1) {
                double qc[OR_MAXV], wc[OR_MAXV];
                for (int v = 0; v < ns; ++v) qc[v] = q[(long)v * ncell + c];
                oracle_cons_to_prim(P, qc, wc);
                oracle_kapila_K(P, wc, K);
            }
            for (int a = 0; a < P->nf - 1; ++a)
                o[i_alpha(P, a)] += (q[(long)i_alpha(P, a) * ncell + c] + K[a]) * divu;
            if (six(P)) {
                double src[OR_MAXF];
                six_work(P, q, ncell, c, src);
                for (int a = 0; a < P->nf; ++a) o[i_int(P, a)] -= src[a] * divu;
            }
        }
    }
    if (fmax)
        for (int v = 0; v < ns; ++v) fmax[v] = fm[v];
}

/* max over cells of max_d (|u_d| + c)/dx_d; *bad counts cells with a
 * non-finite state or c^2 <= 0. */
double oracle_max_rate(const oracle_params *P, const double *q, long *bad) {
    int ns = sys_size(P);
    long ncell = (long)P->n[0] * P->n[1] * P->n[2];
    double m = 0.0;
    long nbad = 0;
#pragma omp parallel for schedule(static) reduction(max : m) reduction(+ : nbad)
    for (long c = 0; c < ncell; ++c) {
        double qc[OR_MAXV], w[OR_MAXV];
        for (int v = 0; v < ns; ++v) qc[v] = q[(long)v * ncell + c];
        oracle_cons_to_prim(P, qc, w);
        double c2 = sound_speed_sq(P, w);
        if (!(c2 > 0.0) || !isfinite(c2)) { nbad += 1; continue; }
        double cs = sqrt(c2);
        int ci[3] = {(int)(c % P->n[0]), (int)((c / P->n[0]) % P->n[1]), (int)(c / ((long)P->n[0] * P->n[1]))};
        for (int d = 0; d < P->ndim; ++d) {
            double r = P->tab[d] ? (fabs(w[i_mom(P, d)]) + cs) * tab_row(P, d, ci[d])[TAB_IDX]
                                 : (fabs(w[i_mom(P, d)]) + cs) / P->dx[d];
            if (r > m) m = r;
        }
    }
    *bad = nbad;
    return m;
}
