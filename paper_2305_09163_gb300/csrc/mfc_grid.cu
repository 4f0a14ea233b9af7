// Non-uniform grids (Sec. 4.1: a structured mesh with non-uniform spacing;
// Listing 1 of Sec. 4.2 reconstructs with per-index coefficient tables).  Host
// code: for every cell of a direction the WENO5 coefficients of the
// finite-volume reconstruction on its five-cell stencil, in the form the
// sweeps use, uploaded once per grid.
//
// For cell c with faces x_{c-5/2} .. x_{c+5/2} (scaled by dx_c, origin at
// x_{c-1/2}):
//  * candidate r (cells c-2+r .. c+r) is p_r = P_r', P_r the cubic through the
//    primitive function V at the candidate's four faces; its value at an edge
//    x_e is sum_m l_m'(x_e) V(x_m) with the Lagrange basis l_m (Shu's formula
//    for the derivative of the basis at a node);
//  * the ideal weights reproduce the five-cell (quintic) value: only candidate
//    0 touches cell c-2 and only candidate 2 cell c+2, so d0 and d2 follow from
//    those two coefficients and d1 = 1 - d0 - d2;
//  * beta_r = int_0^1 (P_r'')^2 + (P_r''')^2 dy in scaled coordinates (the
//    dx_c^(2l-1) factors of the definition cancel), from the Newton divided
//    differences of V, as a quadratic form in the candidate's two differences.
//
// A row (28 values, each stored as an FP32 pair hi + lo for the FP64 path's
// float-float arithmetic; the FP32 path reads hi): for the edges at c+1/2 and
// c-1/2 the candidate increments p_r - v_c = ea_r Da_r + eb_r Db_r with (Da, Db)
// the candidate's differences ((D0,D1), (D1,D2), (D2,D3)), the ideal weights of
// both edges, beta_r = qa Da^2 + qab Da Db + qb Db^2, and 1/dx_c.
#include <cmath>
#include <cstring>
#include <vector>

#include "mfc_grid.h"

namespace mfc {

namespace {

// d/dx of the Lagrange basis polynomial of node m over nodes x[0..np-1] at xe.
double lagrange_basis_derivative(const double* x, int np, int m, double xe) {
    double den = 1.0;
    for (int q = 0; q < np; ++q)
        if (q != m) den *= x[m] - x[q];
    double num = 0.0;
    for (int l = 0; l < np; ++l) {
        if (l == m) continue;
        double t = 1.0;
        for (int q = 0; q < np; ++q)
            if (q != m && q != l) t *= xe - x[q];
        num += t;
    }
    return num / den;
}

// Edge value coefficients (over the stencil's cells) of the polynomial whose
// derivative interpolates the primitive function at faces x[0..ncell].
void edge_coeffs(const double* x, int ncell, double xe, double* c) {
    double w[6];
    for (int m = 0; m <= ncell; ++m) w[m] = lagrange_basis_derivative(x, ncell + 1, m, xe);
    for (int j = 0; j < ncell; ++j) {
        double s = 0.0;
        for (int m = j + 1; m <= ncell; ++m) s += w[m];
        c[j] = s * (x[j + 1] - x[j]);
    }
}

// beta of one candidate as a quadratic form in its cell values (3x3), by the
// Newton form of the cubic through V at its four faces x[0..3]; the cell is
// [0, 1].
void beta_form(const double* x, double B[3][3]) {
    double a[3], b[3], cc[3];   // P'' = a + b y, P''' = cc, per unit cell value
    for (int j = 0; j < 3; ++j) {
        double V[4] = {0, 0, 0, 0};
        for (int m = 1; m < 4; ++m) V[m] = V[m - 1] + (m - 1 == j ? x[m] - x[m - 1] : 0.0);
        // divided differences f[x0,x1], f[x0,x1,x2], f[x0..x3] (V(x0) = 0)
        double d01 = (V[1] - V[0]) / (x[1] - x[0]), d12 = (V[2] - V[1]) / (x[2] - x[1]);
        double d23 = (V[3] - V[2]) / (x[3] - x[2]);
        double d012 = (d12 - d01) / (x[2] - x[0]), d123 = (d23 - d12) / (x[3] - x[1]);
        double d0123 = (d123 - d012) / (x[3] - x[0]);
        // P = ... + d012 (y-x0)(y-x1) + d0123 (y-x0)(y-x1)(y-x2)
        // P'' = 2 d012 + d0123 (6 y - 2 (x0 + x1 + x2)),  P''' = 6 d0123
        a[j] = 2.0 * d012 - 2.0 * d0123 * (x[0] + x[1] + x[2]);
        b[j] = 6.0 * d0123;
        cc[j] = 6.0 * d0123;
    }
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            B[j][k] = a[j] * a[k] + 0.5 * (a[j] * b[k] + a[k] * b[j]) + b[j] * b[k] / 3.0 + cc[j] * cc[k];
}

// One row from the widths of cells c-2..c+2.
void cell_row(const double* h5, double* row) {
    double f[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 5; ++i) f[i + 1] = f[i] + h5[i];
    const double x0 = f[2];
    for (int i = 0; i < 6; ++i) f[i] = (f[i] - x0) / h5[2];   // scaled, cell c = [0, 1]
    for (int side = 0; side < 2; ++side) {
        const double xe = side == 0 ? f[3] : f[2];
        double cand[3][3], big[5];
        for (int r = 0; r < 3; ++r) edge_coeffs(f + r, 3, xe, cand[r]);
        edge_coeffs(f, 5, xe, big);
        const double d0 = big[0] / cand[0][0], d2 = big[4] / cand[2][2];
        double* e = row + 6 * side;
        // increments over v_c in the candidate's own differences
        e[0] = -cand[0][0];
        e[1] = -(cand[0][0] + cand[0][1]);
        e[2] = -cand[1][0];
        e[3] = cand[1][2];
        e[4] = cand[2][1] + cand[2][2];
        e[5] = cand[2][2];
        double* d = row + 12 + 3 * side;
        d[0] = d0;
        d[1] = 1.0 - d0 - d2;
        d[2] = d2;
    }
    for (int r = 0; r < 3; ++r) {
        double B[3][3];
        beta_form(f + r, B);
        // v = (0, Da, Da + Db): beta = qa Da^2 + qab Da Db + qb Db^2
        const double qa = B[1][1] + B[2][2] + 2.0 * B[1][2];
        const double qab = 2.0 * (B[1][2] + B[2][2]);
        const double qb = B[2][2];
        row[18 + 3 * r] = qa;
        row[19 + 3 * r] = qab;
        row[20 + 3 * r] = qb;
    }
    row[27] = 1.0 / h5[2];
}

}  // namespace

bool grid_tables(const double* faces, int n, bool periodic, std::vector<float>& out) {
    if (n < 3 || !faces) return false;
    std::vector<double> h(n);
    for (int i = 0; i < n; ++i) {
        h[i] = faces[i + 1] - faces[i];
        if (!(h[i] > 0.0) || !std::isfinite(h[i])) return false;
    }
    auto width = [&](int i) {   // ghost widths mirror (or wrap) the interior ones
        int m;
        if (periodic) m = ((i % n) + n) % n;
        else m = i < 0 ? -i - 1 : (i >= n ? 2 * n - 1 - i : i);
        return h[m];
    };
    out.assign((size_t)(n + 2) * kGridRow * 2, 0.f);
    for (int c = -1; c <= n; ++c) {
        double h5[5], row[kGridRow];
        for (int k = 0; k < 5; ++k) h5[k] = width(c - 2 + k);
        cell_row(h5, row);
        float* o = out.data() + (size_t)(c + 1) * kGridRow * 2;
        for (int k = 0; k < kGridRow; ++k) {
            if (!std::isfinite(row[k])) return false;
            const float hi = (float)row[k];
            o[2 * k] = hi;
            o[2 * k + 1] = (float)(row[k] - (double)hi);
        }
    }
    return true;
}

}  // namespace mfc

extern "C" int mfc_grid_table(const double* faces, int n, int periodic, float* out, long long out_len) {
    std::vector<float> tab;
    if (!mfc::grid_tables(faces, n, periodic != 0, tab)) return -1;
    if (!out || out_len < (long long)tab.size()) return (int)tab.size();
    std::memcpy(out, tab.data(), tab.size() * sizeof(float));
    return 0;
}
