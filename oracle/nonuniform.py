"""WENO5 coefficients on a non-uniform grid, from their definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 4.1 of arXiv 2305.09163 discretises on a structured mesh with
non-uniform spacing (tanh stretching; the face coordinates come from the
input generators); Listing 1 (Sec. 4.2) reconstructs with per-index coefficient tables
(candidate, smoothness-indicator and ideal-weight coefficients per cell).  The
tables follow from the finite-volume WENO construction (Jiang & Shu; Shu's
notes, which Sec. 3.2 cites for the details), written here directly:

* candidate r of cell i (cells i-2+r .. i+r) is p_r = P_r', P_r the cubic
  interpolating the primitive function V(x) = int v at the four faces of its
  cells; its edge values at x_{i+1/2} and x_{i-1/2} are linear in the cell
  values;
* the ideal weights d_r make sum_r d_r p_r(x_e) the value at x_e of the
  derivative of the quintic through V at the six faces of cells i-2..i+2
  (a consistent 5x3 linear system, solved by least squares and checked);
* beta_r = sum_{l=1,2} dx_i^(2l-1) int_{cell i} (p_r^(l))^2 dx, a quadratic form
  in the three cell values.

Coordinates are shifted to x_{i-1/2} and scaled by dx_i before fitting, so
every polynomial is well conditioned.  The grid is given by its face
coordinates per direction; ghost cells repeat the widths of the interior cells
they mirror (periodic: wrap around).
"""
from __future__ import annotations

import numpy as np

GHOST = 3


def ghost_widths(faces: np.ndarray, periodic: bool) -> np.ndarray:
    """Cell widths with GHOST ghost cells on each side: index 0 is cell -GHOST."""
    h = np.diff(np.asarray(faces, dtype=np.float64))
    n = h.size
    idx = np.arange(-GHOST, n + GHOST)
    if periodic:
        m = idx % n
    else:
        m = np.where(idx < 0, -idx - 1, np.where(idx >= n, 2 * n - 1 - idx, idx))
    return h[m]


def _face_positions(h5: np.ndarray) -> np.ndarray:
    """Six face coordinates of five cells of widths h5, scaled by the middle
    cell's width, with the middle cell's left face at 0."""
    f = np.concatenate([[0.0], np.cumsum(h5)])
    return (f - f[2]) / h5[2]


def _primitive_derivative_rows(faces: np.ndarray, cells: range, x_eval: float, deriv: int = 0) -> np.ndarray:
    """Row vector c with sum_j c_j v_j = d^(deriv+1)/dx^(deriv+1) of the polynomial
    interpolating V = int v at the faces of `cells` (indices into the five-cell
    stencil), evaluated at x_eval; in scaled coordinates."""
    fc = faces[cells.start:cells.stop + 1]
    deg = len(fc) - 1
    V = np.vander(fc, deg + 1, increasing=True)         # V @ coef = values at faces
    Vinv = np.linalg.inv(V)
    # values at the faces for a unit cell value: primitive = cumulative width
    width = np.diff(fc)
    C = np.zeros((len(fc), 5))
    for m in range(1, len(fc)):
        for j in range(m):
            C[m, cells.start + j] = width[j]
    coef = Vinv @ C                                     # polynomial coefficients per unit value
    k = deriv + 1
    powers = np.array([np.prod(np.arange(p - k + 1, p + 1)) * x_eval ** (p - k) if p >= k else 0.0
                       for p in range(deg + 1)])
    return powers @ coef


def _beta_matrix(faces: np.ndarray, r: int) -> np.ndarray:
    """Quadratic form of beta_r over the five-cell stencil (scaled coordinates:
    the middle cell is [0, 1], so dx_i^(2l-1) = 1)."""
    cells = range(r, r + 3)
    fc = faces[r:r + 4]
    V = np.vander(fc, 4, increasing=True)
    width = np.diff(fc)
    C = np.zeros((4, 5))
    for m in range(1, 4):
        for j in range(m):
            C[m, r + j] = width[j]
    coef = np.linalg.inv(V) @ C                         # cubic P per unit value: coef[p, j]
    M = np.zeros((5, 5))
    for l in (1, 2):                                    # derivative order of p = P'
        k = l + 1
        # d^k P / dx^k as a polynomial per unit value
        dcoef = np.array([[np.prod(np.arange(p - k + 1, p + 1)) if p >= k else 0.0 for p in range(4)]]).T * coef
        # shift powers: term p of P becomes power p - k
        for a in range(4):
            for b in range(4):
                if a < k or b < k:
                    continue
                e = (a - k) + (b - k)
                integ = 1.0 / (e + 1)                   # int_0^1 x^e dx
                M += integ * np.outer(dcoef[a], dcoef[b])
    return M


def cell_tables(h5: np.ndarray):
    """Coefficients of one cell from the widths of cells i-2..i+2.

    Returns a dict of arrays over the five-cell stencil:
      cL[r] (5,), cR[r] (5,): candidate values at x_{i+1/2} and x_{i-1/2};
      dL (3,), dR (3,): ideal weights;  B[r] (5, 5): beta_r = v B_r v.
    """
    f = _face_positions(np.asarray(h5, dtype=np.float64))
    out = {"cL": np.zeros((3, 5)), "cR": np.zeros((3, 5)), "B": np.zeros((3, 5, 5))}
    for side, xe in (("L", f[3]), ("R", f[2])):
        c = np.array([_primitive_derivative_rows(f, range(r, r + 3), xe) for r in range(3)])
        C5 = _primitive_derivative_rows(f, range(0, 5), xe)
        d, res, rank, _ = np.linalg.lstsq(c.T, C5, rcond=None)
        if np.abs(c.T @ d - C5).max() > 1e-9 * np.abs(C5).max():
            raise ValueError("no ideal weights for this stencil")
        out["c" + side] = c
        out["d" + side] = d
    for r in range(3):
        out["B"][r] = _beta_matrix(f, r)
    return out


def direction_tables(faces: np.ndarray, periodic: bool) -> np.ndarray:
    """Packed table of one direction for the C oracle: for the cells -1..n
    (n + 2 rows), 63 values per row: cL[3][5], cR[3][5], dL[3], dR[3],
    B[3][3][3] (beta_r over its own three cells), then 1/dx of the cell."""
    hg = ghost_widths(faces, periodic)
    n = len(faces) - 1
    rows = []
    for i in range(-1, n + 1):
        k = i + GHOST
        t = cell_tables(hg[k - 2:k + 3])
        B3 = np.array([t["B"][r][r:r + 3, r:r + 3] for r in range(3)])
        rows.append(np.concatenate([t["cL"].ravel(), t["cR"].ravel(), t["dL"], t["dR"], B3.ravel(),
                                    [1.0 / hg[k]]]))
    return np.ascontiguousarray(np.array(rows))


TABLE_ROW = 3 * 5 + 3 * 5 + 3 + 3 + 27 + 1   # 64
