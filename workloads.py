"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method (no equation of state, no
reconstruction, no flux): it only lays out PRIMITIVE fields
w = (a_1 r_1 .. a_N r_N, u_1 .. u_d, p, a_1 .. a_{N-1}) as float64 arrays of shape
[sys_size][nz][ny][nx].  Each side (the CUDA path through its own
``mfc_set_state_prim``, the oracle through its own conversion) turns them into
conserved variables.

The geometry follows the synthetic shock/bubble workloads used to exercise the
method of arXiv 2305.09163 (Sec. 5 measures a 3D two-component air/water
problem; Sec. 6.1 a bubble cloud hit by a pressure wave; Sec. 6.2 bubbles beside
a stiff solid).  No dataset is involved.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Stiffened-gas parameters (gamma, pi_inf [Pa]) and pure-phase densities.
WATER = (4.4, 6.0e8)
AIR = (1.4, 0.0)
SOLID = (3.0, 1.0e10)
RHO_WATER, RHO_AIR, RHO_SOLID = 1000.0, 1.0, 2000.0
P_AMBIENT = 1.0e5
P_SHOCK = 1.0e9
ALPHA_MIN = 1.0e-6

# Water behind a shock that raises p from 1e5 Pa to 1e9 Pa in water at rest
# (Rankine-Hugoniot for the stiffened gas above).  Written by
# ``oracle/shock_constants.py``; a CPU test recomputes them with the oracle.
SHOCK_RHO = 1230.377372836252
SHOCK_U = 432.69216080845405
SHOCK_SPEED = 2310.880784462928

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_CHARACTERISTIC = 0, 1, 2, 3


@dataclass
class Workload:
    """Everything needed to set up one run: grid, BCs, fluids and the initial
    primitive state (as a callable, so large arrays are only built on demand)."""
    name: str
    n: tuple
    lo: tuple
    hi: tuple
    bc: tuple
    gamma: tuple
    pi_inf: tuple
    cfl: float
    steps: int
    t_end: float | None = None
    seed: int | None = None
    notes: str = ""
    builder: object = field(default=None, repr=False)
    faces: tuple | None = None   # non-uniform grid: face coordinates per direction (or None)

    @property
    def ndim(self) -> int:
        return 3 if self.n[2] > 1 else (2 if self.n[1] > 1 else 1)

    @property
    def nf(self) -> int:
        return len(self.gamma)

    @property
    def sys_size(self) -> int:
        return 2 * self.nf + self.ndim

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def prims(self) -> np.ndarray:
        return self.builder(self)


def _centers(n, lo, hi, faces=None):
    out = []
    for d in range(3):
        if faces is not None and faces[d] is not None:
            f = np.asarray(faces[d], dtype=np.float64)
            out.append(0.5 * (f[1:] + f[:-1]))
        else:
            out.append(lo[d] + (np.arange(n[d]) + 0.5) * (hi[d] - lo[d]) / n[d])
    return out


def stretched_faces(n: int, lo: float, hi: float, a: float, xa: float, xb: float) -> np.ndarray:
    """Face coordinates of n cells after the hyperbolic-tangent stretching the
    paper gives for its droplet case (Sec. 6.3): x_s = x + (x/a)[log cosh(a(x-xa)/L)
    + log cosh(a(x-xb)/L) - 2 log cosh(a(xb-xa)/(2L))] applied to the uniform
    faces of [lo, hi], L = hi - lo; cells are finest between xa and xb."""
    x = np.linspace(lo, hi, n + 1)
    L = hi - lo
    lc = lambda z: np.log(np.cosh(z))
    return x + (x / a) * (lc(a * (x - xa) / L) + lc(a * (x - xb) / L) - 2.0 * lc(a * (xb - xa) / (2.0 * L)))


def _pack(nf, ndim, rho_k, alpha, u, p):
    """Stack primitive fields: alpha[k] for all N fluids, rho_k pure densities."""
    shape = p.shape
    w = np.empty((2 * nf + ndim,) + shape)
    for k in range(nf):
        w[k] = alpha[k] * rho_k[k]
    for d in range(ndim):
        w[nf + d] = u[d]
    w[nf + ndim] = p
    for k in range(nf - 1):
        w[nf + ndim + 1 + k] = alpha[k]
    return w


def _smear(r, radius, width):
    """Indicator of r < radius smeared by tanh over about two cells: 1 inside."""
    return 0.5 * (1.0 - np.tanh((r - radius) / width))


# --------------------------------------------------------------------------
# 1D water/air shock tube (1000 cells on [0,1], interface at x = 0.7)
# --------------------------------------------------------------------------
def _build_shock_tube(wl: Workload) -> np.ndarray:
    x = _centers(wl.n, wl.lo, wl.hi)[0]
    left = x < 0.7
    a_w = np.where(left, 1.0 - ALPHA_MIN, ALPHA_MIN)
    a_a = 1.0 - a_w
    p = np.where(left, P_SHOCK, P_AMBIENT)
    u = [np.zeros_like(x)]
    w = _pack(2, 1, (RHO_WATER, RHO_AIR), (a_w, a_a), u, p)
    return w.reshape(w.shape[0], 1, 1, wl.n[0])


def shock_tube(n: int = 1000) -> Workload:
    return Workload(
        name="water_air_shock_tube_1d_%d" % n, n=(n, 1, 1), lo=(0.0, 0.0, 0.0),
        hi=(1.0, 1.0, 1.0), bc=(BC_TRANSMISSIVE,) * 6, gamma=(WATER[0], AIR[0]),
        pi_inf=(WATER[1], AIR[1]), cfl=0.3, steps=0, t_end=240e-6,
        notes="left water p=1e9 | right air p=1e5, interface x=0.7, alpha in [1e-6, 1-1e-6]",
        builder=_build_shock_tube)


# --------------------------------------------------------------------------
# 3D shock-bubble and shock-bubble-cloud workloads
# --------------------------------------------------------------------------
def _bubble_field(n, lo, hi, bubbles, width, faces=None):
    """max over bubbles of the smeared indicator; each bubble only touches its
    bounding box so large grids stay cheap."""
    cen = _centers(n, lo, hi, faces)
    xc, yc, zc = cen
    ind = np.zeros((n[2], n[1], n[0]))
    for (cx, cy, cz, rad) in bubbles:
        reach = rad + 6.0 * width
        sl = []
        for d, c in enumerate((cx, cy, cz)):
            a = int(np.searchsorted(cen[d], c - reach))
            b = int(np.searchsorted(cen[d], c + reach)) + 1
            sl.append(slice(max(0, a), min(n[d], b)))
        if any(s.start >= s.stop for s in sl):
            continue
        X = xc[sl[0]][None, None, :]
        Y = yc[sl[1]][None, :, None]
        Z = zc[sl[2]][:, None, None]
        r = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2)
        blk = ind[sl[2], sl[1], sl[0]]
        np.maximum(blk, _smear(r, rad, width), out=blk)
    return ind


def _shock_region(n, lo, hi, x_shock, faces=None):
    xc = _centers(n, lo, hi, faces)[0]
    return np.broadcast_to((xc < x_shock)[None, None, :], (n[2], n[1], n[0]))


def _two_fluid_bubbles(wl: Workload, bubbles, width=None) -> np.ndarray:
    dx = (wl.hi[0] - wl.lo[0]) / wl.n[0] if width is None else width
    air = _bubble_field(wl.n, wl.lo, wl.hi, bubbles, dx, wl.faces)
    a_air = ALPHA_MIN + (1.0 - 2.0 * ALPHA_MIN) * air
    a_w = 1.0 - a_air
    shocked = _shock_region(wl.n, wl.lo, wl.hi, wl.lo[0] + 0.05, wl.faces)
    rho_w = np.where(shocked, SHOCK_RHO, RHO_WATER)
    p = np.where(shocked, P_SHOCK, P_AMBIENT)
    ux = np.where(shocked, SHOCK_U, 0.0)
    zero = np.zeros_like(p)
    w = np.empty((7,) + p.shape)
    w[0] = a_w * rho_w
    w[1] = a_air * RHO_AIR
    w[2] = ux
    w[3] = zero
    w[4] = zero
    w[5] = p
    w[6] = a_w
    return w


def _build_shock_bubble(wl: Workload) -> np.ndarray:
    return _two_fluid_bubbles(wl, [(0.5, 0.5, 0.5, 0.1)])


def shock_bubble(n: int = 256, steps: int = 1000) -> Workload:
    return Workload(
        name="shock_bubble_3d_%d" % n, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        bc=(BC_TRANSMISSIVE,) * 6, gamma=(WATER[0], AIR[0]), pi_inf=(WATER[1], AIR[1]),
        cfl=0.3, steps=steps,
        notes="air bubble R=0.1 at the centre of a water cube; 1e9 Pa shocked water for x<0.05",
        builder=_build_shock_bubble)


def six_equation_prims(w: np.ndarray, nf: int, spread: float = 0.0, seed: int = 0) -> np.ndarray:
    """Primitive state of the six-equation model from a five-equation one:
    the same rows (the pressure row stands for the mixture pressure) followed
    by N phase pressures, equal to the mixture pressure times
    (1 + spread * N(0,1) noise) per phase and cell (spread = 0: pressure
    equilibrium)."""
    w = np.asarray(w, dtype=np.float64)
    ndim = w.shape[0] - 2 * nf
    p = w[nf + ndim]
    rng = np.random.default_rng(seed)
    pk = [p * (1.0 + spread * rng.standard_normal(p.shape)) if spread else p.copy() for _ in range(nf)]
    return np.concatenate([w, np.stack(pk)], axis=0)


def shock_bubble_cbc(n: int = 256, steps: int = 1000) -> Workload:
    """The shock-bubble with characteristic (non-reflecting) boundaries on all
    six faces instead of transmissive ghost cells; same initial state."""
    return Workload(
        name="shock_bubble_cbc_3d_%d" % n, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        bc=(BC_CHARACTERISTIC,) * 6, gamma=(WATER[0], AIR[0]), pi_inf=(WATER[1], AIR[1]),
        cfl=0.3, steps=steps,
        notes="shock_bubble_3d with non-reflecting faces",
        builder=_build_shock_bubble)


def _build_shock_bubble_stretched(wl: Workload) -> np.ndarray:
    c = [0.5 * (wl.lo[d] + wl.hi[d]) for d in range(3)]
    # the interface is smeared over about two of the (smallest) cells around the bubble
    width = float(min(np.diff(wl.faces[d]).min() for d in range(3)))
    return _two_fluid_bubbles(wl, [(c[0], c[1], c[2], 0.1)], width)


def shock_bubble_stretched(n: int = 256, a: float = 4.0, steps: int = 1000) -> Workload:
    """The shock-bubble on a grid stretched as the paper's droplet case
    (Sec. 6.3): the mapping of stretched_faces on [-0.5, 0.5] per direction with
    x_a = -0.12, x_b = 0.12 (1.2 bubble diameters), shifted to start at 0; the
    air bubble (R = 0.1) sits at the centre of the refined region, the shocked
    water at x < 0.05."""
    f = stretched_faces(n, -0.5, 0.5, a, -0.12, 0.12)
    f = f - f[0]
    faces = (f, f.copy(), f.copy())
    return Workload(
        name="shock_bubble_stretched_3d_%d" % n, n=(n, n, n), lo=(0.0,) * 3, hi=(float(f[-1]),) * 3,
        bc=(BC_TRANSMISSIVE,) * 6, gamma=(WATER[0], AIR[0]), pi_inf=(WATER[1], AIR[1]),
        cfl=0.3, steps=steps, faces=faces,
        notes="shock-bubble on a tanh-stretched grid (a = %g), cells finest around the bubble" % a,
        builder=_build_shock_bubble_stretched)


def bubble_cloud_layout(count, seed, box_lo, box_hi, median_r, sigma, min_gap, max_tries=200000):
    """Lognormal radii (median, sigma of ln r), uniform centres, rejection of
    overlaps closer than min_gap (surface to surface)."""
    rng = np.random.default_rng(seed)
    out = []
    tries = 0
    while len(out) < count and tries < max_tries:
        tries += 1
        r = float(np.exp(np.log(median_r) + sigma * rng.standard_normal()))
        c = [float(rng.uniform(box_lo[d] + r, box_hi[d] - r)) for d in range(3)]
        ok = True
        for (x, y, z, rr) in out:
            if math.dist(c, (x, y, z)) < r + rr + min_gap:
                ok = False
                break
        if ok:
            out.append((c[0], c[1], c[2], r))
    if len(out) < count:
        raise RuntimeError("could not place %d bubbles" % count)
    return out


def _build_cloud(wl: Workload) -> np.ndarray:
    dx = 1.0 / wl.n[0]
    bubbles = bubble_cloud_layout(64, wl.seed, (0.15, 0.05, 0.05), (0.95, 0.95, 0.95),
                                  0.02, 0.3, 2.0 * dx)
    return _two_fluid_bubbles(wl, bubbles)


def bubble_cloud(n: int = 384, steps: int = 500, seed: int = 230509163) -> Workload:
    return Workload(
        name="shock_bubble_cloud_3d_%d" % n, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        bc=(BC_TRANSMISSIVE,) * 6, gamma=(WATER[0], AIR[0]), pi_inf=(WATER[1], AIR[1]),
        cfl=0.3, steps=steps, seed=seed,
        notes="64 air bubbles, lognormal radii (median 0.02, sigma 0.3), seeded",
        builder=_build_cloud)


def _build_cloud_box(wl: Workload) -> np.ndarray:
    # the bubbles of the full cloud (layout gap from its own cell size), on this
    # box's cells, interfaces smeared over this grid's cell width
    bubbles = bubble_cloud_layout(64, wl.seed, (0.15, 0.05, 0.05), (0.95, 0.95, 0.95),
                                  0.02, 0.3, 2.0 / wl.layout_n)
    return _two_fluid_bubbles(wl, bubbles)


def bubble_cloud_box(n: int, lo=(0.0, 0.25, 0.25), hi=(0.5, 0.75, 0.75), layout_n: int = 384,
                     seed: int = 230509163) -> Workload:
    """A box of the bubble cloud (the bubbles of the layout_n^3 cloud, the same
    shock) on n cells per direction: with the default box, n = layout_n / 2 has
    the full cloud's cell size and n = layout_n half of it."""
    wl = Workload(
        name="shock_bubble_cloud_box_%d" % n, n=(n, n, n), lo=tuple(lo), hi=tuple(hi),
        bc=(BC_TRANSMISSIVE,) * 6, gamma=(WATER[0], AIR[0]), pi_inf=(WATER[1], AIR[1]),
        cfl=0.3, steps=0, seed=seed,
        notes="box [%g,%g]x[%g,%g]x[%g,%g] of the %d^3 bubble cloud" % (lo[0], hi[0], lo[1], hi[1], lo[2], hi[2],
                                                                       layout_n),
        builder=_build_cloud_box)
    wl.layout_n = layout_n
    return wl


def _build_three_fluid(wl: Workload) -> np.ndarray:
    dx = 1.0 / wl.n[0]
    bubbles = bubble_cloud_layout(128, wl.seed, (0.15, 0.05, 0.05), (0.7, 0.95, 0.95),
                                  0.02, 0.3, 2.0 * dx)
    air = _bubble_field(wl.n, wl.lo, wl.hi, bubbles, dx)
    xc = _centers(wl.n, wl.lo, wl.hi)[0]
    slab = 0.25 * (1.0 + np.tanh((xc - 0.75) / dx)) * (1.0 - np.tanh((xc - 0.9) / dx))
    slab = np.broadcast_to(slab[None, None, :], air.shape)
    a_solid = ALPHA_MIN + (1.0 - 3.0 * ALPHA_MIN) * slab
    a_air = ALPHA_MIN + (1.0 - 3.0 * ALPHA_MIN) * air * (1.0 - slab)
    a_w = 1.0 - a_air - a_solid
    shocked = _shock_region(wl.n, wl.lo, wl.hi, 0.05)
    rho_w = np.where(shocked, SHOCK_RHO, RHO_WATER)
    p = np.where(shocked, P_SHOCK, P_AMBIENT)
    ux = np.where(shocked, SHOCK_U, 0.0)
    w = np.empty((9,) + p.shape)
    w[0] = a_w * rho_w
    w[1] = a_air * RHO_AIR
    w[2] = a_solid * RHO_SOLID
    w[3] = ux
    w[4] = 0.0
    w[5] = 0.0
    w[6] = p
    w[7] = a_w
    w[8] = a_air
    return w


def three_fluid(n: int = 512, steps: int = 200, seed: int = 230509164) -> Workload:
    return Workload(
        name="three_fluid_3d_%d" % n, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        bc=(BC_TRANSMISSIVE,) * 6, gamma=(WATER[0], AIR[0], SOLID[0]),
        pi_inf=(WATER[1], AIR[1], SOLID[1]), cfl=0.3, steps=steps, seed=seed,
        notes="water with 128 air bubbles beside a stiff slab (gamma=3, pinf=1e10) at x in [0.75,0.9]",
        builder=_build_three_fluid)


# --------------------------------------------------------------------------
# Random but physical states for parity tests
# --------------------------------------------------------------------------
def random_prims(n, nf, seed, water_air=True, jumps=True, noise=0.05):
    """Smooth random fields plus optional sharp jumps, all physical.

    Partial densities and pressure stay positive and volume fractions stay in
    (0,1) with margins, so every WENO5 face state remains physical.
    """
    n = tuple(n) + (1,) * (3 - len(n))
    ndim = 3 if n[2] > 1 else (2 if n[1] > 1 else 1)
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    grids = np.meshgrid(*[np.arange(m) / max(m, 1) for m in (n[2], n[1], n[0])], indexing="ij")

    def smooth(amp):
        f = np.zeros(shape)
        for _ in range(3):
            k = rng.integers(1, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            f += np.sin(2 * np.pi * (k[0] * grids[0] + k[1] * grids[1] + k[2] * grids[2]) + ph)
        return amp * f / 3.0

    def jump_mask():
        if not jumps:
            return np.zeros(shape)
        nrm = rng.standard_normal(3)
        off = rng.uniform(0.3, 0.7)
        s = nrm[0] * grids[0] + nrm[1] * grids[1] + nrm[2] * grids[2]
        return (s > off * (abs(nrm).sum() * 0.5)).astype(np.float64)

    J = jump_mask()
    a = np.empty((nf,) + shape)
    base = rng.dirichlet(np.ones(nf) * 4.0)
    raw = np.empty((nf,) + shape)
    for k in range(nf):
        raw[k] = base[k] * (1.0 + smooth(0.3)) * (1.0 + 0.6 * J * (1 if k == 0 else -0.5)) \
            + 0.05 + noise * rng.uniform(0, 1, shape) * 0.2
    a[:] = raw / raw.sum(axis=0)
    if water_air and nf >= 2:
        rho_pure = [RHO_WATER, RHO_AIR, RHO_SOLID][:nf]
    else:
        rho_pure = [1.0 + k for k in range(nf)]
    w = np.empty((2 * nf + ndim,) + shape)
    for k in range(nf):
        w[k] = a[k] * rho_pure[k] * (1.0 + smooth(0.2)) * (1.0 + noise * rng.uniform(-1, 1, shape))
    vel_scale = 100.0 if water_air else 0.5
    for d in range(ndim):
        w[nf + d] = vel_scale * (smooth(1.0) + 0.5 * J * rng.uniform(-1, 1)
                                 + noise * rng.uniform(-1, 1, shape))
    p0 = 1.0e6 if water_air else 1.0
    w[nf + ndim] = p0 * (1.0 + smooth(0.4)) * (1.0 + 2.0 * J) * (1.0 + noise * rng.uniform(-1, 1, shape))
    for k in range(nf - 1):
        w[nf + ndim + 1 + k] = a[k]
    return w


def fluids(nf, water_air=True):
    """(gamma, pi_inf) tuples for random-state tests."""
    if water_air:
        tab = [WATER, AIR, SOLID][:nf]
    else:
        tab = [(1.4, 0.0), (1.6, 0.0), (2.0, 0.0)][:nf]
    return tuple(t[0] for t in tab), tuple(t[1] for t in tab)
