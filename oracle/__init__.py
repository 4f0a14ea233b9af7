"""CPU FP64 oracle for the five-equation diffuse-interface right-hand side.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA product
path never imports, links or calls it, and it imports nothing from the product
package.

Contents (each cites the passage of arXiv 2305.09163 it follows):
  * ``mfc_oracle.c`` (loaded with ctypes): EOS (Sec. 2.1, Eq. "soe"), the Allaire
    and Kapila five-equation models (Sec. 2.1), the six-equation model and its
    pressure relaxation (Sec. 2.3), WENO5-JS
    and WENO3-JS (Sec. 3.2), HLLC (Sec. 3.2.1), ghost cells (Sec. 3.3), the semi-discrete
    operator (Sec. 3.1, Eq. "fvmdis") and the CFL rate.
  * this module: SSP-RK1/2/3 (Sec. 3.4, Gottlieb & Shu TVD Runge-Kutta; for the
    six-equation model every stage is followed by the pressure relaxation) and
    the CFL time step, in plain numpy on top of the C right-hand side.
  * ``exact_riemann``: exact two-material stiffened-gas Riemann solution used to
    judge shock-tube runs.
  * ``mlp``: FP64 forward/backward of the learned-weight network.
  * ``nonuniform``: WENO5 coefficient tables of a non-uniform grid (Sec. 4.1,
    Listing 1) from their definitions, and the tanh stretching of Sec. 6.3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mfc_oracle.c")
_LIB = os.path.join(_HERE, "libmfc_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_CHARACTERISTIC = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no fused multiply-add, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("ndim", ctypes.c_int),
        ("nf", ctypes.c_int),
        ("dx", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 6),
        ("gamma", ctypes.c_double * 3),
        ("pi_inf", ctypes.c_double * 3),
        ("eps", ctypes.c_double),
        ("fallback", ctypes.c_int),
        ("weno_order", ctypes.c_int),
        ("model", ctypes.c_int),
        ("tab", ctypes.POINTER(ctypes.c_double) * 3),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(Params)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_long)
            lib.oracle_sys_size.argtypes = [P]
            lib.oracle_sys_size.restype = ctypes.c_int
            lib.oracle_cons_to_prim.argtypes = [P, dp, dp]
            lib.oracle_prim_to_cons.argtypes = [P, dp, dp]
            lib.oracle_prim_to_cons_array.argtypes = [P, dp, dp, ctypes.c_long]
            lib.oracle_cons_to_prim_array.argtypes = [P, dp, dp, ctypes.c_long]
            lib.oracle_weno5.argtypes = [dp, ctypes.c_double]
            lib.oracle_weno5.restype = ctypes.c_double
            lib.oracle_weno5_weights.argtypes = [dp, ctypes.c_double, dp, dp]
            lib.oracle_weno5_beta.argtypes = [dp, dp]
            lib.oracle_kapila_K.argtypes = [P, dp, dp]
            lib.oracle_weno3.argtypes = [dp, ctypes.c_double]
            lib.oracle_weno3.restype = ctypes.c_double
            lib.oracle_weno3_weights.argtypes = [dp, ctypes.c_double, dp, dp]
            lib.oracle_hllc.argtypes = [P, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_face.argtypes = [P, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, dp, dp]
            lib.oracle_face.restype = ctypes.c_int
            lib.oracle_rhs.argtypes = [P, dp, dp, dp]
            lib.oracle_rhs.restype = ctypes.c_long
            lib.oracle_rhs_cells.argtypes = [P, dp, ctypes.c_long, lp, dp, dp]
            lib.oracle_max_rate.argtypes = [P, dp, lp]
            lib.oracle_max_rate.restype = ctypes.c_double
            lib.oracle_relax6.argtypes = [P, dp]
            lib.oracle_relax6.restype = ctypes.c_double
            lib.oracle_relax6_array.argtypes = [P, dp, ctypes.c_long]
            lib.oracle_relax6_array.restype = ctypes.c_long
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Problem:
    """Grid, boundary types and fluids of one problem (Sec. 3.1 uniform grid)."""

    MODELS = {"allaire": 0, "kapila": 1, "six": 2}

    def __init__(self, n, lo, hi, bc, gamma, pi_inf, eps=1e-6, fallback=False, weno_order=5, model="allaire",
                 faces=None):
        """faces: optional per-direction face coordinates (None or a sequence of up
        to three arrays or None) for a non-uniform grid (WENO5 only); lo/hi of a
        non-uniform direction are taken from its faces and dx[d] becomes its
        smallest cell width."""
        n = list(n) + [1] * (3 - len(n))
        self.n = tuple(int(v) for v in n)
        self.ndim = 3 if self.n[2] > 1 else (2 if self.n[1] > 1 else 1)
        self.nf = len(gamma)
        self.lo = tuple(float(v) for v in (list(lo) + [0.0] * (3 - len(lo))))
        self.hi = tuple(float(v) for v in (list(hi) + [1.0] * (3 - len(hi))))
        self.dx = tuple((self.hi[d] - self.lo[d]) / self.n[d] for d in range(3))
        self.bc = tuple(int(b) for b in bc) + (1,) * (6 - len(bc))
        self.gamma = tuple(float(g) for g in gamma)
        self.pi_inf = tuple(float(p) for p in pi_inf)
        self.eps = float(eps)
        self.fallback = bool(fallback)
        if weno_order not in (3, 5):
            raise ValueError("weno_order must be 3 or 5")
        self.weno_order = int(weno_order)
        if model not in self.MODELS:
            raise ValueError("model must be 'allaire', 'kapila' or 'six'")
        self.model = model
        if model != "allaire" and BC_CHARACTERISTIC in self.bc[:2 * self.ndim]:
            raise ValueError("characteristic boundaries are written for the Allaire model")
        # six-equation model: the phase internal energies (conserved) or pressures
        # (primitive) follow the volume fractions
        self.sys_size = (3 if model == "six" else 2) * self.nf + self.ndim
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.faces = [None, None, None]
        self._tabs = [None, None, None]
        if faces is not None:
            from . import nonuniform
            if self.weno_order != 5:
                raise ValueError("non-uniform grids need weno_order 5")
            lo_l, hi_l, dx_l = list(self.lo), list(self.hi), list(self.dx)
            for d, f in enumerate(list(faces)[:3]):
                if f is None:
                    continue
                f = np.ascontiguousarray(f, dtype=np.float64)
                if d >= self.ndim or f.size != self.n[d] + 1 or not np.all(np.diff(f) > 0):
                    raise ValueError("faces[%d] must hold n+1 increasing coordinates of an active direction" % d)
                periodic = self.bc[2 * d] == BC_PERIODIC
                self.faces[d] = f
                self._tabs[d] = nonuniform.direction_tables(f, periodic)
                lo_l[d], hi_l[d], dx_l[d] = f[0], f[-1], float(np.diff(f).min())
            self.lo, self.hi, self.dx = tuple(lo_l), tuple(hi_l), tuple(dx_l)

    def params(self) -> Params:
        p = Params()
        for d in range(3):
            p.n[d] = self.n[d]
            p.dx[d] = self.dx[d]
        p.ndim = self.ndim
        p.nf = self.nf
        for i in range(6):
            p.bc[i] = self.bc[i]
        for k in range(self.nf):
            p.gamma[k] = self.gamma[k]
            p.pi_inf[k] = self.pi_inf[k]
        p.eps = self.eps
        p.fallback = 1 if self.fallback else 0
        p.weno_order = self.weno_order
        p.model = self.MODELS[self.model]
        for d in range(3):
            if self._tabs[d] is not None:
                p.tab[d] = _dp(self._tabs[d])
        return p

    def shape(self):
        """Array shape of a state: [sys_size][nz][ny][nx]."""
        return (self.sys_size, self.n[2], self.n[1], self.n[0])


def _state(pb: Problem, q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    assert q.size == pb.sys_size * pb.ncell, (q.shape, pb.shape())
    return q


def cons_from_prims(pb: Problem, w) -> np.ndarray:
    w = _state(pb, w)
    q = np.empty_like(w)
    _load().oracle_prim_to_cons_array(ctypes.byref(pb.params()), _dp(w), _dp(q), pb.ncell)
    return q.reshape(pb.shape())


def prims_from_cons(pb: Problem, q) -> np.ndarray:
    q = _state(pb, q)
    w = np.empty_like(q)
    _load().oracle_cons_to_prim_array(ctypes.byref(pb.params()), _dp(q), _dp(w), pb.ncell)
    return w.reshape(pb.shape())


def rhs(pb: Problem, q, return_info: bool = False):
    """R(q) of Eq. "fvmdis"; with return_info also (per-variable max |F|, fallback faces)."""
    q = _state(pb, q)
    out = np.empty_like(q)
    fmax = np.zeros(pb.sys_size)
    nfb = _load().oracle_rhs(ctypes.byref(pb.params()), _dp(q), _dp(out), _dp(fmax))
    out = out.reshape(pb.shape())
    if return_info:
        return out, fmax, int(nfb)
    return out


_COUNTED_SRC = os.path.join(_HERE, "mfc_oracle_counted.cpp")
_COUNTED_LIB = os.path.join(_HERE, "libmfc_oracle_counted.so")
_counted = None


def _load_counted():
    """The operation-counting build (mfc_oracle_counted.cpp + flop_count.h):
    the same C source compiled as C++ with every double a counting type, one
    thread, no OpenMP."""
    global _counted
    with _lock:
        if _counted is None:
            deps = [_SRC, _COUNTED_SRC, os.path.join(_HERE, "flop_count.h")]
            if not os.path.exists(_COUNTED_LIB) or any(os.path.getmtime(_COUNTED_LIB) < os.path.getmtime(d)
                                                       for d in deps):
                tmp = _COUNTED_LIB + ".tmp%d" % os.getpid()
                subprocess.check_call(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                                       "-o", tmp, _COUNTED_SRC, "-lm"])
                os.replace(tmp, _COUNTED_LIB)
            lib = ctypes.CDLL(_COUNTED_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_rhs.argtypes = [ctypes.POINTER(Params), dp, dp, dp]
            lib.oracle_rhs.restype = ctypes.c_long
            lib.oracle_face.argtypes = [ctypes.POINTER(Params), dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, dp, dp]
            lib.oracle_face.restype = ctypes.c_int
            lib.oracle_cons_to_prim_array.argtypes = [ctypes.POINTER(Params), dp, dp, ctypes.c_long]
            lib.oracle_flop_reset.argtypes = []
            lib.oracle_flop_read.restype = ctypes.c_ulonglong
            _counted = lib
    return _counted


def rhs_flops(pb: Problem, q):
    """Floating-point operations (+ - * / and sqrt, one each) that the oracle's
    plain formulation spends on one R(q), counted by the counting build; and
    R(q) itself (equal to ``rhs``)."""
    q = _state(pb, q)
    out = np.empty_like(q)
    fmax = np.zeros(pb.sys_size)
    lib = _load_counted()
    lib.oracle_flop_reset()
    lib.oracle_rhs(ctypes.byref(pb.params()), _dp(q), _dp(out), _dp(fmax))
    return int(lib.oracle_flop_read()), out.reshape(pb.shape())


def rhs_flop_breakdown(pb: Problem, q) -> dict:
    """The algorithmic work of one R(q), from the counting build, per unit of
    the method (Sec. 3.1-3.2): ``prims`` per cell (conserved -> primitive, once
    per cell), ``face`` per face and direction (WENO edges of every variable on
    both sides plus HLLC, averaged over the faces: HLLC's branch decides part of
    the count), ``div`` per cell and direction (flux difference and
    volume-fraction source), and ``per_cell_sweep`` = prims/ndim + face + div,
    the work of one directional sweep per cell with one face per cell.  The
    oracle itself recomputes the primitives of the six cells around every face
    and visits n + 1 faces per row; those repeats are taken out here."""
    q = _state(pb, q)
    lib = _load_counted()
    P = pb.params()
    w = np.empty_like(q)
    lib.oracle_flop_reset()
    lib.oracle_cons_to_prim_array(ctypes.byref(P), _dp(q), _dp(w), pb.ncell)
    c_prim = lib.oracle_flop_read() / pb.ncell
    total, _ = rhs_flops(pb, q)
    F = np.empty(pb.sys_size)
    ut = np.empty(1)
    face_work = 0.0        # WENO + HLLC over all faces (one face per cell and direction)
    face_calls = 0.0       # everything oracle_face counted, per direction
    for d in range(pb.ndim):
        m = list(pb.n)
        m[d] += 1
        cnt = 0
        for k in range(m[2]):
            for j in range(m[1]):
                for i in range(m[0]):
                    lib.oracle_flop_reset()
                    lib.oracle_face(ctypes.byref(P), _dp(q), d, i, j, k, _dp(F), _dp(ut))
                    cnt += lib.oracle_flop_read()
        nface = m[0] * m[1] * m[2]
        face_calls += cnt
        face_work += (cnt / nface - 6 * c_prim) * pb.ncell
    c_div = (total - face_calls) / (pb.ncell * pb.ndim)
    c_face = face_work / (pb.ncell * pb.ndim)
    return {"prims": c_prim, "face": c_face, "div": c_div, "rhs_total": total,
            "per_cell_sweep": c_prim / pb.ndim + c_face + c_div}


def rhs_cells(pb: Problem, q, cells, return_fmax: bool = False):
    """R at the given flat cell indices; result [len(cells)][sys_size]
    (and, with return_fmax, the per-variable max |F| over the faces visited)."""
    q = _state(pb, q)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.empty((cells.size, pb.sys_size))
    fmax = np.zeros(pb.sys_size)
    _load().oracle_rhs_cells(ctypes.byref(pb.params()), _dp(q), cells.size,
                             cells.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out), _dp(fmax))
    if return_fmax:
        return out, fmax
    return out


def weno5(v, eps=1e-6) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _load().oracle_weno5(_dp(v), eps)


def weno5_weights(v, eps=1e-6):
    v = np.ascontiguousarray(v, dtype=np.float64)
    om = np.zeros(3)
    cand = np.zeros(3)
    _load().oracle_weno5_weights(_dp(v), eps, _dp(om), _dp(cand))
    return om, cand


def weno5_beta(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    b = np.zeros(3)
    _load().oracle_weno5_beta(_dp(v), _dp(b))
    return b


def kapila_K(pb: Problem, w):
    """Kapila coefficients K_k (k < N) of one primitive cell state (Sec. 2.1)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    K = np.zeros(3)
    _load().oracle_kapila_K(ctypes.byref(pb.params()), _dp(w), _dp(K))
    return K[:pb.nf - 1]


def weno3(v, eps=1e-6) -> float:
    """Third-order WENO-JS value at i+1/2 from cells v = (i-1, i, i+1)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _load().oracle_weno3(_dp(v), eps)


def weno3_weights(v, eps=1e-6):
    v = np.ascontiguousarray(v, dtype=np.float64)
    om = np.zeros(2)
    cand = np.zeros(2)
    _load().oracle_weno3_weights(_dp(v), eps, _dp(om), _dp(cand))
    return om, cand


def hllc(pb: Problem, d: int, wL, wR):
    wL = np.ascontiguousarray(wL, dtype=np.float64)
    wR = np.ascontiguousarray(wR, dtype=np.float64)
    F = np.zeros(pb.sys_size)
    ut = np.zeros(1)
    _load().oracle_hllc(ctypes.byref(pb.params()), d, _dp(wL), _dp(wR), _dp(F), _dp(ut))
    return F, float(ut[0])


def cons_from_prim_cell(pb: Problem, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    q = np.zeros(pb.sys_size)
    _load().oracle_prim_to_cons(ctypes.byref(pb.params()), _dp(w), _dp(q))
    return q


def prim_from_cons_cell(pb: Problem, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    w = np.zeros(pb.sys_size)
    _load().oracle_cons_to_prim(ctypes.byref(pb.params()), _dp(q), _dp(w))
    return w


def max_rate(pb: Problem, q):
    """max_cells max_d (|u_d| + c)/dx_d and the number of non-physical cells."""
    q = _state(pb, q)
    bad = ctypes.c_long(0)
    m = _load().oracle_max_rate(ctypes.byref(pb.params()), _dp(q), ctypes.byref(bad))
    return m, int(bad.value)


def cfl_dt(pb: Problem, q, cfl: float) -> float:
    """Time step from the CFL condition: dt = CFL / max_d max_cells (|u_d|+c)/dx_d."""
    m, bad = max_rate(pb, q)
    if bad:
        raise FloatingPointError("non-physical state in %d cells" % bad)
    return cfl / m


def relax(pb: Problem, q) -> np.ndarray:
    """Six-equation model: pressure relaxation with infinite stiffness of every
    cell (Sec. 2.3; oracle_relax6), returning a new state."""
    if pb.model != "six":
        raise ValueError("relaxation belongs to the six-equation model")
    q = np.array(_state(pb, q), dtype=np.float64)
    bad = _load().oracle_relax6_array(ctypes.byref(pb.params()), _dp(q), pb.ncell)
    if bad:
        raise FloatingPointError("relaxation failed in %d cells" % bad)
    return q.reshape(pb.shape())


def relax_cell(pb: Problem, q):
    """Relax one conserved cell state; returns (relaxed state, relaxed pressure p^)."""
    q = np.array(q, dtype=np.float64)
    ph = _load().oracle_relax6(ctypes.byref(pb.params()), _dp(q))
    return q, ph


def _stage_end(pb):
    """What ends every Runge-Kutta stage: the relaxation for the six-equation
    model, nothing otherwise (also for pb = None, a bare ODE)."""
    return (lambda s: relax(pb, s)) if pb is not None and pb.model == "six" else (lambda s: s)


def rk3_step(pb: Problem, q, dt: float, rhs_fn=None):
    """One SSP-RK3 step in Shu-Osher form (Gottlieb & Shu 1998; Sec. 3.4):
    q1 = q + dt R(q); q2 = 3/4 q + 1/4 (q1 + dt R(q1)); q' = 1/3 q + 2/3 (q2 + dt R(q2)).
    Six-equation model: each of q1, q2 and q' is relaxed (Sec. 2.3: the
    hyperbolic update first, then the relaxation).
    """
    f = rhs_fn if rhs_fn is not None else (lambda s: rhs(pb, s))
    g = _stage_end(pb)
    q = np.asarray(q, dtype=np.float64)
    q1 = g(q + dt * f(q))
    q2 = g(0.75 * q + 0.25 * (q1 + dt * f(q1)))
    return g(q / 3.0 + (2.0 / 3.0) * (q2 + dt * f(q2)))


def rk_step(pb: Problem, q, dt: float, order: int = 3, rhs_fn=None):
    """One step of the SSP Runge-Kutta scheme of the given order (Sec. 3.4,
    Gottlieb & Shu TVD Runge-Kutta family): 1 = forward Euler;
    2 = q1 = q + dt R(q), q' = 1/2 q + 1/2 (q1 + dt R(q1)); 3 = rk3_step.
    Six-equation model: every stage is relaxed."""
    f = rhs_fn if rhs_fn is not None else (lambda s: rhs(pb, s))
    g = _stage_end(pb)
    q = np.asarray(q, dtype=np.float64)
    if order == 3:
        return rk3_step(pb, q, dt, rhs_fn=f)
    q1 = g(q + dt * f(q))
    if order == 1:
        return q1
    if order == 2:
        return g(0.5 * q + 0.5 * (q1 + dt * f(q1)))
    raise ValueError("order must be 1, 2 or 3")


def run(pb: Problem, q, t_end: float, cfl: float, max_steps: int = 10 ** 7, rk_order: int = 3):
    """March to t_end with CFL time steps, clipping the last step to hit t_end."""
    t = 0.0
    steps = 0
    q = np.array(q, dtype=np.float64)
    while t < t_end and steps < max_steps:
        dt = cfl_dt(pb, q, cfl)
        if t + dt > t_end:
            dt = t_end - t
        q = rk_step(pb, q, dt, rk_order)
        t += dt
        steps += 1
    return q, t, steps
