"""GB300 (sm_103a) right-hand side and SSP-RK3 step of the five-equation
diffuse-interface model with stiffened-gas fluids (arXiv 2305.09163).

Thin ctypes binding over the C ABI in ``include/mfc.h`` (``libmfc_gb300.so``):
the functions ``mfc_init`` ... ``mfc_finalize`` keep the C names and only
marshal arguments; every step of the computation runs in the library's CUDA
kernels.  ``Solver`` wraps a context for convenience.  Device buffers are torch
tensors (contiguous float64 on the context's GPU); host buffers are numpy
arrays.  There is no CPU fallback: if the library is missing or cannot load,
import of the binding functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

MFC_OK = 0
MFC_ERR_ARG, MFC_ERR_STATE_UNSET, MFC_ERR_OOM, MFC_ERR_CUDA, MFC_ERR_NONPHYSICAL, MFC_ERR_TIMEOUT = 1, 2, 3, 4, 5, 6
MFC_BC_PERIODIC, MFC_BC_TRANSMISSIVE, MFC_BC_REFLECTIVE, MFC_BC_CHARACTERISTIC = 0, 1, 2, 3
MFC_FP64, MFC_MIXED, MFC_LEARNED = 0, 1, 2
PRECISIONS = {"fp64": MFC_FP64, "mixed": MFC_MIXED, "learned": MFC_LEARNED}
PROFILE_CATEGORIES = ("prims", "sweep_x", "sweep_y", "sweep_z", "prims_cfl", "convert", "mlp", "boundary")
MLP_PARAMS = 32 * 5 + 32 + 32 * 32 + 32 + 3 * 32 + 3

_lib = None


class MFCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("mfc status %d: %s" % (status, msg))
        self.status = status


def library_path() -> str:
    return _build.LIB


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    return _build.build(force=force)


def _declare(lib):
    c_int, c_double, c_void_p, c_char_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_char_p
    c_ll = ctypes.c_longlong
    dptr = ctypes.POINTER(c_double)
    lib.mfc_init.argtypes = [ctypes.POINTER(c_void_p), c_int, c_int, c_int, dptr, dptr,
                             ctypes.POINTER(c_int), c_int, dptr, dptr, c_int, c_void_p]
    lib.mfc_init.restype = c_int
    lib.mfc_set_param.argtypes = [c_void_p, c_char_p, c_double]
    lib.mfc_set_param.restype = c_int
    for name in ("mfc_set_state", "mfc_set_state_prim", "mfc_get_state", "mfc_rhs"):
        f = getattr(lib, name)
        f.argtypes = [c_void_p, c_void_p, c_int]
        f.restype = c_int
    lib.mfc_step.argtypes = [c_void_p, c_double]
    lib.mfc_step.restype = c_int
    lib.mfc_cfl_dt.argtypes = [c_void_p, c_double, dptr]
    lib.mfc_cfl_dt.restype = c_int
    lib.mfc_set_mlp.argtypes = [c_void_p, ctypes.POINTER(ctypes.c_float), c_int]
    lib.mfc_set_mlp.restype = c_int
    lib.mfc_sys_size.argtypes = [c_void_p]
    lib.mfc_sys_size.restype = c_int
    lib.mfc_launch_count.argtypes = [c_void_p]
    lib.mfc_launch_count.restype = c_ll
    lib.mfc_fallback_count.argtypes = [c_void_p]
    lib.mfc_fallback_count.restype = c_ll
    lib.mfc_grid_table.argtypes = [c_void_p, c_int, c_int, c_void_p, ctypes.c_longlong]
    lib.mfc_grid_table.restype = c_int
    lib.mfc_set_grid.argtypes = [c_void_p, c_int, c_void_p, c_int]
    lib.mfc_set_grid.restype = c_int
    lib.mfc_network_rows.argtypes = [c_void_p]
    lib.mfc_network_rows.restype = c_ll
    lib.mfc_profile_read.argtypes = [c_void_p, dptr, ctypes.POINTER(c_ll), c_int]
    lib.mfc_profile_read.restype = c_int
    lib.mfc_rhs_noalloc.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, dptr, dptr, ctypes.POINTER(c_int),
                                    c_int, dptr, dptr, c_double, c_int, c_void_p, c_char_p, c_int]
    lib.mfc_rhs_noalloc.restype = c_int
    lib.mfc_get_prims.argtypes = [c_void_p, c_void_p, c_int]
    lib.mfc_get_prims.restype = c_int
    lib.mfc_mlp_forward.argtypes = [c_void_p, c_void_p, c_ll, c_void_p, c_void_p]
    lib.mfc_mlp_forward.restype = c_int
    lib.mfc_mlp_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_ll, ctypes.c_float,
                                 c_void_p, c_void_p, c_void_p, c_void_p]
    lib.mfc_mlp_grad.restype = c_int
    lib.mfc_mlp_grad_mma.argtypes = lib.mfc_mlp_grad.argtypes
    lib.mfc_mlp_grad_mma.restype = c_int
    lib.mfc_mlp_forward_tc.argtypes = [c_void_p, c_void_p, c_ll, c_void_p, c_void_p]
    lib.mfc_mlp_forward_tc.restype = c_int
    lib.mfc_mlp_tc_status.argtypes = []
    lib.mfc_mlp_tc_status.restype = c_int
    lib.mfc_mlp_adam.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float, c_int, c_void_p]
    lib.mfc_mlp_adam.restype = c_int
    lib.mfc_harvest.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_double, c_double, c_ll, ctypes.c_ulonglong,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.mfc_harvest.restype = c_int
    lib.mfc_last_error.argtypes = [c_void_p]
    lib.mfc_last_error.restype = c_char_p
    lib.mfc_finalize.argtypes = [c_void_p]
    lib.mfc_finalize.restype = None
    return lib


def load(build_if_missing: bool = True):
    """Load libmfc_gb300.so (building it first if it is absent or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise OSError("libmfc_gb300.so is not built (run paper_2305_09163_gb300.build())")
        _lib = _declare(ctypes.CDLL(_build.LIB))
    return _lib


def _ptr(buf):
    """(address, on_device) of a torch tensor or numpy array (float64, contiguous)."""
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.float64 or not buf.flags.c_contiguous:
            raise TypeError("host buffers must be contiguous float64 numpy arrays")
        return buf.ctypes.data, 0
    import torch
    if isinstance(buf, torch.Tensor):
        if buf.dtype != torch.float64 or not buf.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return buf.data_ptr(), 1 if buf.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(buf))


def _check(lib, ctx, status):
    if status != MFC_OK:
        msg = lib.mfc_last_error(ctx).decode() if ctx else ""
        raise MFCError(status, msg)


# ---- C ABI, same names -------------------------------------------------------
def mfc_init(n, lo, hi, bc, gamma, pi_inf, precision=MFC_FP64, stream=None):
    """Create a context; returns the opaque handle (an int)."""
    lib = load()
    n = list(n) + [1] * (3 - len(n))
    lo3 = (ctypes.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    hi3 = (ctypes.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
    bc6 = (ctypes.c_int * 6)(*(list(bc) + [1] * (6 - len(bc))))
    g = (ctypes.c_double * len(gamma))(*gamma)
    p = (ctypes.c_double * len(pi_inf))(*pi_inf)
    h = ctypes.c_void_p()
    st = lib.mfc_init(ctypes.byref(h), int(n[0]), int(n[1]), int(n[2]), lo3, hi3, bc6, len(gamma), g, p,
                      int(precision), ctypes.c_void_p(stream or 0))
    _check(lib, None, st)
    return h.value


def mfc_set_param(ctx, name, value):
    lib = load()
    _check(lib, ctx, lib.mfc_set_param(ctx, name.encode(), float(value)))


def mfc_set_state(ctx, q):
    lib = load()
    a, dev = _ptr(q)
    _check(lib, ctx, lib.mfc_set_state(ctx, a, dev))


def mfc_set_state_prim(ctx, w):
    lib = load()
    a, dev = _ptr(w)
    _check(lib, ctx, lib.mfc_set_state_prim(ctx, a, dev))


def mfc_get_state(ctx, q):
    lib = load()
    a, dev = _ptr(q)
    _check(lib, ctx, lib.mfc_get_state(ctx, a, dev))


def mfc_rhs(ctx, rhs):
    lib = load()
    a, dev = _ptr(rhs)
    _check(lib, ctx, lib.mfc_rhs(ctx, a, dev))


def mfc_step(ctx, dt):
    lib = load()
    _check(lib, ctx, lib.mfc_step(ctx, float(dt)))


def mfc_cfl_dt(ctx, cfl):
    lib = load()
    out = ctypes.c_double(0.0)
    _check(lib, ctx, lib.mfc_cfl_dt(ctx, float(cfl), ctypes.byref(out)))
    return out.value


def mfc_set_mlp(ctx, params):
    lib = load()
    params = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib, ctx, lib.mfc_set_mlp(ctx, params.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), params.size))


def mfc_sys_size(ctx):
    return load().mfc_sys_size(ctx)


def mfc_launch_count(ctx):
    return load().mfc_launch_count(ctx)


def mfc_fallback_count(ctx):
    return load().mfc_fallback_count(ctx)


def mfc_set_grid(ctx, direction, faces):
    """Face coordinates (n+1, increasing) of a non-uniform direction."""
    import numpy as np
    f = np.ascontiguousarray(faces, dtype=np.float64)
    lib = load()
    _check(lib, ctx, lib.mfc_set_grid(ctx, int(direction), f.ctypes.data, int(f.size)))


def mfc_grid_table(faces, periodic=False):
    """The per-cell WENO5 rows of a non-uniform direction as [n+2, 28, 2] float32."""
    import numpy as np
    f = np.ascontiguousarray(faces, dtype=np.float64)
    n = f.size - 1
    out = np.zeros((n + 2, 28, 2), dtype=np.float32)
    st = load().mfc_grid_table(f.ctypes.data, n, 1 if periodic else 0, out.ctypes.data, out.size)
    if st != 0:
        raise MFCError(MFC_ERR_ARG, "faces must be finite and strictly increasing")
    return out


def mfc_network_rows(ctx):
    return load().mfc_network_rows(ctx)


def mfc_profile_read(ctx):
    lib = load()
    ms = (ctypes.c_double * 8)()
    cnt = (ctypes.c_longlong * 8)()
    k = lib.mfc_profile_read(ctx, ms, cnt, 8)
    return {PROFILE_CATEGORIES[i]: (ms[i], cnt[i]) for i in range(min(k, len(PROFILE_CATEGORIES)))}


def mfc_get_prims(ctx, w):
    lib = load()
    a, dev = _ptr(w)
    _check(lib, ctx, lib.mfc_get_prims(ctx, a, dev))


MLP_GRAD_BLOCKS = 608
MLP_WORK_FLOATS = 608 * 4 * 1348


def _dev32(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def mfc_mlp_forward(params, x, omega, stream=None):
    """omega[B,3] = softmax weights of the network for inputs x[B,5] (device float32)."""
    lib = load()
    st = lib.mfc_mlp_forward(_dev32(params, "params"), _dev32(x, "x"), x.shape[0], _dev32(omega, "omega"),
                             _stream(stream))
    if st != MFC_OK:
        raise MFCError(st, "mfc_mlp_forward")


def mfc_mlp_forward_tc(params, x, omega, stream=None):
    """As mfc_mlp_forward, on the tcgen05 tensor cores."""
    lib = load()
    st = lib.mfc_mlp_forward_tc(_dev32(params, "params"), _dev32(x, "x"), x.shape[0], _dev32(omega, "omega"),
                                _stream(stream))
    if st != MFC_OK:
        raise MFCError(st, "mfc_mlp_forward_tc")


def _grad_call(fn, name, params, x, phat, target, mask, lam, grad, loss, work, stream):
    st = fn(_dev32(params, "params"), _dev32(x, "x"), _dev32(phat, "phat"), _dev32(target, "target"),
            _dev32(mask, "mask"), x.shape[0], float(lam), _dev32(grad, "grad"),
            _dev32(loss, "loss") if loss is not None else None, _dev32(work, "work"), _stream(stream))
    if st != MFC_OK:
        raise MFCError(st, name)


def mfc_mlp_grad(params, x, phat, target, mask, lam, grad, loss, work, stream=None):
    """Loss and gradient of a batch on the tcgen05 tensor cores."""
    _grad_call(load().mfc_mlp_grad, "mfc_mlp_grad", params, x, phat, target, mask, lam, grad, loss, work, stream)


def mfc_mlp_grad_mma(params, x, phat, target, mask, lam, grad, loss, work, stream=None):
    """The same on warp-level mma.sync tiles."""
    _grad_call(load().mfc_mlp_grad_mma, "mfc_mlp_grad_mma", params, x, phat, target, mask, lam, grad, loss, work,
               stream)


def mfc_mlp_tc_status():
    """1 if a bounded tensor-core wait gave up since the last call (then cleared), else 0 (synchronises)."""
    st = load().mfc_mlp_tc_status()
    if st < 0:
        raise MFCError(MFC_ERR_CUDA, "mfc_mlp_tc_status")
    return st


def mfc_mlp_adam(params, grad, m, v, lr, beta1, beta2, eps, step, stream=None):
    lib = load()
    st = lib.mfc_mlp_adam(_dev32(params, "params"), _dev32(grad, "grad"), _dev32(m, "m"), _dev32(v, "v"),
                          params.numel(), float(lr), float(beta1), float(beta2), float(eps), int(step),
                          _stream(stream))
    if st != MFC_OK:
        raise MFCError(st, "mfc_mlp_adam")


def mfc_harvest(w_fine, n_fine, num_fluids, weno_eps, tau, n_samples, seed, x, phat, target, smooth, js,
                stream=None):
    """Training samples from a fine primitive field (device float64 tensor)."""
    lib = load()
    wa, dev = _ptr(w_fine)
    if not dev:
        raise TypeError("w_fine must be a device tensor")
    n = list(n_fine) + [1] * (3 - len(n_fine))
    st = lib.mfc_harvest(wa, int(n[0]), int(n[1]), int(n[2]), int(num_fluids), float(weno_eps), float(tau),
                         int(n_samples), int(seed) & 0xFFFFFFFFFFFFFFFF, _dev32(x, "x"), _dev32(phat, "phat"),
                         _dev32(target, "target"), _dev32(smooth, "smooth"), _dev32(js, "js"), _stream(stream))
    if st != MFC_OK:
        raise MFCError(st, "mfc_harvest")


NOALLOC_MAX_CELLS = 262144


def mfc_rhs_noalloc(q, rhs, n, lo, hi, bc, gamma, pi_inf, weno_eps=1e-6, fallback=1, stream=None):
    """Allocation-free R(q) for callers that cannot let the library allocate
    device memory; q and rhs are device tensors (float64, contiguous) on the
    current CUDA device, each holding (2 N + d) * nx * ny * nz values (the C
    side trusts the pointers, so the sizes and the device are checked here)."""
    import torch
    lib = load()
    qa, qdev = _ptr(q)
    ra, rdev = _ptr(rhs)
    if not (qdev and rdev):
        raise TypeError("mfc_rhs_noalloc takes device buffers")
    n = list(n) + [1] * (3 - len(n))
    ndim = 3 if n[2] > 1 else (2 if n[1] > 1 else 1)
    need = (2 * len(gamma) + ndim) * int(n[0]) * int(n[1]) * int(n[2])
    if q.numel() != need or rhs.numel() != need:
        raise ValueError("mfc_rhs_noalloc: q and rhs must hold (2N + d) * cells = %d values (got %d and %d)"
                         % (need, q.numel(), rhs.numel()))
    cur = torch.cuda.current_device()
    if q.device.index != cur or rhs.device.index != cur:
        raise ValueError("mfc_rhs_noalloc: q and rhs must be on the current CUDA device (cuda:%d)" % cur)
    lo3 = (ctypes.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    hi3 = (ctypes.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
    bc6 = (ctypes.c_int * 6)(*(list(bc) + [1] * (6 - len(bc))))
    g = (ctypes.c_double * len(gamma))(*gamma)
    p = (ctypes.c_double * len(pi_inf))(*pi_inf)
    err = ctypes.create_string_buffer(512)
    st = lib.mfc_rhs_noalloc(qa, ra, int(n[0]), int(n[1]), int(n[2]), lo3, hi3, bc6, len(gamma), g, p,
                             float(weno_eps), int(fallback), ctypes.c_void_p(stream or 0), err, 512)
    if st != MFC_OK:
        raise MFCError(st, err.value.decode())


def mfc_last_error(ctx):
    return load().mfc_last_error(ctx).decode()


def mfc_finalize(ctx):
    if ctx:
        load().mfc_finalize(ctx)


# ---- convenience wrapper ----------------------------------------------------------
class Solver:
    """One context: grid, boundaries, fluids, precision, stream."""

    def __init__(self, n, lo, hi, bc, gamma, pi_inf, precision="fp64", stream=None, **params):
        import torch
        self.n = tuple(list(n) + [1] * (3 - len(n)))
        self.ndim = 3 if self.n[2] > 1 else (2 if self.n[1] > 1 else 1)
        self.nf = len(gamma)
        self.sys_size = 2 * self.nf + self.ndim
        self.shape = (self.sys_size, self.n[2], self.n[1], self.n[0])
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.ctx = mfc_init(self.n, lo, hi, bc, gamma, pi_inf, prec, stream)
        for k, v in params.items():
            self.set_param(k, v)

    def set_param(self, name, value):
        mfc_set_param(self.ctx, name, value)
        if name == "model":   # the six-equation model adds the phase internal energies
            self.sys_size = mfc_sys_size(self.ctx)
            self.shape = (self.sys_size, self.n[2], self.n[1], self.n[0])

    def set_state(self, q):
        mfc_set_state(self.ctx, q)

    def set_state_prim(self, w):
        mfc_set_state_prim(self.ctx, w)

    def get_state(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        mfc_get_state(self.ctx, out)
        return out

    def rhs(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        mfc_rhs(self.ctx, out)
        return out

    def step(self, dt):
        mfc_step(self.ctx, dt)

    def cfl_dt(self, cfl):
        return mfc_cfl_dt(self.ctx, cfl)

    def set_mlp(self, params):
        mfc_set_mlp(self.ctx, params)

    def get_prims(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        mfc_get_prims(self.ctx, out)
        return out

    def launch_count(self):
        return mfc_launch_count(self.ctx)

    def fallback_count(self):
        return mfc_fallback_count(self.ctx)

    def set_grid(self, direction, faces):
        mfc_set_grid(self.ctx, direction, faces)

    def network_rows(self):
        return mfc_network_rows(self.ctx)

    def profile(self):
        return mfc_profile_read(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            mfc_finalize(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
