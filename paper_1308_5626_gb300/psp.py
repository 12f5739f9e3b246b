"""ctypes binding of libpsp (the C ABI declared in include/psp.h).

Argument marshalling only: every function below forwards to the C entry point of the
same name, and every step of the solver runs in libpsp's CUDA kernels.  Device arrays are
passed as torch CUDA tensors (their data_ptr); the caller's current torch stream is the
stream handed to psp_create.

There is no CPU fallback: if libpsp.so is missing or was not built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsp.so")

PSP_OK, PSP_ERR_ARG, PSP_ERR_CUDA, PSP_ERR_OOM, PSP_ERR_NOCONV, PSP_ERR_NUMERIC, PSP_ERR_DEVICE = range(7)
PSP_SOLVER_GMRES, PSP_SOLVER_BICGSTAB = 0, 1
PSP_FP64, PSP_MIXED = 0, 1
PSP_FLAG_SINGULAR_FIT = 0x1
PSP_FLAG_CANDIDATE_TRIED = 0x2
PSP_FLAG_CANDIDATE_ACCEPTED = 0x4
PSP_FLAG_FACTOR_FAILED = 0x8
PSP_FLAG_BREAKDOWN = 0x10
PSP_FLAG_FITTED = 0x20
PSP_FLAG_DF_RESTART = 0x40

STATUS_NAMES = {0: "PSP_OK", 1: "PSP_ERR_ARG", 2: "PSP_ERR_CUDA", 3: "PSP_ERR_OOM", 4: "PSP_ERR_NOCONV",
                5: "PSP_ERR_NUMERIC", 6: "PSP_ERR_DEVICE"}


class psp_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("length", ctypes.c_double * 3)]


class psp_term(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("dir", ctypes.c_int), ("alpha", ctypes.c_double)]


class psp_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("intercept", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("max_hist_cols", ctypes.c_int), ("inner_tol", ctypes.c_double), ("accept_rule", ctypes.c_int),
                ("fuse_matvec", ctypes.c_int), ("adjoint", ctypes.c_int), ("cyclic", ctypes.c_int),
                ("solver", ctypes.c_int), ("onchip", ctypes.c_int), ("cycle_loop", ctypes.c_int)]


class psp_step_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("flags", ctypes.c_int), ("rel_res", ctypes.c_double), ("hist_cols", ctypes.c_int),
                ("singular_rows", ctypes.c_int), ("launches", ctypes.c_int)]


# kernel classes of psp_profile (index = class)
PSP_K_PRECOND, PSP_K_STENCIL, PSP_K_CGS1, PSP_K_CGS2, PSP_K_CGS3, PSP_K_COUNT = 0, 1, 2, 3, 4, 5
PSP_K_NAMES = ["precond", "stencil", "orth_dots", "unused", "orth_update"]


class psp_tuning_class(ctypes.Structure):
    _fields_ = [("log2_n", ctypes.c_int), ("choice", ctypes.c_int), ("samples", ctypes.c_int * 4),
                ("us_per_iter", ctypes.c_double * 4)]


class psp_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * PSP_K_COUNT), ("bytes", ctypes.c_double * PSP_K_COUNT),
                ("launches", ctypes.c_int64 * PSP_K_COUNT)]


# name -> (argtypes)
_VP = ctypes.c_void_p
_SIGS = {
    "psp_default_opts": [ctypes.POINTER(psp_opts)],
    "psp_create": [ctypes.POINTER(psp_grid), ctypes.c_int, ctypes.POINTER(psp_term), ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.POINTER(psp_opts), _VP, ctypes.POINTER(_VP)],
    "psp_destroy": [_VP],
    "psp_create_banded": [ctypes.c_int64, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(psp_opts), _VP,
                          ctypes.POINTER(_VP)],
    "psp_step": [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(psp_step_info)],
    "psp_step_host": [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(psp_step_info)],
    "psp_step_bdf2": [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(psp_step_info)],
    "psp_step_sdirk2": [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(psp_step_info)],
    "psp_matvec": [_VP, _VP, _VP, ctypes.c_double],
    "psp_matvec_f32": [_VP, _VP, _VP, ctypes.c_double],
    "psp_apply_L": [_VP, ctypes.c_int, _VP, _VP],
    "psp_step_batch": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                       ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_int, ctypes.POINTER(psp_step_info),
                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)],
    "psp_fit_band": [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_int)],
    "psp_fit_band_f32": [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_int)],
    "psp_get_history": [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "psp_set_band": [_VP, _VP],
    "psp_set_band_from": [_VP, _VP, ctypes.c_int],
    "psp_adjoint_grads": [_VP, _VP, _VP, ctypes.c_double, _VP],
    "psp_get_band": [_VP, _VP],
    "psp_apply_precond": [_VP, _VP, _VP, ctypes.c_int],
    "psp_apply_precond_f32": [_VP, _VP, _VP, ctypes.c_int],
    "psp_get_stencil": [_VP, _VP, ctypes.POINTER(ctypes.c_int)],
    "psp_reset": [_VP],
    "psp_set_profiling": [_VP, ctypes.c_int],
    "psp_get_profile": [_VP, ctypes.POINTER(psp_profile), ctypes.c_int],
    "psp_last_cycle_residuals": [_VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "psp_batch_tuner": [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "psp_fit_band_static": [_VP, _VP, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _VP,
                            ctypes.POINTER(ctypes.c_int), _VP],
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libpsp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpsp.so is not built; run paper_1308_5626_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, argtypes in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = argtypes
            fn.restype = ctypes.c_int
        L.psp_last_error.argtypes = []
        L.psp_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


class PspError(RuntimeError):
    """A failing call: `status` is the psp_status; the message is the library's
    psp_last_error() text, or `msg` for a refusal made by this binding before the call."""

    def __init__(self, status: int, where: str, msg: Optional[str] = None):
        if msg is None:
            msg = lib().psp_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))
        self.status = status


def _check(status: int, where: str, allow=(PSP_OK,)) -> int:
    if status not in allow:
        raise PspError(status, where)
    return status


def _ptr(t) -> int:
    return int(t.data_ptr())


# --------------------------------------------------------------------------------------
# thin wrappers with the C names
# --------------------------------------------------------------------------------------

def psp_default_opts() -> psp_opts:
    o = psp_opts()
    _check(lib().psp_default_opts(ctypes.byref(o)), "psp_default_opts")
    return o


def psp_create(shape: Sequence[int], order: int, terms: Sequence, b: int, m: int,
               opts: Optional[psp_opts] = None, stream: int = 0, lengths: Optional[Sequence[float]] = None):
    g = psp_grid()
    g.ndim = len(shape)
    for d in range(3):
        g.n[d] = int(shape[d]) if d < len(shape) else 1
        g.length[d] = float(lengths[d]) if lengths is not None and d < len(shape) else (2.0 * math.pi)
    tt = (psp_term * len(terms))()
    for i, t in enumerate(terms):
        k, d, a = (t.k, t.dir, t.alpha) if hasattr(t, "k") else t
        tt[i].k, tt[i].dir, tt[i].alpha = int(k), int(d), float(a)
    h = ctypes.c_void_p()
    _check(lib().psp_create(ctypes.byref(g), int(order), tt, len(terms), int(b), int(m),
                            ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(stream),
                            ctypes.byref(h)), "psp_create")
    return h


def psp_destroy(h) -> None:
    lib().psp_destroy(h)


def psp_step(h, u_n, u_np1, dt: float, tol: float, allow_noconv: bool = False) -> psp_step_info:
    info = psp_step_info()
    allow = (PSP_OK, PSP_ERR_NOCONV) if allow_noconv else (PSP_OK,)
    _check(lib().psp_step(h, _ptr(u_n), _ptr(u_np1), float(dt), float(tol), ctypes.byref(info)), "psp_step", allow)
    return info


def psp_step_bdf2(h, u_nm1, u_n, u_np1, dt: float, tol: float, allow_noconv: bool = False) -> psp_step_info:
    """BDF2 step (I - 2/3 dt L) u^{n+1} = (4 u^n - u^{n-1}) / 3; device float64 tensors."""
    info = psp_step_info()
    allow = (PSP_OK, PSP_ERR_NOCONV) if allow_noconv else (PSP_OK,)
    _check(lib().psp_step_bdf2(h, _ptr(u_nm1), _ptr(u_n), _ptr(u_np1), float(dt), float(tol), ctypes.byref(info)),
           "psp_step_bdf2", allow)
    return info


def psp_step_sdirk2(h, u_n, u_np1, dt: float, tol: float, allow_noconv: bool = False) -> psp_step_info:
    """Two-stage SDIRK step (gamma = 1 - 1/sqrt 2); device float64 tensors."""
    info = psp_step_info()
    allow = (PSP_OK, PSP_ERR_NOCONV) if allow_noconv else (PSP_OK,)
    _check(lib().psp_step_sdirk2(h, _ptr(u_n), _ptr(u_np1), float(dt), float(tol), ctypes.byref(info)),
           "psp_step_sdirk2", allow)
    return info


def psp_step_host(h, u_n_host, u_np1_host, dt: float, tol: float) -> psp_step_info:
    """u_n_host / u_np1_host: CPU tensors or numpy arrays of n float64 (contiguous)."""
    info = psp_step_info()
    pin = u_n_host.data_ptr() if hasattr(u_n_host, "data_ptr") else u_n_host.ctypes.data
    pout = u_np1_host.data_ptr() if hasattr(u_np1_host, "data_ptr") else u_np1_host.ctypes.data
    _check(lib().psp_step_host(h, ctypes.c_void_p(pin), ctypes.c_void_p(pout), float(dt), float(tol),
                               ctypes.byref(info)), "psp_step_host")
    return info


def psp_matvec(h, x, y, dt: float) -> None:
    fn = lib().psp_matvec_f32 if str(x.dtype) == "torch.float32" else lib().psp_matvec
    _check(fn(h, _ptr(x), _ptr(y), float(dt)), "psp_matvec")


def psp_step_batch(handles, u_n, u_np1, dt, tol: float, nthreads: int = 8, allow_noconv: bool = False):
    """One step of every handle (lists of equal length; u tensors float64 on the device).
    Returns (infos, seconds, statuses)."""
    cnt = len(handles)
    hs = (_VP * cnt)(*[h for h in handles])
    ui = (_VP * cnt)(*[_ptr(u) for u in u_n])
    uo = (_VP * cnt)(*[_ptr(u) for u in u_np1])
    dts = (ctypes.c_double * cnt)(*[float(d) for d in dt])
    infos = (psp_step_info * cnt)()
    secs = (ctypes.c_double * cnt)()
    sts = (ctypes.c_int * cnt)()
    st = lib().psp_step_batch(hs, cnt, ui, uo, dts, float(tol), int(nthreads), infos, secs, sts)
    if st != PSP_OK and not (allow_noconv and st == PSP_ERR_NOCONV):
        _check(st, "psp_step_batch")
    return list(infos), list(secs), list(sts)


def psp_batch_tuner(mode: int = -1):
    """Switch the batch autotuner on (1: and forget its measurements) or off (0), or only
    query it (-1); returns its table: one dict per size class seen."""
    arr = (psp_tuning_class * 32)()
    k = ctypes.c_int(0)
    _check(lib().psp_batch_tuner(int(mode), ctypes.cast(arr, ctypes.c_void_p), 32, ctypes.byref(k)), "psp_batch_tuner")
    names = ["graphs", "onchip128", "onchip256", "onchip512"]
    out = []
    for c in arr[:k.value]:
        out.append({"log2_n": c.log2_n, "choice": {-1: None, 0: "graphs"}.get(c.choice, "onchip%d" % c.choice),
                    "samples": dict(zip(names, list(c.samples))),
                    "us_per_iter": dict(zip(names, [round(v, 3) for v in c.us_per_iter]))})
    return out


def psp_apply_L(h, term: int, x, y) -> None:
    """y = L x (term < 0) or the unit-alpha derivative of term `term` (FP64 tensors)."""
    _check(lib().psp_apply_L(h, int(term), _ptr(x), _ptr(y)), "psp_apply_L")


def psp_fit_band(h, Px, Py, N_band, ld: Optional[int] = None, M: Optional[int] = None) -> int:
    """Px, Py: torch tensors shaped (M, ld) (row c = history column c); returns singular rows."""
    M = int(Px.shape[0]) if M is None else int(M)
    ld = int(Px.shape[1]) if ld is None else int(ld)
    sing = ctypes.c_int(0)
    fn = lib().psp_fit_band_f32 if str(Px.dtype) == "torch.float32" else lib().psp_fit_band
    _check(fn(h, _ptr(Px), _ptr(Py), ld, M, _ptr(N_band), ctypes.byref(sing)), "psp_fit_band")
    return sing.value


def psp_fit_band_static(Px, Py, N_band, b: int, intercept: int = 1, ld: Optional[int] = None,
                        M: Optional[int] = None, n: Optional[int] = None, stream: int = 0,
                        want_count: bool = True) -> Optional[int]:
    """Allocation-free band fit (no handle).  Px, Py: contiguous float64 CUDA tensors shaped
    (M, ld) (row c = history column c), N_band: contiguous float64 CUDA tensor of at least
    n (2b+1) values.  Returns the number of degenerate rows, or None with want_count=False
    (required while the stream is captured into a graph).  Tensors of another dtype, device
    or shape are refused here, before any pointer reaches the library."""
    import torch
    for name, t in (("Px", Px), ("Py", Py), ("N_band", N_band)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise PspError(PSP_ERR_ARG, "psp_fit_band_static", "%s must be a contiguous float64 CUDA tensor" % name)
    if Px.dim() != 2 or Py.shape != Px.shape:
        raise PspError(PSP_ERR_ARG, "psp_fit_band_static", "Px and Py must both be shaped (M, ld)")
    M = int(Px.shape[0]) if M is None else int(M)
    ld = int(Px.shape[1]) if ld is None else int(ld)
    n = ld if n is None else int(n)
    if not (1 <= M <= Px.shape[0] and n <= ld <= Px.shape[1] and n >= 1 and 1 <= int(b)):
        raise PspError(PSP_ERR_ARG, "psp_fit_band_static", "need 1 <= M <= rows and n <= ld <= columns of Px")
    if N_band.numel() < n * (2 * int(b) + 1):
        raise PspError(PSP_ERR_ARG, "psp_fit_band_static", "N_band holds fewer than n (2b+1) values")
    sing = ctypes.c_int(0)
    _check(lib().psp_fit_band_static(_ptr(Px), _ptr(Py), ld, M, n, int(b), int(intercept), _ptr(N_band),
                                     ctypes.byref(sing) if want_count else None, ctypes.c_void_p(stream)),
           "psp_fit_band_static")
    return sing.value if want_count else None


def psp_get_history(h, n: int):
    """The handle's matvec history, oldest pair first: (Px, Py) float64 CUDA tensors shaped
    (cols, n) (row c = history column c)."""
    import torch
    c = ctypes.c_int(0)
    _check(lib().psp_get_history(h, None, None, int(n), 0, ctypes.byref(c)), "psp_get_history")
    Px = torch.empty((max(c.value, 1), n), dtype=torch.float64, device="cuda")
    Py = torch.empty_like(Px)
    _check(lib().psp_get_history(h, _ptr(Px), _ptr(Py), int(n), c.value, ctypes.byref(c)), "psp_get_history")
    return Px[:c.value], Py[:c.value]


def psp_set_band(h, N_band) -> None:
    _check(lib().psp_set_band(h, _ptr(N_band)), "psp_set_band")


def psp_set_band_from(dst, src, transpose: int = 1) -> None:
    """Adopt src's preconditioner (transposed with transpose=1) in dst."""
    _check(lib().psp_set_band_from(dst, src, int(transpose)), "psp_set_band_from")


def psp_adjoint_grads(h, lam, u, dt: float, nterms: int):
    """[dLoss/d dt, dLoss/d alpha_0, ...] of one implicit step from the adjoint state lam and
    u^{n+1} (FP64 device tensors); a list of 1 + nterms floats."""
    g = (ctypes.c_double * (1 + int(nterms)))()
    _check(lib().psp_adjoint_grads(h, _ptr(lam), _ptr(u), float(dt), g), "psp_adjoint_grads")
    return list(g)


def psp_get_band(h, N_band) -> None:
    _check(lib().psp_get_band(h, _ptr(N_band)), "psp_get_band")


def psp_apply_precond(h, v, y, transpose: int = 0) -> None:
    fn = lib().psp_apply_precond_f32 if str(v.dtype) == "torch.float32" else lib().psp_apply_precond
    _check(fn(h, _ptr(v), _ptr(y), int(transpose)), "psp_apply_precond")


def psp_get_stencil(h):
    r = ctypes.c_int(0)
    _check(lib().psp_get_stencil(h, None, ctypes.byref(r)), "psp_get_stencil")
    w = (ctypes.c_double * (3 * (2 * r.value + 1)))()
    _check(lib().psp_get_stencil(h, w, ctypes.byref(r)), "psp_get_stencil")
    R = r.value
    return [[w[d * (2 * R + 1) + j] for j in range(2 * R + 1)] for d in range(3)], R


def psp_reset(h) -> None:
    _check(lib().psp_reset(h), "psp_reset")


def psp_set_profiling(h, enable: bool) -> None:
    _check(lib().psp_set_profiling(h, int(bool(enable))), "psp_set_profiling")


def psp_last_cycle_residuals(h, maxk: int = 64):
    R = (ctypes.c_double * maxk)()
    k = ctypes.c_int(0)
    _check(lib().psp_last_cycle_residuals(h, R, int(maxk), ctypes.byref(k)), "psp_last_cycle_residuals")
    return [R[i] for i in range(min(k.value, maxk))]


def psp_get_profile(h, reset: bool = False) -> dict:
    p = psp_profile()
    _check(lib().psp_get_profile(h, ctypes.byref(p), int(bool(reset))), "psp_get_profile")
    return {name: {"ms": p.ms[i], "bytes": p.bytes[i], "launches": int(p.launches[i])}
            for i, name in enumerate(PSP_K_NAMES)}


# --------------------------------------------------------------------------------------
# convenience: a handle bound to torch tensors
# --------------------------------------------------------------------------------------

def _opts(precision, intercept, max_restarts, max_hist_cols, inner_tol, accept_rule, fuse_matvec, adjoint, cyclic=0,
          solver=0, onchip=-1, cycle_loop=0):
    o = psp_default_opts()
    o.precision, o.intercept, o.max_restarts = int(precision), int(intercept), int(max_restarts)
    o.max_hist_cols, o.inner_tol, o.accept_rule = int(max_hist_cols), float(inner_tol), int(accept_rule)
    o.fuse_matvec, o.adjoint, o.cyclic, o.solver = int(fuse_matvec), int(adjoint), int(cyclic), int(solver)
    o.onchip = int(onchip)
    o.cycle_loop = int(cycle_loop)
    return o


def psp_create_banded(n: int, A_band, w: int, b: int, m: int, opts: psp_opts, stream: int = 0):
    """Handle for an explicit banded operator (A_band: device float64 tensor, n x (2w+1))."""
    out = _VP()
    _check(lib().psp_create_banded(int(n), _ptr(A_band), int(w), int(b), int(m), ctypes.byref(opts),
                                   _VP(stream), ctypes.byref(out)), "psp_create_banded")
    return out


class Solver:
    """Owns one psp handle for a workload; vectors are torch CUDA float64 tensors."""

    def __init__(self, shape, order, terms, b, m, precision=PSP_FP64, intercept=1, max_restarts=200,
                 max_hist_cols=0, inner_tol=1e-5, accept_rule=1, fuse_matvec=1, adjoint=0, stream=None, cyclic=0,
                 solver=0, onchip=-1, cycle_loop=0):
        import torch
        o = _opts(precision, intercept, max_restarts, max_hist_cols, inner_tol, accept_rule, fuse_matvec, adjoint,
                  cyclic, solver, onchip, cycle_loop)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self.shape = tuple(int(v) for v in shape)
        self.n = 1
        for v in self.shape:
            self.n *= v
        self.b = int(b)
        self.handle = psp_create(self.shape, order, terms, b, m, o, int(s.cuda_stream))

    @classmethod
    def banded(cls, A_band, w, b, m, precision=PSP_FP64, intercept=1, max_restarts=200, max_hist_cols=0,
               inner_tol=1e-5, accept_rule=1, adjoint=0, stream=None, onchip=-1, cycle_loop=0):
        """A solver whose operator is the explicit banded matrix A_band (device float64, n x (2w+1))."""
        import torch
        obj = cls.__new__(cls)
        o = _opts(precision, intercept, max_restarts, max_hist_cols, inner_tol, accept_rule, 0, adjoint, 0, 0, onchip,
                  cycle_loop)
        s = stream if stream is not None else torch.cuda.current_stream()
        obj.stream = s
        obj.n = A_band.numel() // (2 * int(w) + 1)
        obj.shape = (obj.n,)
        obj.b = int(b)
        obj.handle = psp_create_banded(obj.n, A_band.contiguous(), w, b, m, o, int(s.cuda_stream))
        return obj

    def step(self, u_n, dt, tol, out=None, allow_noconv=False):
        import torch
        out = torch.empty_like(u_n) if out is None else out
        info = psp_step(self.handle, u_n, out, dt, tol, allow_noconv)
        return out, info

    def step_bdf2(self, u_nm1, u_n, dt, tol, out=None, allow_noconv=False):
        import torch
        out = torch.empty_like(u_n) if out is None else out
        info = psp_step_bdf2(self.handle, u_nm1, u_n, out, dt, tol, allow_noconv)
        return out, info

    def step_sdirk2(self, u_n, dt, tol, out=None, allow_noconv=False):
        import torch
        out = torch.empty_like(u_n) if out is None else out
        info = psp_step_sdirk2(self.handle, u_n, out, dt, tol, allow_noconv)
        return out, info

    def close(self):
        if self.handle is not None:
            psp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workload_dt(w) -> float:
    """A workload's time step: w.dt, or for a spectral-radius rule (rho(L) dt = w.rho_dt)
    rho = max |lambda| of the library's own stencil of L (psp_get_stencil) over the grid's
    Fourier modes, lambda(theta) = sum_d sum_j w_dj e^{i j theta_d}."""
    if w.dt is not None:
        return float(w.dt)
    import numpy as np
    s = Solver(w.shape, w.order, w.terms, w.b, 2, max_hist_cols=4)
    wst, R = psp_get_stencil(s.handle)
    s.close()
    lam = np.zeros(tuple(reversed(w.shape)), dtype=np.complex128)
    for d, nd in enumerate(w.shape):
        th = 2.0 * np.pi * np.arange(nd) / nd
        ld = sum(wst[d][j + R] * np.exp(1j * j * th) for j in range(-R, R + 1))
        shp = [1] * len(w.shape)
        shp[len(w.shape) - 1 - d] = nd
        lam = lam + ld.reshape(shp)
    return float(w.rho_dt / np.abs(lam).max())
