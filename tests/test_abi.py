"""The C ABI library builds for sm_103a, loads without a GPU and exports every entry point
that include/psp.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "psp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:psp_status|const char \*|void)\s*\*?\s*(psp_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpsp():
    from paper_1308_5626_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("psp_create", "psp_step", "psp_fit_band", "psp_apply_precond", "psp_destroy",
              "psp_get_band", "psp_set_band", "psp_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(libpsp):
    for name in _declared():
        assert hasattr(libpsp, name), name


def test_binding_covers_the_header():
    from paper_1308_5626_gb300 import psp
    for name in _declared():
        if name in ("psp_last_error",):
            continue
        assert name in psp._SIGS, name


def test_binding_constants_match_the_header():
    """Every #define PSP_* value of include/psp.h (status codes, precisions, flags) is the
    binding's constant of the same name."""
    import os
    import re
    from paper_1308_5626_gb300 import psp
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "psp.h")).read()
    found = re.findall(r"^#define (PSP_[A-Z0-9_]+) +(0x[0-9a-fA-F]+|[0-9]+)\b", hdr, re.M)
    found += re.findall(r"\b(PSP_[A-Z0-9_]+) = (0x[0-9a-fA-F]+|[0-9]+)\b", hdr)   # enumerators
    assert len(found) >= 15
    for name, val in found:
        assert hasattr(psp, name), name
        assert getattr(psp, name) == int(val, 0), name


def test_default_opts_without_gpu(libpsp):
    from paper_1308_5626_gb300 import psp
    o = psp.psp_default_opts()
    assert o.precision == psp.PSP_FP64 and o.intercept == 1 and o.max_restarts == 200
    assert o.accept_rule == 1 and abs(o.inner_tol - 1e-5) < 1e-20
    assert o.fuse_matvec == 1


def test_argument_errors_need_no_gpu(libpsp):
    from paper_1308_5626_gb300 import psp
    h = ctypes.c_void_p()
    st = psp.lib().psp_create(None, 4, None, 0, 2, 30, None, None, ctypes.byref(h))
    assert st == psp.PSP_ERR_ARG
    assert b"NULL" in psp.lib().psp_last_error()
    assert psp.lib().psp_step(None, None, None, 0.1, 1e-8, None) == psp.PSP_ERR_ARG


NULL_HANDLE_CALLS = ["psp_default_opts", "psp_step", "psp_step_host", "psp_step_bdf2", "psp_step_sdirk2",
                     "psp_matvec", "psp_matvec_f32", "psp_apply_L", "psp_fit_band", "psp_fit_band_f32",
                     "psp_get_history", "psp_set_band", "psp_set_band_from", "psp_adjoint_grads", "psp_get_band",
                     "psp_apply_precond", "psp_apply_precond_f32", "psp_get_stencil", "psp_reset",
                     "psp_set_profiling", "psp_get_profile", "psp_last_cycle_residuals", "psp_fit_band_static",
                     "psp_create_banded"]


@pytest.mark.parametrize("name", NULL_HANDLE_CALLS)
def test_null_arguments_are_refused_without_gpu(libpsp, name):
    """Every entry point called with NULL pointers (and a NULL handle where it takes one)
    returns PSP_ERR_ARG with a message, before touching the device; psp_destroy(NULL) is a
    no-op that returns PSP_OK."""
    from paper_1308_5626_gb300 import psp
    fn = getattr(psp.lib(), name)
    args = [0.1 if t is ctypes.c_double else (1 if t in (ctypes.c_int, ctypes.c_int64) else None)
            for t in fn.argtypes]
    assert fn(*args) == psp.PSP_ERR_ARG
    assert len(psp.lib().psp_last_error()) > 0
    assert psp.lib().psp_destroy(None) == psp.PSP_OK


def test_batch_entry_points_without_gpu(libpsp):
    """The batch call refuses NULL arrays, a negative count and a non-positive tolerance, and
    an empty batch does nothing; the tuner's switch and report are host state (a fresh tuner
    has measured no class) and an unknown mode is refused."""
    from paper_1308_5626_gb300 import psp
    L = psp.lib()
    assert L.psp_step_batch(None, 1, None, None, None, 1e-8, 4, None, None, None) == psp.PSP_ERR_ARG
    hs = (ctypes.c_void_p * 1)()
    ui = (ctypes.c_void_p * 1)()
    uo = (ctypes.c_void_p * 1)()
    dts = (ctypes.c_double * 1)(0.1)
    assert L.psp_step_batch(hs, -1, ui, uo, dts, 1e-8, 4, None, None, None) == psp.PSP_ERR_ARG
    assert L.psp_step_batch(hs, 0, ui, uo, dts, 0.0, 4, None, None, None) == psp.PSP_ERR_ARG
    assert L.psp_step_batch(hs, 1, ui, uo, dts, 1e-8, 4, None, None, None) == psp.PSP_ERR_ARG   # NULL handle
    assert L.psp_step_batch(hs, 0, ui, uo, dts, 1e-8, 4, None, None, None) == psp.PSP_OK
    k = ctypes.c_int(-1)
    assert L.psp_batch_tuner(1, None, 0, ctypes.byref(k)) == psp.PSP_OK and k.value == 0
    assert L.psp_batch_tuner(-1, None, 0, ctypes.byref(k)) == psp.PSP_OK and k.value == 0
    assert L.psp_batch_tuner(0, None, 0, None) == psp.PSP_OK
    assert L.psp_batch_tuner(2, None, 0, None) == psp.PSP_ERR_ARG


def test_opts_layout_matches_the_header(libpsp):
    """psp_default_opts writes exactly the ctypes psp_opts: a C struct with a field the
    binding lacks would write past it (guard bytes), and the new options default to off."""
    from paper_1308_5626_gb300 import psp
    size = ctypes.sizeof(psp.psp_opts)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    assert psp.lib().psp_default_opts(ctypes.cast(buf, ctypes.POINTER(psp.psp_opts))) == psp.PSP_OK
    assert all(b == 0xAB for b in bytes(buf)[size:])
    o = psp.psp_opts.from_buffer_copy(bytes(buf)[:size])
    assert o.adjoint == 0 and o.cyclic == 0 and o.solver == psp.PSP_SOLVER_GMRES
    assert o.onchip == -1 and o.cycle_loop == 0


def _create(shape, order=2, b=2, m=8, **opt):
    from paper_1308_5626_gb300 import psp
    g = psp.psp_grid()
    g.ndim = len(shape)
    for d in range(3):
        g.n[d] = shape[d] if d < len(shape) else 1
        g.length[d] = 6.283185307179586
    t = (psp.psp_term * 1)()
    t[0].k, t[0].dir, t[0].alpha = 2, 0, 1.0
    o = psp.psp_default_opts()
    for k, v in opt.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    return psp.lib().psp_create(ctypes.byref(g), order, t, 1, b, m, ctypes.byref(o), None, ctypes.byref(h))


@pytest.mark.parametrize("shape,kw,what", [
    ((1 << 16, 1 << 16), {}, b"2^31"),                                    # 2^32 unknowns
    ((64, 64), {"cyclic": 1}, b"cyclic"),                                 # cyclic band off a 1D grid
    ((9,), {"cyclic": 1}, b"cyclic"),                                     # n < 4b + 2
    ((64,), {"solver": 1, "precision": 1}, b"BiCGSTAB"),                  # BiCGSTAB in the mixed form
    ((64,), {"solver": 1, "m": 2}, b"BiCGSTAB"),                          # m < 3
    ((64,), {"solver": 7}, b"solver"),
    ((64,), {"precision": 5}, b"precision"),
    ((0,), {}, b"positive"),                                              # empty grid
    ((4,), {}, b"2b+1"),                                                  # n < 2b + 1
    ((64,), {"m": 65}, b"restart length"),                                # m above 64
])
def test_create_refuses_bad_arguments_without_gpu(libpsp, shape, kw, what):
    from paper_1308_5626_gb300 import psp
    m = kw.pop("m", 8)
    assert _create(shape, m=m, **kw) == psp.PSP_ERR_ARG
    assert what in psp.lib().psp_last_error()


def test_static_fit_binding_refuses_host_and_fp32_tensors():
    """The allocation-free fit's binding passes raw pointers to an FP64-only kernel: tensors
    that are not contiguous float64 CUDA tensors (here CPU and FP32 ones) are refused with
    PSP_ERR_ARG before the library is called (no GPU needed)."""
    import torch
    from paper_1308_5626_gb300 import psp
    x = torch.zeros((4, 100), dtype=torch.float64)
    out = torch.zeros((100, 3), dtype=torch.float64)
    for args in ((x, x, out), (x.float(), x.float(), out)):
        with pytest.raises(psp.PspError) as e:
            psp.psp_fit_band_static(*args, 1)
        assert e.value.status == psp.PSP_ERR_ARG
