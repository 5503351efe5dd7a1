"""Python binding of libamg (ctypes): the coarse-grid correction of DD-alpha-AMG on GB300.

Argument marshalling only.  Every function has the name of the C entry point
it calls (include/amg.h); pointers may be given as ints, torch tensors
(``data_ptr()``), numpy arrays (host memory, where the C function accepts
host memory) or None.  A non-zero status raises ``AmgError`` except where a
function documents otherwise.  The library must have been built
(``__graft_entry__.build()``); importing this module without it fails.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libamg.so")

AMG_OK = 0
AMG_ERR_INVALID_ARG = 1
AMG_ERR_UNSUPPORTED = 2
AMG_ERR_OOM = 3
AMG_ERR_CUDA = 4
AMG_ERR_TIMEOUT = 5
AMG_ERR_RANK_DEFICIENT = 6
AMG_ERR_NONFINITE = 7

AMG_FP64 = 0
AMG_FP32 = 1
AMG_FP16_SCALED = 2
AMG_BF16 = 3

AMG_SETUP_FP64 = 0
AMG_SETUP_F32PAIR = 1


class amg_params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int * 4),
        ("B", ctypes.c_int * 4),
        ("ntv", ctypes.c_int),
        ("max_nrhs", ctypes.c_int),
        ("m0", ctypes.c_double),
        ("csw", ctypes.c_double),
        ("link_prec", ctypes.c_int),
        ("r_prec", ctypes.c_int),
        ("vec_prec", ctypes.c_int),
        ("setup_arith", ctypes.c_int),
    ]


class amg_vcycle_params(ctypes.Structure):
    _fields_ = [
        ("coarse_tol", ctypes.c_double),
        ("coarse_restart", ctypes.c_int),
        ("coarse_max_applies", ctypes.c_int),
        ("n_smoother", ctypes.c_int),
        ("n_mr", ctypes.c_int),
    ]


class amg_level2_params(ctypes.Structure):
    _fields_ = [
        ("n_mr", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("max_applies", ctypes.c_int),
        ("tol", ctypes.c_double),
    ]


class AmgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = amg_last_error() if status in (AMG_ERR_CUDA, AMG_ERR_OOM, AMG_ERR_INVALID_ARG) else ""
        super().__init__("%s: %s (status %d) %s" % (where, amg_status_string(status), status, detail))


if not os.path.exists(_LIB_PATH):
    raise ImportError("libamg.so is not built (run __graft_entry__.build()); there is no fallback")
lib = ctypes.CDLL(_LIB_PATH)

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_proto = {
    "amg_setup_coarse": [ctypes.POINTER(amg_params), _vp, _vp, _vp, ctypes.POINTER(_vp)],
    "amg_restrict": [_vp, _vp, _vp, _i, _vp],
    "amg_coarse_apply": [_vp, _vp, _vp, _i, _vp],
    "amg_prolong": [_vp, _vp, _vp, _i, _vp],
    "amg_coarse_solve": [_vp, _vp, _vp, _i, _d, _i, _i, _vp, ctypes.POINTER(_d)],
    "amg_coarse_solve_noalloc": [_vp, _vp, _vp, _i, _d, _i, _i, _vp, ctypes.POINTER(_d)],
    "amg_coarse_solve_mixed": [_vp, _vp, _vp, _vp, _i, _d, _d, _i, _i, _i, _vp, ctypes.POINTER(_d)],
    "amg_cgc": [_vp, _vp, _vp, _i, _d, _i, _i, _vp, ctypes.POINTER(_d)],
    "amg_setup_evenodd": [_vp, _vp],
    "amg_schur_apply": [_vp, _vp, _vp, _i, _vp],
    "amg_coarse_solve_eo": [_vp, _vp, _vp, _i, _d, _i, _i, _vp, ctypes.POINTER(_d)],
    "amg_cgc_eo": [_vp, _vp, _vp, _i, _d, _i, _i, _vp, ctypes.POINTER(_d)],
    "amg_export_Dinv": [_vp, _vp],
    "amg_setup_fine": [_vp, _vp, _vp],
    "amg_dirac_apply": [_vp, _vp, _vp, _i, _vp],
    "amg_sap": [_vp, _vp, _vp, _i, _i, _i, _vp],
    "amg_vcycle": [_vp, ctypes.POINTER(amg_vcycle_params), _vp, _vp, _i, _vp],
    "amg_adaptive_setup": [_vp, ctypes.POINTER(amg_vcycle_params), _vp, _vp, _i, _vp],
    "amg_solve": [_vp, ctypes.POINTER(amg_vcycle_params), _vp, _vp, _i, _d, _i, _i, _vp, ctypes.POINTER(_d)],
    "amg_batch_cgc": [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                      ctypes.POINTER(_i), _vp],
    "amg_batch_autotune": [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                           ctypes.POINTER(_i), _vp, ctypes.POINTER(_d)],
    "amg_batch_test_hook": [_vp, _i],
    "amg_solve_test_hook": [_vp, _i],
    "amg_grid_cap_test_hook": [_vp, _i],
    "amg_setup_level2": [_vp, ctypes.POINTER(amg_params), _vp, _vp, ctypes.POINTER(_vp)],
    "amg_restrict2": [_vp, _vp, _vp, _i, _vp],
    "amg_prolong2": [_vp, _vp, _vp, _i, _vp],
    "amg_attach_level2": [_vp, _vp, ctypes.POINTER(amg_level2_params)],
    "amg_two_grid": [_vp, _vp, _vp, _i, _vp],
    "amg_export_R": [_vp, _vp],
    "amg_export_Dc": [_vp, _vp],
    "amg_export_clover": [_vp, _vp],
    "amg_export_Dc_stored": [_vp, _vp],
    "amg_setup_timings": [_vp, ctypes.POINTER(_d)],
    "amg_kernel_launches": [_vp, ctypes.POINTER(ctypes.c_ulonglong)],
    "amg_sync_status": [_vp],
    "amg_destroy": [_vp],
}
for _name, _args in _proto.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
lib.amg_status_string.argtypes = [ctypes.c_int]
lib.amg_status_string.restype = ctypes.c_char_p
lib.amg_last_error.argtypes = []
lib.amg_last_error.restype = ctypes.c_char_p
lib.amg_noalloc_scratch_bytes.argtypes = []
lib.amg_noalloc_scratch_bytes.restype = ctypes.c_size_t

EXPORTED = sorted(list(_proto) + ["amg_status_string", "amg_last_error", "amg_noalloc_scratch_bytes"])


def amg_noalloc_scratch_bytes():
    return lib.amg_noalloc_scratch_bytes()


def amg_last_error():
    return lib.amg_last_error().decode()


def amg_status_string(status):
    return lib.amg_status_string(int(status)).decode()


def ptr(x):
    """Address of a buffer: int, None, torch tensor or numpy array."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def stream_ptr(s):
    """cudaStream_t of a torch stream, an int handle, or None (legacy default stream)."""
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status, where, allow=()):
    if status != AMG_OK and status not in allow:
        raise AmgError(status, where)
    return status


def make_params(L, B, ntv, max_nrhs=1, m0=-0.3, csw=1.0, link_prec=AMG_FP32, r_prec=AMG_FP32,
                vec_prec=AMG_FP32, setup_arith=AMG_SETUP_FP64):
    p = amg_params()
    p.L[:] = list(L)
    p.B[:] = list(B)
    p.ntv = ntv
    p.max_nrhs = max_nrhs
    p.m0 = m0
    p.csw = csw
    p.link_prec = link_prec
    p.r_prec = r_prec
    p.vec_prec = vec_prec
    p.setup_arith = setup_arith
    return p


def amg_setup_coarse(params, U, tv, stream=None, allow_rank_deficient=False):
    """Returns (handle, status); raises on any error except, when allowed, rank deficiency."""
    h = _vp()
    st = lib.amg_setup_coarse(ctypes.byref(params), ptr(U), ptr(tv), stream_ptr(stream), ctypes.byref(h))
    _check(st, "amg_setup_coarse", (AMG_ERR_RANK_DEFICIENT,) if allow_rank_deficient else ())
    return h.value, st


def amg_restrict(h, y, yc, nrhs=1, stream=None):
    return _check(lib.amg_restrict(h, ptr(y), ptr(yc), nrhs, stream_ptr(stream)), "amg_restrict")


def amg_coarse_apply(h, xc, yc, nrhs=1, stream=None):
    return _check(lib.amg_coarse_apply(h, ptr(xc), ptr(yc), nrhs, stream_ptr(stream)), "amg_coarse_apply")


def amg_prolong(h, xc, x, nrhs=1, stream=None):
    return _check(lib.amg_prolong(h, ptr(xc), ptr(x), nrhs, stream_ptr(stream)), "amg_prolong")


def _info(nrhs, want):
    return (ctypes.c_double * (2 * nrhs))() if want else None


def _info_out(info, nrhs):
    if info is None:
        return None
    return [(int(info[2 * r]), float(info[2 * r + 1])) for r in range(nrhs)]


def amg_coarse_solve(h, b, x, nrhs=1, tol=0.05, restart=30, max_applies=200, stream=None, info=True):
    """Returns [(applies, implicit relative residual)] per right-hand side when info is True."""
    buf = _info(nrhs, info)
    _check(lib.amg_coarse_solve(h, ptr(b), ptr(x), nrhs, tol, restart, max_applies, stream_ptr(stream), buf),
           "amg_coarse_solve")
    return _info_out(buf, nrhs)


def amg_coarse_solve_noalloc(h, b, x, nrhs=1, tol=0.05, restart=30, max_applies=200, stream=None, info=True):
    """amg_coarse_solve on the library's fixed scratch array: allocates no device memory."""
    buf = _info(nrhs, info)
    _check(lib.amg_coarse_solve_noalloc(h, ptr(b), ptr(x), nrhs, tol, restart, max_applies,
                                        stream_ptr(stream), buf), "amg_coarse_solve_noalloc")
    return _info_out(buf, nrhs)


def amg_coarse_solve_mixed(h_outer, h_inner, b, x, nrhs=1, tol=1e-4, inner_tol=0.05, restart=30,
                           max_inner_applies=200, max_outer=20, stream=None, info=True):
    """Returns [(inner applications, outer passes, true relative residual)] per right-hand side."""
    buf = (ctypes.c_double * (3 * nrhs))() if info else None
    _check(lib.amg_coarse_solve_mixed(h_outer, h_inner, ptr(b), ptr(x), nrhs, tol, inner_tol, restart,
                                      max_inner_applies, max_outer, stream_ptr(stream), buf),
           "amg_coarse_solve_mixed")
    if buf is None:
        return None
    return [(int(buf[3 * r]), int(buf[3 * r + 1]), float(buf[3 * r + 2])) for r in range(nrhs)]


def amg_cgc(h, y, x, nrhs=1, tol=0.05, restart=30, max_applies=200, stream=None, info=True):
    buf = _info(nrhs, info)
    _check(lib.amg_cgc(h, ptr(y), ptr(x), nrhs, tol, restart, max_applies, stream_ptr(stream), buf), "amg_cgc")
    return _info_out(buf, nrhs)


def make_vcycle_params(coarse_tol=0.05, coarse_restart=30, coarse_max_applies=200, n_smoother=4, n_mr=4):
    return amg_vcycle_params(coarse_tol, coarse_restart, coarse_max_applies, n_smoother, n_mr)


def amg_setup_fine(h, U, stream=None):
    return _check(lib.amg_setup_fine(h, ptr(U), stream_ptr(stream)), "amg_setup_fine")


def amg_dirac_apply(h, psi, out, nrhs=1, stream=None):
    return _check(lib.amg_dirac_apply(h, ptr(psi), ptr(out), nrhs, stream_ptr(stream)), "amg_dirac_apply")


def amg_sap(h, y, x, nrhs=1, n_cycles=1, n_mr=4, stream=None):
    return _check(lib.amg_sap(h, ptr(y), ptr(x), nrhs, n_cycles, n_mr, stream_ptr(stream)), "amg_sap")


def amg_vcycle(h, vp, y, x, nrhs=1, stream=None):
    return _check(lib.amg_vcycle(h, ctypes.byref(vp), ptr(y), ptr(x), nrhs, stream_ptr(stream)), "amg_vcycle")


def amg_setup_level2(h1, params2, tv2, stream=None, allow_rank_deficient=False):
    """Level-2 handle from the level-1 handle h1 and level-1 test vectors tv2; returns (handle, status)."""
    h = _vp()
    st = lib.amg_setup_level2(h1, ctypes.byref(params2), ptr(tv2), stream_ptr(stream), ctypes.byref(h))
    _check(st, "amg_setup_level2", (AMG_ERR_RANK_DEFICIENT,) if allow_rank_deficient else ())
    return h.value, st


def amg_restrict2(h2, yc, ycc, nrhs=1, stream=None):
    return _check(lib.amg_restrict2(h2, ptr(yc), ptr(ycc), nrhs, stream_ptr(stream)), "amg_restrict2")


def amg_prolong2(h2, xcc, xc, nrhs=1, stream=None):
    return _check(lib.amg_prolong2(h2, ptr(xcc), ptr(xc), nrhs, stream_ptr(stream)), "amg_prolong2")


def make_level2_params(n_mr=2, restart=30, max_applies=200, tol=0.05):
    return amg_level2_params(n_mr, restart, max_applies, tol)


def amg_attach_level2(h1, h2, lp=None):
    """Makes h2 the third level of h1 (h2 None detaches)."""
    return _check(lib.amg_attach_level2(h1, h2, ctypes.byref(lp) if lp is not None else None),
                  "amg_attach_level2")


def amg_two_grid(h1, yc, xc, nrhs=1, stream=None):
    return _check(lib.amg_two_grid(h1, ptr(yc), ptr(xc), nrhs, stream_ptr(stream)), "amg_two_grid")


def amg_adaptive_setup(h, vp, U, tv, n_setup=1, stream=None, allow_rank_deficient=False):
    allow = (AMG_ERR_RANK_DEFICIENT,) if allow_rank_deficient else ()
    return _check(lib.amg_adaptive_setup(h, ctypes.byref(vp), ptr(U), ptr(tv), n_setup, stream_ptr(stream)),
                  "amg_adaptive_setup", allow)


def amg_solve(h, vp, f, u, nrhs=1, tol=1e-10, restart=30, max_applies=500, stream=None, info=True):
    buf = _info(nrhs, info)
    _check(lib.amg_solve(h, ctypes.byref(vp), ptr(f), ptr(u), nrhs, tol, restart, max_applies, stream_ptr(stream),
                         buf), "amg_solve")
    return _info_out(buf, nrhs)


def amg_setup_evenodd(h, stream=None):
    return _check(lib.amg_setup_evenodd(h, stream_ptr(stream)), "amg_setup_evenodd")


def amg_schur_apply(h, xe, ye, nrhs=1, stream=None):
    return _check(lib.amg_schur_apply(h, ptr(xe), ptr(ye), nrhs, stream_ptr(stream)), "amg_schur_apply")


def amg_coarse_solve_eo(h, b, x, nrhs=1, tol=0.05, restart=30, max_applies=200, stream=None, info=True):
    """Even/odd-reduced coarse solve; returns [(applications of S, reduced relative residual)]."""
    buf = _info(nrhs, info)
    _check(lib.amg_coarse_solve_eo(h, ptr(b), ptr(x), nrhs, tol, restart, max_applies, stream_ptr(stream), buf),
           "amg_coarse_solve_eo")
    return _info_out(buf, nrhs)


def amg_cgc_eo(h, y, x, nrhs=1, tol=0.05, restart=30, max_applies=200, stream=None, info=True):
    buf = _info(nrhs, info)
    _check(lib.amg_cgc_eo(h, ptr(y), ptr(x), nrhs, tol, restart, max_applies, stream_ptr(stream), buf),
           "amg_cgc_eo")
    return _info_out(buf, nrhs)


def amg_export_Dinv(h, out):
    return _check(lib.amg_export_Dinv(h, ptr(out)), "amg_export_Dinv")


def amg_batch_cgc(hs, ys, xs, nrhs, stream=None):
    n = len(hs)
    H = (_vp * n)(*hs)
    Y = (_vp * n)(*[ptr(y) for y in ys])
    X = (_vp * n)(*[ptr(x) for x in xs])
    R = (_i * n)(*nrhs)
    return _check(lib.amg_batch_cgc(H, n, Y, X, R, stream_ptr(stream)), "amg_batch_cgc")


def amg_batch_autotune(hs, ys, xs, nrhs, stream=None):
    """Returns the time in ms of the fastest launch shape, which hs[0] keeps."""
    n = len(hs)
    best = ctypes.c_double()
    _check(lib.amg_batch_autotune((_vp * n)(*hs), n, (_vp * n)(*[ptr(y) for y in ys]),
                                  (_vp * n)(*[ptr(x) for x in xs]), (_i * n)(*nrhs), stream_ptr(stream),
                                  ctypes.byref(best)), "amg_batch_autotune")
    return best.value


def amg_batch_test_hook(h0, extra_need):
    return _check(lib.amg_batch_test_hook(h0, extra_need), "amg_batch_test_hook")


def amg_solve_test_hook(h, extra_arrivals):
    return _check(lib.amg_solve_test_hook(h, extra_arrivals), "amg_solve_test_hook")


def amg_grid_cap_test_hook(h, max_ctas):
    return _check(lib.amg_grid_cap_test_hook(h, max_ctas), "amg_grid_cap_test_hook")


def amg_export_R(h, out):
    return _check(lib.amg_export_R(h, ptr(out)), "amg_export_R")


def amg_export_Dc(h, out):
    return _check(lib.amg_export_Dc(h, ptr(out)), "amg_export_Dc")


def amg_export_clover(h, out):
    return _check(lib.amg_export_clover(h, ptr(out)), "amg_export_clover")


def amg_export_Dc_stored(h, out):
    return _check(lib.amg_export_Dc_stored(h, ptr(out)), "amg_export_Dc_stored")


def amg_setup_timings(h):
    out = (ctypes.c_double * 4)()
    _check(lib.amg_setup_timings(h, out), "amg_setup_timings")
    return list(out)


def amg_kernel_launches(h):
    out = ctypes.c_ulonglong()
    _check(lib.amg_kernel_launches(h, ctypes.byref(out)), "amg_kernel_launches")
    return out.value


def amg_sync_status(h):
    """Returns the status (does not raise)."""
    return lib.amg_sync_status(h)


def amg_destroy(h):
    return _check(lib.amg_destroy(h), "amg_destroy")
