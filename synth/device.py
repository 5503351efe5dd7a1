"""Device-side generation of the synthetic inputs (ctypes binding of libsynth.so).

The values equal those of ``synth.inputs`` up to the last bits of the
transcendental functions (the link exponential is a scaled Taylor series
here, an eigen-decomposition on the host); see ``synth/csrc/synth.cu``.
Buffers are torch tensors on the current CUDA device.
"""
import ctypes
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth.so")
_lib = None


def _get():
    global _lib
    if _lib is None:
        if not os.path.exists(_PATH):
            raise ImportError("libsynth.so is not built (run __graft_entry__.build())")
        _lib = ctypes.CDLL(_PATH)
        vp, ll, i, d, u = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong
        _lib.synth_links.argtypes = [vp, ll, d, u, vp]
        _lib.synth_test_vectors.argtypes = [vp, ll, i, u, vp]
        _lib.synth_fine_rhs.argtypes = [vp, ll, i, u, i, vp]
        _lib.synth_coarse_vector.argtypes = [vp, ll, i, i, u, i, vp]
    return _lib


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed with CUDA error %d" % (what, rc))


def links(seed, eps, L):
    import torch
    V = L[0] * L[1] * L[2] * L[3]
    out = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    _check(_get().synth_links(out.data_ptr(), V, eps, seed, _stream()), "synth_links")
    return out


def test_vectors(seed, ntv, L):
    import torch
    V = L[0] * L[1] * L[2] * L[3]
    out = torch.empty((V, 4, 3, ntv), dtype=torch.complex128, device="cuda")
    _check(_get().synth_test_vectors(out.data_ptr(), V, ntv, seed, _stream()), "synth_test_vectors")
    return out


def fine_rhs(seed, nrhs, L, dtype=None):
    import torch
    dtype = dtype or torch.complex64
    V = L[0] * L[1] * L[2] * L[3]
    out = torch.empty((V, 4, 3, nrhs), dtype=dtype, device="cuda")
    prec = 0 if dtype == torch.complex128 else 1
    _check(_get().synth_fine_rhs(out.data_ptr(), V, nrhs, seed, prec, _stream()), "synth_fine_rhs")
    return out


def coarse_vector(seed, ntv, nrhs, Vc, dtype=None):
    import torch
    dtype = dtype or torch.complex64
    out = torch.empty((Vc, 2, ntv, nrhs), dtype=dtype, device="cuda")
    prec = 0 if dtype == torch.complex128 else 1
    _check(_get().synth_coarse_vector(out.data_ptr(), Vc, ntv, nrhs, seed, prec, _stream()), "synth_coarse_vector")
    return out
