"""The C-ABI libraries load and export every symbol their headers declare (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def built():
    amg = os.path.join(ROOT, "paper_1512_04506_gb300", "libamg.so")
    syn = os.path.join(ROOT, "synth", "libsynth.so")
    if not (os.path.exists(amg) and os.path.exists(syn)):
        import __graft_entry__
        __graft_entry__.build()
    return amg, syn


def _declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[A-Za-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(built):
    amg_path, _ = built
    lib = ctypes.CDLL(amg_path)
    names = _declared(os.path.join(ROOT, "include", "amg.h"))
    assert "amg_setup_coarse" in names and "amg_coarse_apply" in names
    for n in names:
        assert hasattr(lib, n), "libamg.so does not export %s" % n
    lib.amg_status_string.restype = ctypes.c_char_p
    assert lib.amg_status_string(6).decode().startswith("test vectors")


def test_binding_covers_header(built):
    import paper_1512_04506_gb300 as amg
    names = _declared(os.path.join(ROOT, "include", "amg.h"))
    assert sorted(amg.EXPORTED) == names
    for n in names:
        assert callable(getattr(amg, n))


def test_synth_library_exports(built):
    _, syn = built
    lib = ctypes.CDLL(syn)
    for n in ("synth_links", "synth_test_vectors", "synth_fine_rhs", "synth_coarse_vector"):
        assert hasattr(lib, n)


def test_params_struct_layout(built):
    import paper_1512_04506_gb300 as amg
    # int L[4], B[4], ntv, max_nrhs, double m0, csw, 4 enums
    assert ctypes.sizeof(amg.amg_params) == 4 * 10 + 2 * 8 + 4 * 4
    assert amg.amg_params.m0.offset == 40
    assert amg.amg_params.setup_arith.offset == 68


def test_argument_validation_without_gpu(built):
    """Validation happens before any CUDA call: bad parameters are rejected on a host without a GPU."""
    import paper_1512_04506_gb300 as amg
    h = ctypes.c_void_p()
    bad = [
        amg.make_params((4, 4, 4, 4), (3, 2, 2, 2), 8),           # block does not divide
        amg.make_params((4, 4, 4, 4), (4, 2, 2, 2), 8),           # coarse extent 1
        amg.make_params((4, 4, 4, 4), (2, 2, 2, 2), 0),           # ntv < 1
        amg.make_params((4, 4, 4, 4), (1, 1, 1, 1), 7),           # ntv > 6 Vb
        amg.make_params((4, 4, 4, 4), (2, 2, 2, 2), 8, max_nrhs=0),
        amg.make_params((4, 4, 4, 4), (2, 2, 2, 2), 8, link_prec=9),
        amg.make_params((4, 4, 4, 4), (2, 2, 2, 2), 8, setup_arith=2),
    ]
    for p in bad:
        st = amg.lib.amg_setup_coarse(ctypes.byref(p), 16, 16, None, ctypes.byref(h))
        assert st == amg.AMG_ERR_INVALID_ARG
    p = amg.make_params((4, 4, 4, 4), (2, 2, 2, 2), 8)
    assert amg.lib.amg_setup_coarse(ctypes.byref(p), 17, 16, None, ctypes.byref(h)) == amg.AMG_ERR_INVALID_ARG
    assert amg.lib.amg_setup_coarse(ctypes.byref(p), None, 16, None, ctypes.byref(h)) == amg.AMG_ERR_INVALID_ARG
    # unsupported precision combinations
    p = amg.make_params((4, 4, 4, 4), (2, 2, 2, 2), 8, link_prec=amg.AMG_FP32, r_prec=amg.AMG_FP64,
                        vec_prec=amg.AMG_FP64)
    assert amg.lib.amg_setup_coarse(ctypes.byref(p), 16, 16, None, ctypes.byref(h)) == amg.AMG_ERR_UNSUPPORTED
    assert amg.lib.amg_restrict(None, 16, 16, 1, None) == amg.AMG_ERR_INVALID_ARG
    assert amg.lib.amg_destroy(None) == amg.AMG_ERR_INVALID_ARG


def test_level2_params_layout_and_validation(built):
    """amg_level2_params is int n_mr, restart, max_applies, double tol; the three-level calls
    reject missing handles and parameters before any CUDA call."""
    import paper_1512_04506_gb300 as amg
    assert ctypes.sizeof(amg.amg_level2_params) == 24
    assert amg.amg_level2_params.tol.offset == 16
    h = ctypes.c_void_p()
    p = amg.make_params((4, 4, 4, 4), (2, 2, 2, 2), 4)
    assert amg.lib.amg_setup_level2(None, ctypes.byref(p), 16, None, ctypes.byref(h)) == amg.AMG_ERR_INVALID_ARG
    assert amg.lib.amg_setup_level2(None, ctypes.byref(p), 16, None, None) == amg.AMG_ERR_INVALID_ARG
    lp = amg.make_level2_params()
    assert amg.lib.amg_attach_level2(None, None, ctypes.byref(lp)) == amg.AMG_ERR_INVALID_ARG
    assert amg.lib.amg_two_grid(None, 16, 32, 1, None) == amg.AMG_ERR_INVALID_ARG
    assert amg.lib.amg_restrict2(None, 16, 32, 1, None) == amg.AMG_ERR_INVALID_ARG
    assert amg.lib.amg_prolong2(None, 16, 32, 1, None) == amg.AMG_ERR_INVALID_ARG
