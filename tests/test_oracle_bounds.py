"""Pins of the oracle's reduced-precision helpers (coarse.abs_apply, coarse.reduced_precision_bound),
which set the tolerances of the FP16 / BF16 parity tests.

abs_apply is checked against |M| |x| with the dense coarse matrix M (equal when no coarse extent
is 2, at least as large when the +mu and -mu neighbours coincide).  The bound is checked against
operators whose entries are rounded to p significant bits (round half to even, written here from
the definition: p = 11 for the FP16 significand, p = 8 for BF16), applied with FP64 and with FP32
accumulation: it must hold, and it must not be loose by more than a factor 100.
"""
import numpy as np
import pytest

from oracle import coarse, lattice as lat


def _random_system(Lc, ntv, seed, nrhs=2):
    rng = np.random.default_rng(seed)
    Vc, nc = int(np.prod(Lc)), 2 * ntv
    shape = (Vc, lat.NDIR, nc, nc)
    mag = 10.0 ** rng.uniform(-3, 1, size=shape)
    Dc = mag * (rng.normal(size=shape) + 1j * rng.normal(size=shape))
    x = rng.normal(size=(Vc, 2, ntv, nrhs)) + 1j * rng.normal(size=(Vc, 2, ntv, nrhs))
    return Dc, x


def _round_bits(v, p):
    """Real v rounded to p significant bits, ties to even (np.round rounds half to even)."""
    m, e = np.frexp(v)  # v = m 2^e, 1/2 <= |m| < 1
    return np.ldexp(np.round(np.ldexp(m, p)), e - p)


def _round_complex(a, p):
    return _round_bits(a.real, p) + 1j * _round_bits(a.imag, p)


def test_round_bits_definition():
    # 8 significant bits: spacing 2^-7 on [1, 2); ties go to the even neighbour
    assert _round_bits(np.array([1.0 + 2.0 ** -8]), 8)[0] == 1.0
    assert _round_bits(np.array([1.0 + 3 * 2.0 ** -8]), 8)[0] == 1.0 + 2.0 ** -6
    assert _round_bits(np.array([1.0 + 0.75 * 2.0 ** -7]), 8)[0] == 1.0 + 2.0 ** -7
    v = np.random.default_rng(0).normal(size=1000)
    assert np.all(np.abs(_round_bits(v, 11) - v) <= 2.0 ** -11 * np.abs(v))


def test_abs_apply_is_the_dense_absolute_product_without_aliasing():
    Lc = (3, 3, 3, 3)
    Dc, x = _random_system(Lc, 2, 1)
    M = coarse.dense_coarse(Dc, Lc)
    got = coarse.abs_apply(Dc, x, Lc)
    want = (np.abs(M) @ np.abs(x.reshape(M.shape[0], -1))).reshape(got.shape)
    assert np.abs(got - want).max() <= 1e-12 * want.max()


def test_abs_apply_bounds_the_dense_absolute_product_with_aliasing():
    Lc = (2, 3, 2, 3)  # +x/-x and +z/-z reach the same coarse site
    Dc, x = _random_system(Lc, 2, 2)
    M = coarse.dense_coarse(Dc, Lc)
    got = coarse.abs_apply(Dc, x, Lc)
    want = (np.abs(M) @ np.abs(x.reshape(M.shape[0], -1))).reshape(got.shape)
    assert np.all(got >= want * (1 - 1e-12))
    assert np.any(got > want * (1 + 1e-6))  # the two faces are summed in absolute value


@pytest.mark.parametrize("p", [11, 8], ids=["fp16_significand", "bf16"])
@pytest.mark.parametrize("Lc", [(3, 3, 3, 3), (2, 3, 2, 3)], ids=["no_alias", "alias"])
def test_reduced_precision_bound_holds_and_is_not_vacuous(p, Lc):
    Dc, x = _random_system(Lc, 2, 3 + p)
    y = coarse.coarse_apply(Dc, x, Lc)
    Dr = _round_complex(Dc, p)
    # FP64 accumulation: only the storage error
    err = np.linalg.norm(coarse.coarse_apply(Dr, x, Lc) - y) / np.linalg.norm(y)
    bound = coarse.reduced_precision_bound(Dc, x, Lc, 2.0 ** -p, u_acc=0.0)
    assert err <= bound
    assert bound <= 100 * err
    # FP32 accumulation on top
    y32 = coarse.coarse_apply(Dr.astype(np.complex64), x.astype(np.complex64), Lc).astype(np.complex128)
    err32 = np.linalg.norm(y32 - y) / np.linalg.norm(y)
    x32 = x.astype(np.complex64).astype(np.complex128)  # the rounded input is the product's input
    bound32 = coarse.reduced_precision_bound(Dc, x32, Lc, 2.0 ** -p + 2.0 ** -24)
    assert err32 <= bound32 + np.linalg.norm(coarse.coarse_apply(Dc, x32 - x, Lc)) / np.linalg.norm(y)


@pytest.mark.parametrize("ntv", [2, 4])
@pytest.mark.parametrize("Lc", [(3, 3, 3, 3), (2, 3, 2, 3)], ids=["no_alias", "alias"])
def test_accumulation_term_alone_holds_and_is_not_vacuous(ntv, Lc):
    """Storage exact (D_c and x already FP32 numbers, u_store = 0): the only error left is the FP32
    arithmetic of the product, so the bound is (K + 2) u_acc || |D||x| || / ||D x|| with the FP32 unit
    roundoff u_acc = 2^-24, K = 9 * 2 N_tv.  It must hold, and with K = 36 or 72 it must not exceed
    the measured error by more than a factor 1000 (worst case (K + 2) u against the observed
    rounding of a few u): a unit roundoff taken 16 times too large (2^-20) fails here."""
    Dc, x = _random_system(Lc, ntv, 7)
    D32 = Dc.astype(np.complex64).astype(np.complex128)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y = coarse.coarse_apply(D32, x32, Lc)
    y32 = coarse.coarse_apply(D32.astype(np.complex64), x32.astype(np.complex64), Lc).astype(np.complex128)
    err = np.linalg.norm(y32 - y) / np.linalg.norm(y)
    bound = coarse.reduced_precision_bound(D32, x32, Lc, 0.0)
    assert 0.0 < err <= bound
    assert bound <= 1000 * err
