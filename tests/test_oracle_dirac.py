"""Pins of the oracle's fine-lattice pieces against closed forms.

None of these compares the oracle with itself: each expected value comes
from an analytic result (gamma algebra, plane waves of the free operator,
the clover of a constant abelian field) or from an independently written
construction (the entry-by-entry dense D).
"""
import numpy as np
import pytest

from oracle import dirac, lattice as lat
from synth import inputs as si

import helpers as H


def test_gamma_algebra_chiral_basis():
    g = dirac.gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))
    # chiral basis: gamma_5 = diag(1, 1, -1, -1), gamma_mu off-diagonal
    assert np.allclose(dirac.gamma5(), np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(g[mu][:2, :2], 0) and np.allclose(g[mu][2:, 2:], 0)


def test_sigma_01_explicit():
    # sigma_01 = (i/2)[g0, g1] = -diag(sigma_3, sigma_3) in this basis (by hand)
    assert np.allclose(dirac.sigma(0, 1), np.diag([-1, 1, -1, 1]))


@pytest.mark.parametrize("L", [(4, 3, 2, 2), (2, 4, 3, 4)])
def test_free_field_plane_waves(L):
    """U = 1: D e^{ipx} chi = e^{ipx} [(4+m0) - sum cos p + i sum gamma sin p] chi."""
    U = H.identity_links(L)
    C = dirac.clover_field(U, H.CSW)
    assert np.abs(C).max() < 1e-14  # clover vanishes on the free field
    rng = np.random.default_rng(7)
    x = lat.coords_fields(L)
    g = dirac.gammas()
    for _ in range(4):
        n = [rng.integers(0, L[mu]) for mu in range(4)]
        p = [2 * np.pi * n[mu] / L[mu] for mu in range(4)]
        phase = np.exp(1j * sum(p[mu] * x[mu] for mu in range(4)))
        chi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = phase[..., None, None] * chi
        out = dirac.apply_dirac(U, C, H.M0, psi)
        Dp = (4 + H.M0 - sum(np.cos(p))) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[..., None, None] * (Dp @ chi)
        assert np.abs(out - expect).max() < 1e-13


def test_free_field_spectrum_dense():
    """Eigenvalues m0 + sum(1 - cos p) +- i |sin p|, each 6-fold, from the dense D."""
    L = (4, 3, 2, 2)
    U = H.identity_links(L)
    C = dirac.clover_field(U, H.CSW)
    D = dirac.dense_dirac(U, C, H.M0)
    ev = np.linalg.eigvals(D)
    expect = []
    for n0 in range(L[0]):
        for n1 in range(L[1]):
            for n2 in range(L[2]):
                for n3 in range(L[3]):
                    p = 2 * np.pi * np.array([n0 / L[0], n1 / L[1], n2 / L[2], n3 / L[3]])
                    re = H.M0 + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.array(expect)
    key = lambda z: (np.round(z.real, 8), np.round(z.imag, 8))
    a = np.array(sorted(ev, key=key))
    b = np.array(sorted(expect, key=key))
    assert np.abs(a - b).max() < 1e-10


def test_constant_abelian_field_clover():
    """U_x(x) = exp(i phi x_y T), others 1: C = (c_sw/2) sigma_01 (x) sin(phi T)."""
    L = (2, 4, 2, 2)
    T = np.array([1.0, 2.0, -3.0])
    phi = 2 * np.pi / L[1]
    U = H.identity_links(L)
    x = lat.coords_fields(L)
    U[0] = 0
    for c in range(3):
        U[0][..., c, c] = np.exp(1j * phi * T[c] * x[1])
    csw = 1.7
    C = dirac.clover_field(U, csw)
    expect = 0.5 * csw * np.einsum("ab,ij->aibj", np.diag([-1.0, 1, -1, 1]), np.diag(np.sin(phi * T)))
    assert np.abs(C - expect).max() < 1e-14


def _random_lattice(L, eps, seed, ntv=None):
    U = H.links_field(seed, eps, L)
    return U


def test_dense_matches_apply_and_gamma5_hermiticity():
    L = (4, 2, 2, 4)
    U = _random_lattice(L, 0.4, 11)
    C = dirac.clover_field(U, H.CSW)
    Cm = C.reshape(C.shape[:4] + (12, 12))
    # clover Hermitian and block-diagonal in chirality (sigma commutes with gamma_5)
    assert np.abs(Cm - np.conj(np.swapaxes(Cm, -1, -2))).max() < 1e-15
    assert np.abs(Cm[..., :6, 6:]).max() == 0 and np.abs(Cm[..., 6:, :6]).max() == 0
    assert np.abs(Cm).max() > 1e-3
    D = dirac.dense_dirac(U, C, H.M0)
    rng = np.random.default_rng(3)
    psi = rng.normal(size=H.field_shape(L) + (4, 3)) + 1j * rng.normal(size=H.field_shape(L) + (4, 3))
    a = dirac.flatten_field(dirac.apply_dirac(U, C, H.M0, psi))
    b = D @ dirac.flatten_field(psi)
    assert np.abs(a - b).max() < 1e-13
    V = int(np.prod(L))
    g5 = np.kron(np.eye(V), np.kron(np.diag([1.0, 1, -1, -1]), np.eye(3)))
    assert np.abs(g5 @ D @ g5 - D.conj().T).max() < 1e-14
    # the block parts add up to D
    B = (2, 2, 2, 2)
    tot = sum(dirac.apply_block_part(U, C, H.M0, psi, B, d) for d in range(9))
    assert np.abs(dirac.flatten_field(tot) - b).max() < 1e-13


def test_gauge_covariance():
    """U -> G U G(x+mu)^dagger gives C -> G C G^dagger and D -> G D G^dagger."""
    L = (4, 2, 4, 2)
    U = _random_lattice(L, 0.5, 21)
    G = H.links_field(99, 1.3, L)[0]
    Ug = dirac.gauge_transform(U, G)
    C = dirac.clover_field(U, H.CSW)
    Cg = dirac.clover_field(Ug, H.CSW)
    expect = np.einsum("...ij,...ajbk,...lk->...aibl", G, C, G.conj())
    assert np.abs(Cg - expect).max() < 1e-14
    rng = np.random.default_rng(5)
    psi = rng.normal(size=H.field_shape(L) + (4, 3)) + 1j * rng.normal(size=H.field_shape(L) + (4, 3))
    Gpsi = np.einsum("...ij,...aj->...ai", G, psi)
    lhs = dirac.apply_dirac(Ug, Cg, H.M0, Gpsi)
    rhs = np.einsum("...ij,...aj->...ai", G, dirac.apply_dirac(U, C, H.M0, psi))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_links_are_su3():
    U = si.links(5, 0.4, np.arange(500))
    eye = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # exp(i eps H) against scipy's Pade/scaling-squaring expm, a different algorithm
    from scipy.linalg import expm
    Hm = si.link_generators(5, np.arange(3))
    for s in range(3):
        for mu in range(4):
            assert np.abs(expm(0.4j * Hm[s, mu]) - U[s, mu]).max() < 1e-14
    assert np.allclose(np.trace(Hm, axis1=-2, axis2=-1), 0)
