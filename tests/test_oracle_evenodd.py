"""Pins of the oracle's even/odd reduction of the coarse system (Alg. 2's even/odd-preconditioned
coarse solve).

Expected values come from the dense coarse matrix (textbook Schur complement with numpy's dense
inverse of the whole odd-odd block, and numpy's dense solve), from the checkerboard geometry
written out by coordinates, and from the block-elimination identity, never from re-running the
same oracle routine.
"""
import numpy as np
import pytest

from oracle import coarse, dirac, evenodd as eo, lattice as lat

import helpers as H

CASES = [((4, 4, 4, 4), (2, 2, 2, 2), 6), ((8, 4, 4, 8), (2, 2, 2, 2), 4)]


def _coarse_system(L, B, ntv, seed):
    U = H.links_field(seed, 0.3, L)
    C = dirac.clover_field(U, H.CSW)
    Q = coarse.orthonormalize(H.tv_field(seed, ntv, L), B)
    Lc = lat.coarse_dims(L, B)
    return coarse.coarse_operator(U, C, H.M0, Q, L, B), Lc


@pytest.fixture(scope="module", params=CASES, ids=["Lc2^4", "Lc4x2x2x4"])
def system(request):
    L, B, ntv = request.param
    Dc, Lc = _coarse_system(L, B, ntv, 911)
    return Dc, Lc


def test_checkerboard_geometry():
    """Every hop joins opposite parities (extent 2 included); the parity-p sites in lexicographic
    order are the sites i with i // 2 = 0, 1, 2, ... (L_x even)."""
    for Lc in [(2, 2, 2, 2), (4, 2, 2, 4), (6, 4, 2, 2)]:
        Vc = int(np.prod(Lc))
        par = np.zeros(Vc, dtype=int)
        for t in range(Lc[3]):
            for z in range(Lc[2]):
                for y in range(Lc[1]):
                    for x in range(Lc[0]):
                        par[((t * Lc[2] + z) * Lc[1] + y) * Lc[0] + x] = (x + y + z + t) % 2
        assert np.array_equal(eo.parity(Lc), par)
        nbr = lat.coarse_neighbours(Lc)
        for d in range(1, lat.NDIR):
            assert np.all(par[nbr[:, d]] != par)
        for p in (0, 1):
            sites = np.nonzero(par == p)[0]
            assert np.array_equal(sites // 2, np.arange(Vc // 2))


def test_odd_extent_is_rejected():
    with pytest.raises(ValueError):
        eo.split(np.zeros((24, 4)), (2, 3, 2, 2))


def _dense_blocks(Dc, Lc):
    M = coarse.dense_coarse(Dc, Lc)
    nc = Dc.shape[2]
    par = eo.parity(Lc)
    idx = lambda p: (np.nonzero(par == p)[0][:, None] * nc + np.arange(nc)[None, :]).ravel()
    e, o = idx(0), idx(1)
    return M, e, o


def test_schur_complement_equals_dense(system):
    Dc, Lc = system
    M, e, o = _dense_blocks(Dc, Lc)
    S = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.inv(M[np.ix_(o, o)]) @ M[np.ix_(o, e)]
    rng = np.random.default_rng(3)
    nc = Dc.shape[2]
    xe = rng.normal(size=(len(e) // nc, nc, 2)) + 1j * rng.normal(size=(len(e) // nc, nc, 2))
    got = eo.schur_apply(Dc, xe, Lc)
    want = np.einsum("ab,bk->ak", S, xe.reshape(len(e), 2)).reshape(xe.shape)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_block_elimination_identity(system):
    """With x_o = -D_oo^{-1} D_oe x_e the full operator gives (S x_e, 0)."""
    Dc, Lc = system
    nc = Dc.shape[2]
    Vc = Dc.shape[0]
    rng = np.random.default_rng(4)
    xe = rng.normal(size=(Vc // 2, nc)) + 1j * rng.normal(size=(Vc // 2, nc))
    M, e, o = _dense_blocks(Dc, Lc)
    xo = -np.linalg.solve(M[np.ix_(o, o)], M[np.ix_(o, e)] @ xe.ravel()).reshape(xe.shape)
    full = eo.merge(xe, xo, Lc).reshape(Vc, 2, nc // 2)
    ye, yo = eo.split(coarse.coarse_apply(Dc, full, Lc).reshape(Vc, nc), Lc)
    assert np.abs(yo).max() <= 1e-12 * np.abs(ye).max()
    assert np.abs(ye - eo.schur_apply(Dc, xe, Lc)).max() <= 1e-11 * np.abs(ye).max()


def test_self_inverses(system):
    Dc, Lc = system
    Dinv = eo.self_inverses(Dc, Lc)
    odd = Dc[eo.parity(Lc) == 1, 0]
    eye = np.eye(Dc.shape[2])
    assert np.abs(np.einsum("iab,ibc->iac", Dinv, odd) - eye).max() < 1e-12


def test_eo_solve_equals_dense_solve(system):
    Dc, Lc = system
    nc = Dc.shape[2]
    Vc = Dc.shape[0]
    rng = np.random.default_rng(5)
    b = rng.normal(size=(Vc, nc)) + 1j * rng.normal(size=(Vc, nc))
    x, hist, n = eo.eo_solve(Dc, b, Lc, tol=1e-13, restart=200, max_applies=400)
    want = np.linalg.solve(coarse.dense_coarse(Dc, Lc), b.ravel()).reshape(b.shape)
    assert np.abs(x - want).max() <= 1e-9 * np.abs(want).max()


def test_eo_solve_residual_is_the_schur_residual(system):
    """At the loose tolerance of Alg. 2 the full residual b - D_c x is zero on the odd half and
    equals the reduced system's residual on the even half."""
    Dc, Lc = system
    nc = Dc.shape[2]
    Vc = Dc.shape[0]
    rng = np.random.default_rng(6)
    b = rng.normal(size=(Vc, nc)) + 1j * rng.normal(size=(Vc, nc))
    x, hist, n = eo.eo_solve(Dc, b, Lc, tol=0.05)
    re, ro = eo.split(b - coarse.coarse_apply(Dc, x.reshape(Vc, 2, nc // 2), Lc).reshape(Vc, nc), Lc)
    M, e, o = _dense_blocks(Dc, Lc)
    be, bo = eo.split(b, Lc)
    rhs = be.ravel() - M[np.ix_(e, o)] @ np.linalg.solve(M[np.ix_(o, o)], bo.ravel())
    assert np.abs(ro).max() <= 1e-12 * np.abs(b).max()
    assert np.linalg.norm(re) <= 0.05 * np.linalg.norm(rhs) * (1 + 1e-9)
    assert n == len(hist)
