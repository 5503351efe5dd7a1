"""Pins of the oracle's coarse-grid pieces (Alg. 2, Alg. 5, Eq. cgo, Eq. dagger).

Expected values come from brute force with the entry-by-entry dense D, from
the closed form of the free-field coarse operator, from Householder QR, from
gamma_5-hermiticity and gauge invariance, never from re-running the same
oracle routine.
"""
import numpy as np
import pytest

from oracle import coarse, dirac, krylov, lattice as lat

import helpers as H


def _setup(L, B, ntv, eps, seed):
    U = H.links_field(seed, eps, L)
    C = dirac.clover_field(U, H.CSW)
    tv = H.tv_field(seed, ntv, L)
    Q = coarse.orthonormalize(tv, B)
    return U, C, tv, Q


def test_aggregate_layout_by_loops():
    """Aggregate dof n of block i, chirality h = (site in block, spin in chirality, colour)."""
    L, B = (4, 2, 2, 4), (2, 2, 1, 2)
    Lc = lat.coarse_dims(L, B)
    idx = coarse.aggregate_dof_indices(L, B)
    for i in range(int(np.prod(Lc))):
        X = lat.coarse_coords(i, Lc)
        for h in range(2):
            n = 0
            for bt in range(B[3]):
                for bz in range(B[2]):
                    for by in range(B[1]):
                        for bx in range(B[0]):
                            x = [X[0] * B[0] + bx, X[1] * B[1] + by, X[2] * B[2] + bz, X[3] * B[3] + bt]
                            s = ((x[3] * L[2] + x[2]) * L[1] + x[1]) * L[0] + x[0]
                            for a in range(2):
                                for c in range(3):
                                    assert idx[i, h, n] == s * 12 + (2 * h + a) * 3 + c
                                    n += 1


def test_gram_schmidt_equals_householder_qr():
    rng = np.random.default_rng(1)
    W = rng.normal(size=(96, 12)) + 1j * rng.normal(size=(96, 12))
    Q = coarse.gram_schmidt(W)
    Qh, Rh = np.linalg.qr(W)  # LAPACK Householder
    ph = np.diag(Rh) / np.abs(np.diag(Rh))
    assert np.abs(Q - Qh * ph[None, :]).max() < 1e-13
    # W = Q T with T upper triangular, real positive diagonal
    T = Q.conj().T @ W
    assert np.abs(np.tril(T, -1)).max() < 1e-13
    assert np.all(np.diag(T).real > 0) and np.abs(np.diag(T).imag).max() < 1e-13


def test_gram_schmidt_rank_deficient():
    rng = np.random.default_rng(2)
    W = rng.normal(size=(48, 5)) + 1j * rng.normal(size=(48, 5))
    W[:, 3] = 2 * W[:, 0] - 1j * W[:, 2]
    with pytest.raises(coarse.RankDeficient):
        coarse.gram_schmidt(W)


def test_tiny_workload_brute_force():
    """4^4, 2^4 blocks (coarse extent 2), Ntv = 8: dense R D P, R P = I, gamma_5."""
    L, B, ntv, eps, off = H.WORKLOADS["tiny_4^4_b2_ntv8"]
    seed = 20151204 + off
    U, C, tv, Q = _setup(L, B, ntv, eps, seed)
    Lc = lat.coarse_dims(L, B)
    Dc = coarse.coarse_operator(U, C, H.M0, Q, L, B)
    D = dirac.dense_dirac(U, C, H.M0)
    R = coarse.dense_restriction(Q, L, B)
    # R P = I
    assert np.abs(R @ R.conj().T - np.eye(R.shape[0])).max() < 1e-14
    # rows of R_i^h span the test vectors restricted to A_i^h
    W = lat.to_aggregates(tv, B)
    resid = W - np.einsum("ihnj,ihjk->ihnk", Q, np.einsum("ihnj,ihnk->ihjk", Q.conj(), W))
    assert np.abs(resid).max() < 1e-12
    # D_c = R D P, block by block
    M = coarse.dense_coarse(Dc, Lc)
    ref = R @ D @ R.conj().T
    assert np.abs(M - ref).max() < 1e-13 * np.abs(ref).max()
    # gamma_5 hermiticity of D_c and Eq. dagger blockwise
    g5 = np.tile(coarse.gamma5_coarse(ntv), int(np.prod(Lc)))
    assert np.abs(g5[:, None] * M * g5[None, :] - M.conj().T).max() < 1e-14
    _check_eq_dagger(Dc, Lc, ntv)
    # restrict / prolong against the dense R
    rng = np.random.default_rng(3)
    y = rng.normal(size=tv.shape[:6]) + 1j * rng.normal(size=tv.shape[:6])
    yc = coarse.restrict(Q, y, B)
    assert np.abs(yc.reshape(-1) - R @ dirac.flatten_field(y)).max() < 1e-13
    x = coarse.prolong(Q, yc, L, B)
    assert np.abs(dirac.flatten_field(x) - R.conj().T @ yc.reshape(-1)).max() < 1e-13
    xc = rng.normal(size=yc.shape) + 1j * rng.normal(size=yc.shape)
    assert np.abs(coarse.coarse_apply(Dc, xc, Lc).reshape(-1) - ref @ xc.reshape(-1)).max() < 1e-12


def _check_eq_dagger(Dc, Lc, N):
    """(D_c)_{ji}^{hh} = (D_c)_{ij}^{hh dagger}, (D_c)_{ji}^{hh'} = -(D_c)_{ij}^{h'h dagger}."""
    nbr = lat.coarse_neighbours(Lc)
    s = coarse.gamma5_coarse(N)
    for i in range(Dc.shape[0]):
        for mu in range(4):
            j = nbr[i, 1 + 2 * mu]
            fwd = Dc[i, 1 + 2 * mu]
            bwd = Dc[j, 2 + 2 * mu]
            assert np.abs(bwd - s[:, None] * fwd.conj().T * s[None, :]).max() < 1e-14
        d0 = Dc[i, 0]
        assert np.abs(d0 - s[:, None] * d0.conj().T * s[None, :]).max() < 1e-14


@pytest.mark.parametrize("L,B", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 4), (2, 2, 2, 2)),
                                 ((6, 4, 4, 8), (2, 2, 4, 4))])
def test_free_field_coarse_operator_closed_form(L, B):
    """U = 1 and the six piecewise-constant test vectors e_{s,c} + e_{s+2,c}:
    D_c is the coarse Wilson operator with hopping 1/b_mu,
    self = (m0 + sum_mu 1/b_mu) 1, +mu = -(1 - gamma_mu)/(2 b_mu), -mu = -(1 + gamma_mu)/(2 b_mu)."""
    U = H.identity_links(L)
    C = dirac.clover_field(U, H.CSW)
    tv = np.zeros(H.field_shape(L) + (4, 3, 6), dtype=np.complex128)
    for s in range(2):
        for c in range(3):
            tv[..., s, c, s * 3 + c] = 1
            tv[..., s + 2, c, s * 3 + c] = 1
    Q = coarse.orthonormalize(tv, B)
    Dc = coarse.coarse_operator(U, C, H.M0, Q, L, B)
    g = dirac.gammas()
    I3 = np.eye(3)
    self_ = (H.M0 + sum(1.0 / b for b in B)) * np.eye(12)
    for i in range(Dc.shape[0]):
        assert np.abs(Dc[i, 0] - self_).max() < 1e-14
        for mu in range(4):
            fwd = -np.kron(np.eye(4) - g[mu], I3) / (2 * B[mu])
            bwd = -np.kron(np.eye(4) + g[mu], I3) / (2 * B[mu])
            assert np.abs(Dc[i, 1 + 2 * mu] - fwd).max() < 1e-14
            assert np.abs(Dc[i, 2 + 2 * mu] - bwd).max() < 1e-14
    # and its spectrum: m0 + sum (1 - cos P)/b +- i sqrt(sum sin^2 P / b^2), 6-fold
    Lc = lat.coarse_dims(L, B)
    ev = np.linalg.eigvals(coarse.dense_coarse(Dc, Lc))
    expect = []
    for n in np.ndindex(*Lc):
        P = 2 * np.pi * np.array(n) / np.array(Lc)
        re = H.M0 + np.sum((1 - np.cos(P)) / np.array(B))
        im = np.sqrt(np.sum(np.sin(P) ** 2 / np.array(B) ** 2))
        expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    key = lambda z: (np.round(z.real, 8), np.round(z.imag, 8))
    a = np.array(sorted(ev, key=key))
    b = np.array(sorted(expect, key=key))
    assert np.abs(a - b).max() < 1e-10


def test_gauge_invariance_of_coarse_operator():
    """U -> G U G^dagger, v -> G v leaves D_c unchanged and rotates R."""
    L, B, ntv = (4, 4, 2, 4), (2, 2, 2, 2), 6
    U, C, tv, Q = _setup(L, B, ntv, 0.4, 31)
    G = H.links_field(77, 1.1, L)[0]
    Ug = dirac.gauge_transform(U, G)
    Cg = dirac.clover_field(Ug, H.CSW)
    tvg = np.einsum("...ij,...ajk->...aik", G, tv)
    Qg = coarse.orthonormalize(tvg, B)
    Dc = coarse.coarse_operator(U, C, H.M0, Q, L, B)
    Dcg = coarse.coarse_operator(Ug, Cg, H.M0, Qg, L, B)
    assert np.abs(Dc - Dcg).max() < 1e-13
    Qrot = lat.to_aggregates(np.einsum("...ij,...ajk->...aik", G, lat.from_aggregates(Q, L, B)), B)
    assert np.abs(Qg - Qrot).max() < 1e-13


def test_matrix_free_galerkin_identity():
    """D_c x_c == R (D (P x_c)) with every piece matrix-free, coarse extent 3 and 2."""
    L, B, ntv = (6, 4, 4, 8), (2, 2, 2, 4), 6
    U, C, tv, Q = _setup(L, B, ntv, 0.3, 41)
    Lc = lat.coarse_dims(L, B)
    Dc = coarse.coarse_operator(U, C, H.M0, Q, L, B)
    _check_eq_dagger(Dc, Lc, ntv)
    rng = np.random.default_rng(4)
    xc = rng.normal(size=(int(np.prod(Lc)), 2, ntv)) + 1j * rng.normal(size=(int(np.prod(Lc)), 2, ntv))
    lhs = coarse.coarse_apply(Dc, xc, Lc)
    rhs = coarse.restrict(Q, dirac.apply_dirac(U, C, H.M0, coarse.prolong(Q, xc, L, B)), B)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()
    # multi-RHS forms agree column by column
    xk = np.stack([xc, 2j * xc], axis=-1)
    yk = coarse.coarse_apply(Dc, xk, Lc)
    assert np.abs(yk[..., 1] - 2j * lhs).max() < 1e-12


def test_sampled_coarse_sites_match_full():
    """Restricting the output to chosen coarse sites changes nothing else."""
    L, B, ntv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U, C, tv, Q = _setup(L, B, ntv, 0.3, 51)
    full = coarse.coarse_operator(U, C, H.M0, Q, L, B)
    part = coarse.coarse_operator(U, C, H.M0, Q, L, B, sites=[3, 9])
    assert np.array_equal(part, full[[3, 9]])


def test_patch_reproduces_periodic_lattice():
    """A 3x3x3x3-block box around a block gives that block's D_c row exactly;
    the GPU parity tests of large lattices rely on this."""
    L, B, ntv = (8, 8, 8, 8), (2, 2, 2, 2), 4
    seed = 61
    U, C, tv, Q = _setup(L, B, ntv, 0.3, seed)
    Lc = lat.coarse_dims(L, B)
    i_glob = lat.coarse_index(np.array([3, 0, 2, 1]), Lc)
    full = coarse.coarse_operator(U, C, H.M0, Q, L, B, sites=[i_glob])
    origin = [(c - 1) * b for c, b in zip([3, 0, 2, 1], B)]
    shape = [3 * b for b in B]
    Up = H.links_field(seed, 0.3, L, origin, shape)
    tvp = H.tv_field(seed, ntv, L, origin, shape)
    Cp = dirac.clover_field(Up, H.CSW)
    Qp = coarse.orthonormalize(tvp, B)
    centre = lat.coarse_index(np.array([1, 1, 1, 1]), (3, 3, 3, 3))
    patch = coarse.coarse_operator(Up, Cp, H.M0, Qp, tuple(shape), B, sites=[centre])
    assert np.abs(patch - full).max() < 1e-14


def test_gmres_minimises_over_krylov_space():
    """After k steps (no restart) the iterate minimises ||b - A x|| over K_k(A, b)."""
    L, B, ntv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U, C, tv, Q = _setup(L, B, ntv, 0.3, 71)
    Lc = lat.coarse_dims(L, B)
    Dc = coarse.coarse_operator(U, C, H.M0, Q, L, B)
    A = coarse.dense_coarse(Dc, Lc)
    rng = np.random.default_rng(8)
    b = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    for k in (1, 4, 9):
        x, hist, n = krylov.fgmres(lambda v: A @ v, b, tol=1e-30, restart=k, max_applies=k)
        assert n == k and len(hist) == k
        K = np.empty((A.shape[0], k), dtype=complex)
        v = b / np.linalg.norm(b)
        for j in range(k):
            K[:, j] = v
            v = A @ v
            v /= np.linalg.norm(v)
        Qk, _ = np.linalg.qr(K)
        c, *_ = np.linalg.lstsq(A @ Qk, b, rcond=None)
        xref = Qk @ c
        assert np.abs(x - xref).max() < 1e-10 * np.abs(xref).max()
        assert abs(hist[-1] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-10


def test_gmres_restarted_reaches_tolerance():
    L, B, ntv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U, C, tv, Q = _setup(L, B, ntv, 0.3, 71)
    Lc = lat.coarse_dims(L, B)
    Dc = coarse.coarse_operator(U, C, H.M0, Q, L, B)
    rng = np.random.default_rng(9)
    b = rng.normal(size=(16, 2, ntv)) + 1j * rng.normal(size=(16, 2, ntv))
    x, hist, n = krylov.fgmres(lambda v: coarse.coarse_apply(Dc, v, Lc), b, tol=1e-6,
                               restart=8, max_applies=400)
    true = np.linalg.norm(b - coarse.coarse_apply(Dc, x, Lc)) / np.linalg.norm(b)
    assert true <= 1.01e-6 and n < 400
