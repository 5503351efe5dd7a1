"""Pins of the oracle's third level (oracle/mg3.py): the level-2 aggregates, Q2,
D_cc = R2 D_c P2, the minimal-residual smoother on D_c, the two-grid cycle on level 1
and the three-level V-cycle.

Expected values come from explicit loops over coordinates (aggregate membership and
the dense R2), dense matrix products (the Galerkin identity), LAPACK least squares (the
MR step) and invariants that hold for any input (gamma_5-hermiticity carried down a
level, Galerkin orthogonality of an exact coarse correction, the reduction to the
two-level cycle when the second coarsening is the identity).
"""
import numpy as np
import pytest

from oracle import coarse, mg, mg3
from oracle import lattice as lat

import helpers as H


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _members(Lc, B2):
    """(aggregate, site in block) of every level-1 site, by loops over coordinates."""
    Lb = [Lc[m] // B2[m] for m in range(4)]
    Vc1 = int(np.prod(Lc))
    agg = np.empty(Vc1, dtype=np.int64)
    loc = np.empty(Vc1, dtype=np.int64)
    for t in range(Lc[3]):
        for z in range(Lc[2]):
            for y in range(Lc[1]):
                for x in range(Lc[0]):
                    s = ((t * Lc[2] + z) * Lc[1] + y) * Lc[0] + x
                    b = [x // B2[0], y // B2[1], z // B2[2], t // B2[3]]
                    l = [x % B2[0], y % B2[1], z % B2[2], t % B2[3]]
                    agg[s] = ((b[3] * Lb[2] + b[2]) * Lb[1] + b[1]) * Lb[0] + b[0]
                    loc[s] = ((l[3] * B2[2] + l[2]) * B2[1] + l[1]) * B2[0] + l[0]
    return agg, loc


def _dense_R2(Q2, Lc, B2):
    """R2 as a dense (2 N_tv2 Vc2 x 2 N_tv1 Vc1) matrix, by loops: row (i, h, j), column
    (s, h, k) holds conj(Q2[i, h, v(s) N_tv1 + k, j]) for the sites s of aggregate i."""
    Vc2, _, n2, ntv2 = Q2.shape
    Vc1 = int(np.prod(Lc))
    ntv1 = n2 // int(np.prod(B2))
    agg, loc = _members(Lc, B2)
    R = np.zeros((Vc2 * 2 * ntv2, Vc1 * 2 * ntv1), dtype=np.complex128)
    for s in range(Vc1):
        i, v = agg[s], loc[s]
        for h in range(2):
            for j in range(ntv2):
                for k in range(ntv1):
                    R[(i * 2 + h) * ntv2 + j, (s * 2 + h) * ntv1 + k] = np.conj(Q2[i, h, v * ntv1 + k, j])
    return R


def _gamma5_hermitian_dc(rng, Lc, ntv1):
    """A random coarse stencil that is gamma_5-hermitian (Eq. dagger): the -mu block of
    site i is G Dc[nbr(i, -mu), +mu]^dagger G, the self block (X + G X^dagger G) / 2."""
    Vc1 = int(np.prod(Lc))
    nc1 = 2 * ntv1
    G = np.diag(np.r_[np.ones(ntv1), -np.ones(ntv1)])
    nbr = lat.coarse_neighbours(Lc)
    Dc = _rand(rng, (Vc1, 9, nc1, nc1))
    for i in range(Vc1):
        Dc[i, 0] = 0.5 * (Dc[i, 0] + G @ Dc[i, 0].conj().T @ G)
    for mu in range(4):
        for i in range(Vc1):
            Dc[i, 2 + 2 * mu] = G @ Dc[nbr[i, 2 + 2 * mu], 1 + 2 * mu].conj().T @ G
    return Dc, G


CASES = [((4, 2, 6, 4), (2, 1, 3, 2), 3, 2),  # extent-1 and extent-3 blocks; level-2 lattice 2^4
         ((4, 4, 2, 2), (2, 2, 1, 1), 2, 3),
         ((6, 2, 2, 4), (2, 1, 1, 2), 2, 2)]  # level-2 extent 3 in x: +x and -x neighbours differ


@pytest.mark.parametrize("Lc,B2,ntv1,ntv2", CASES)
def test_aggregates2_membership_and_round_trip(Lc, B2, ntv1, ntv2):
    rng = np.random.default_rng(1)
    Vc1 = int(np.prod(Lc))
    v = _rand(rng, (Vc1, 2, ntv1, 3))
    a = mg3.to_aggregates2(v, Lc, B2)
    agg, loc = _members(Lc, B2)
    for s in range(Vc1):
        for h in range(2):
            np.testing.assert_array_equal(a[agg[s], h, loc[s] * ntv1:(loc[s] + 1) * ntv1], v[s, h])
    np.testing.assert_array_equal(mg3.from_aggregates2(a, Lc, B2), v)


@pytest.mark.parametrize("Lc,B2,ntv1,ntv2", CASES)
def test_q2_orthonormal_spanning(Lc, B2, ntv1, ntv2):
    rng = np.random.default_rng(2)
    tv2 = _rand(rng, (int(np.prod(Lc)), 2, ntv1, ntv2))
    Q2 = mg3.orthonormalize2(tv2, Lc, B2)
    W = mg3.to_aggregates2(tv2, Lc, B2)
    for i in range(Q2.shape[0]):
        for h in range(2):
            q = Q2[i, h]
            assert np.abs(q.conj().T @ q - np.eye(ntv2)).max() < 1e-13
            assert np.abs(q @ (q.conj().T @ W[i, h]) - W[i, h]).max() < 1e-12 * np.abs(W[i, h]).max()


@pytest.mark.parametrize("Lc,B2,ntv1,ntv2", CASES)
def test_coarse2_operator_is_the_galerkin_product(Lc, B2, ntv1, ntv2):
    """dense(D_cc) = R2 dense(D_c) R2^dagger with R2 written out by loops; any D_c."""
    rng = np.random.default_rng(3)
    Vc1 = int(np.prod(Lc))
    Dc = _rand(rng, (Vc1, 9, 2 * ntv1, 2 * ntv1))
    tv2 = _rand(rng, (Vc1, 2, ntv1, ntv2))
    Q2 = mg3.orthonormalize2(tv2, Lc, B2)
    Dcc = mg3.coarse2_operator(Dc, Q2, Lc, B2)
    Lc2 = lat.coarse_dims(Lc, B2)
    R2 = _dense_R2(Q2, Lc, B2)
    ref = R2 @ coarse.dense_coarse(Dc, Lc) @ R2.conj().T
    got = coarse.dense_coarse(Dcc, Lc2)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # the application agrees with the dense product as well
    x = _rand(rng, (int(np.prod(Lc2)), 2, ntv2))
    y = coarse.coarse_apply(Dcc, x, Lc2)
    assert np.abs(y.ravel() - ref @ x.ravel()).max() < 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("Lc,B2,ntv1,ntv2", CASES)
def test_gamma5_hermiticity_carries_to_level2(Lc, B2, ntv1, ntv2):
    rng = np.random.default_rng(4)
    Dc, G1 = _gamma5_hermitian_dc(rng, Lc, ntv1)
    D1 = coarse.dense_coarse(Dc, Lc)
    g1 = np.kron(np.eye(int(np.prod(Lc))), G1)
    assert np.abs(g1 @ D1 @ g1 - D1.conj().T).max() < 1e-12 * np.abs(D1).max()
    Q2 = mg3.orthonormalize2(_rand(rng, (int(np.prod(Lc)), 2, ntv1, ntv2)), Lc, B2)
    Lc2 = lat.coarse_dims(Lc, B2)
    D2 = coarse.dense_coarse(mg3.coarse2_operator(Dc, Q2, Lc, B2), Lc2)
    G2 = np.diag(np.r_[np.ones(ntv2), -np.ones(ntv2)])
    g2 = np.kron(np.eye(int(np.prod(Lc2))), G2)
    assert np.abs(g2 @ D2 @ g2 - D2.conj().T).max() < 1e-12 * np.abs(D2).max()


def test_identity_coarsening_keeps_dc():
    """B2 = 1 and the unit vectors as test vectors: Q2 = I, so D_cc = D_c, R2 = P2 = 1."""
    Lc, ntv1 = (2, 4, 2, 2), 3
    rng = np.random.default_rng(5)
    Vc1 = int(np.prod(Lc))
    Dc = _rand(rng, (Vc1, 9, 2 * ntv1, 2 * ntv1))
    tv2 = np.zeros((Vc1, 2, ntv1, ntv1), dtype=np.complex128)
    tv2[:, :, np.arange(ntv1), np.arange(ntv1)] = 1.0
    Q2 = mg3.orthonormalize2(tv2, Lc, (1, 1, 1, 1))
    np.testing.assert_allclose(mg3.coarse2_operator(Dc, Q2, Lc, (1, 1, 1, 1)), Dc, rtol=0, atol=1e-14)
    y = _rand(rng, (Vc1, 2, ntv1))
    np.testing.assert_allclose(mg3.restrict2(Q2, y, Lc, (1, 1, 1, 1)), y, atol=1e-14)
    np.testing.assert_allclose(mg3.prolong2(Q2, y, Lc, (1, 1, 1, 1)), y, atol=1e-14)


def test_mr_step_is_the_least_squares_step():
    """One MR step: alpha minimises ||r - alpha D r|| (LAPACK least squares), the new
    residual is orthogonal to D r; n steps never raise the residual."""
    Lc, ntv1 = (2, 2, 4, 2), 3
    rng = np.random.default_rng(6)
    Vc1 = int(np.prod(Lc))
    Dc = _rand(rng, (Vc1, 9, 2 * ntv1, 2 * ntv1))
    Dc[:, 0] += 12 * np.eye(2 * ntv1)  # keep it well away from singular
    A = coarse.dense_coarse(Dc, Lc)
    b = _rand(rng, (Vc1, 2, ntv1))
    apply = lambda v: coarse.coarse_apply(Dc, v, Lc)
    x1 = mg3.mr(apply, b, 1)
    w = A @ b.ravel()
    alpha = np.linalg.lstsq(w[:, None], b.ravel(), rcond=None)[0][0]
    assert np.abs(x1.ravel() - alpha * b.ravel()).max() < 1e-12 * np.abs(x1).max()
    r1 = b.ravel() - A @ x1.ravel()
    assert abs(np.vdot(w, r1)) < 1e-10 * np.linalg.norm(w) * np.linalg.norm(r1)
    prev = np.linalg.norm(b)
    for n in (1, 2, 3, 5):
        rn = np.linalg.norm(b.ravel() - A @ mg3.mr(apply, b, n).ravel())
        assert rn <= prev * (1 + 1e-12)
        prev = rn


def test_exact_coarse_correction_is_galerkin_orthogonal():
    """With no smoothing and an exact level-2 solve the two-grid result leaves a residual
    that R2 maps to zero."""
    Lc, B2, ntv1, ntv2 = (4, 2, 2, 4), (2, 1, 1, 2), 2, 3
    rng = np.random.default_rng(7)
    Vc1 = int(np.prod(Lc))
    Dc = _rand(rng, (Vc1, 9, 2 * ntv1, 2 * ntv1))
    Dc[:, 0] += 10 * np.eye(2 * ntv1)
    l2 = mg3.Level2(Dc, Lc, B2, _rand(rng, (Vc1, 2, ntv1, ntv2)), n_mr=0, tol=1e-13, restart=200,
                    max_applies=400)
    y = _rand(rng, (Vc1, 2, ntv1))
    x = l2.two_grid(y)
    r = y - coarse.coarse_apply(Dc, x, Lc)
    rc = mg3.restrict2(l2.Q2, r, Lc, B2)
    assert np.linalg.norm(rc) < 1e-10 * np.linalg.norm(y)
    # and the dense statement of the same: x = P2 (R2 A P2)^{-1} R2 y
    R2 = _dense_R2(l2.Q2, Lc, B2)
    A = coarse.dense_coarse(Dc, Lc)
    ref = R2.conj().T @ np.linalg.solve(R2 @ A @ R2.conj().T, R2 @ y.ravel())
    assert np.abs(x.ravel() - ref).max() < 1e-9 * np.abs(ref).max()


def test_three_level_cycle_reduces_to_two_level_with_identity_coarsening():
    """B2 = 1, unit test vectors and no level-1 smoothing: the level-1 cycle is the same
    FGMRES on the same operator, so the three-level V-cycle is the two-level one."""
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    seed = 31
    U = H.links_field(seed, 0.3, L)
    from oracle import dirac
    C = dirac.clover_field(U, H.CSW)
    tv = H.tv_field(seed, 3, L)
    h = mg.Hierarchy(U, C, H.M0, L, B, n_smoother=1, n_mr=2, coarse_tol=0.1, coarse_restart=8,
                     coarse_max_applies=16)
    h.build_coarse(tv)
    Lc = h.Lc
    Vc1 = int(np.prod(Lc))
    tv2 = np.zeros((Vc1, 2, 3, 3), dtype=np.complex128)
    tv2[:, :, np.arange(3), np.arange(3)] = 1.0
    l2 = mg3.Level2(h.Dc, Lc, (1, 1, 1, 1), tv2, n_mr=0, tol=0.1, restart=8, max_applies=16)
    y = H.rhs_field(seed, 1, L)[..., 0]
    np.testing.assert_allclose(mg3.vcycle3(h, l2, y), h.vcycle(y), rtol=0, atol=1e-12 * np.abs(y).max())
