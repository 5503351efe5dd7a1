"""Pins of the oracle's two-level method: the smoother of Alg. 3 (SAP with exact or
minimal-residual block solves), the coarse-grid correction (Alg. 2), the V-cycle
(Alg. 1), the adaptive setup (Alg. 4) and the outer FGMRES (Sec. 1).

Expected values come from the entry-by-entry dense D (dirac.dense_dirac, itself
pinned by the free-field spectrum and gamma_5-hermiticity): block matrices cut out
of it with block membership computed by explicit loops here, error propagators
written as dense matrix products, a per-block MR loop on those dense blocks, a
scalar least-squares solve for the MR step, LAPACK solves and least squares; and
from invariants that hold whatever the input (a fixed point, a vanishing residual).
"""
import numpy as np
import pytest

from oracle import coarse, dirac, krylov, mg, smoother
from oracle import lattice as lat

import helpers as H

L4, B2 = (4, 4, 4, 4), (2, 2, 2, 2)


def _block_ids(L, Bs):
    """Block number and colour of every site, by loops (x fastest everywhere)."""
    Lb = [L[m] // Bs[m] for m in range(4)]
    V = int(np.prod(L))
    blk = np.empty(V, dtype=np.int64)
    for t in range(L[3]):
        for z in range(L[2]):
            for y in range(L[1]):
                for x in range(L[0]):
                    s = ((t * L[2] + z) * L[1] + y) * L[0] + x
                    b = [x // Bs[0], y // Bs[1], z // Bs[2], t // Bs[3]]
                    blk[s] = ((b[3] * Lb[2] + b[2]) * Lb[1] + b[1]) * Lb[0] + b[0]
    colour = np.empty(int(np.prod(Lb)), dtype=np.int64)
    for i in range(len(colour)):
        c = [i % Lb[0], (i // Lb[0]) % Lb[1], (i // (Lb[0] * Lb[1])) % Lb[2], i // (Lb[0] * Lb[1] * Lb[2])]
        colour[i] = sum(c) % 2
    return blk, colour


class Dense:
    """The fine system as dense matrices on a tiny lattice."""

    def __init__(self, L, Bs, seed, eps=0.3):
        self.L, self.Bs = L, Bs
        self.U = H.links_field(seed, eps, L)
        self.C = dirac.clover_field(self.U, H.CSW)
        self.D = dirac.dense_dirac(self.U, self.C, H.M0)
        blk, self.colour = _block_ids(L, Bs)
        self.dof_blk = np.repeat(blk, 12)
        self.blocks = [np.flatnonzero(self.dof_blk == b) for b in range(len(self.colour))]
        self.Bd = np.where(self.dof_blk[:, None] == self.dof_blk[None, :], self.D, 0)

    def K(self, colours):
        """sum over blocks of the given colours of I_b B_b^{-1} I_b^T."""
        K = np.zeros_like(self.D)
        for b, idx in enumerate(self.blocks):
            if self.colour[b] in colours:
                K[np.ix_(idx, idx)] = np.linalg.inv(self.D[np.ix_(idx, idx)])
        return K

    def field(self, v):
        return v.reshape(H.field_shape(self.L) + (4, 3))


@pytest.fixture(scope="module")
def dense():
    return Dense(L4, B2, 31)


def _vec(seed, n):
    rng = np.random.default_rng(seed)
    return rng.normal(size=n) + 1j * rng.normal(size=n)


def test_block_matrices_are_the_dense_intra_block_couplings(dense):
    Bm = smoother.block_matrices(dense.U, dense.C, H.M0, dense.L, dense.Bs)
    idx = coarse.aggregate_dof_indices(dense.L, dense.Bs).reshape(len(dense.blocks), -1)
    for b in range(len(dense.blocks)):
        assert sorted(idx[b]) == list(dense.blocks[b])
        assert np.abs(Bm[b] - dense.D[np.ix_(idx[b], idx[b])]).max() < 1e-14
    # B psi is the dense block-diagonal part of D applied to psi
    v = _vec(1, dense.D.shape[0])
    got = smoother.block_apply(dense.U, dense.C, H.M0, dense.field(v), dense.Bs).ravel()
    assert np.abs(got - dense.Bd @ v).max() < 1e-13 * np.abs(dense.Bd @ v).max()


def test_block_colouring(dense):
    col = smoother.block_colour(dense.L, dense.Bs).ravel()
    blk = dense.dof_blk[::12]
    assert np.array_equal(col, dense.colour[blk])
    # no coupling of D joins two different blocks of one colour
    for b1, i1 in enumerate(dense.blocks):
        for b2, i2 in enumerate(dense.blocks):
            if b1 != b2 and dense.colour[b1] == dense.colour[b2]:
                assert not np.any(dense.D[np.ix_(i1, i2)])


def test_one_mr_step_is_the_scalar_least_squares_step(dense):
    r = _vec(2, dense.D.shape[0])
    mask = np.ones(H.field_shape(dense.L), dtype=bool)
    e = smoother.block_solve_mr(dense.U, dense.C, H.M0, dense.field(r), mask, dense.Bs, 1).ravel()
    for idx in dense.blocks:
        Bb = dense.D[np.ix_(idx, idx)]
        p = Bb @ r[idx]
        alpha, *_ = np.linalg.lstsq(p[:, None], r[idx], rcond=None)
        assert np.abs(e[idx] - alpha[0] * r[idx]).max() < 1e-13 * np.abs(e[idx]).max()


def test_mr_block_solve_equals_a_dense_per_block_mr_loop(dense):
    r = _vec(3, dense.D.shape[0])
    col = smoother.block_colour(dense.L, dense.Bs)
    e = smoother.block_solve_mr(dense.U, dense.C, H.M0, dense.field(r), col == 1, dense.Bs, 5).ravel()
    want = np.zeros_like(r)
    for b, idx in enumerate(dense.blocks):
        if dense.colour[b] != 1:
            continue
        Bb = dense.D[np.ix_(idx, idx)]
        rho, x = r[idx].copy(), np.zeros(len(idx), dtype=complex)
        for _ in range(5):
            p = Bb @ rho
            a = np.vdot(p, rho) / np.vdot(p, p)
            x += a * rho
            rho -= a * p
        want[idx] = x
    assert np.abs(e - want).max() < 1e-12 * np.abs(want).max()


def test_mr_converges_to_the_exact_block_solve(dense):
    """With a positive definite Hermitian part MR converges (Saad, Thm. 5.10)."""
    for idx in dense.blocks:
        Bb = dense.D[np.ix_(idx, idx)]
        assert np.linalg.eigvalsh((Bb + Bb.conj().T) / 2).min() > 0
    r = _vec(4, dense.D.shape[0])
    mask = np.ones(H.field_shape(dense.L), dtype=bool)
    e = smoother.block_solve_mr(dense.U, dense.C, H.M0, dense.field(r), mask, dense.Bs, 400).ravel()
    want = np.linalg.solve(dense.Bd, r)
    assert np.abs(e - want).max() < 1e-9 * np.abs(want).max()


def test_sap_exact_is_the_product_of_colour_propagators(dense):
    y, x0 = _vec(5, dense.D.shape[0]), _vec(6, dense.D.shape[0])
    K0, K1 = dense.K({0}), dense.K({1})
    x = x0.copy()
    for _ in range(2):
        x = x + K0 @ (y - dense.D @ x)
        x = x + K1 @ (y - dense.D @ x)
    got = smoother.sap(dense.U, dense.C, H.M0, dense.field(y), dense.field(x0), dense.Bs, 2).ravel()
    assert np.abs(got - x).max() < 1e-11 * np.abs(x).max()
    # error propagator (1 - K1 D)(1 - K0 D) per cycle
    I = np.eye(dense.D.shape[0])
    E = (I - K1 @ dense.D) @ (I - K0 @ dense.D)
    u = np.linalg.solve(dense.D, y)
    assert np.abs((got - u) - E @ E @ (x0 - u)).max() < 1e-10 * np.abs(x0 - u).max()


def test_sap_additive_form_of_alg3(dense):
    y, x0 = _vec(7, dense.D.shape[0]), _vec(8, dense.D.shape[0])
    want = x0 + np.linalg.solve(dense.Bd, y - dense.D @ x0)
    got = smoother.sap(dense.U, dense.C, H.M0, dense.field(y), dense.field(x0), dense.Bs, 1, colours=1).ravel()
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


def test_sap_exact_leaves_no_residual_on_the_last_colour(dense):
    y = _vec(9, dense.D.shape[0])
    x = smoother.sap(dense.U, dense.C, H.M0, dense.field(y), dense.field(np.zeros_like(y)), dense.Bs, 1).ravel()
    r = y - dense.D @ x
    on1 = dense.colour[dense.dof_blk] == 1
    assert np.abs(r[on1]).max() < 1e-12 * np.abs(y).max()
    assert np.abs(r[~on1]).max() > 1e-3 * np.abs(y).max()


@pytest.mark.parametrize("n_mr", [None, 4])
def test_solution_is_a_fixed_point_of_the_smoother(dense, n_mr):
    y = _vec(10, dense.D.shape[0])
    u = np.linalg.solve(dense.D, y)
    got = smoother.sap(dense.U, dense.C, H.M0, dense.field(y), dense.field(u), dense.Bs, 3, n_mr=n_mr).ravel()
    assert np.abs(got - u).max() < 1e-11 * np.abs(u).max()


def test_smoother_rejects_uncolourable_block_lattices():
    L = (6, 4, 4, 4)
    U = H.links_field(1, 0.3, L)
    C = dirac.clover_field(U, H.CSW)
    y = np.zeros(H.field_shape(L) + (4, 3), dtype=complex)
    with pytest.raises(ValueError):
        smoother.sap(U, C, H.M0, y, y, (2, 2, 2, 2), 1, n_mr=2)  # 3 blocks in x
    with pytest.raises(ValueError):
        smoother.sap(U, C, H.M0, y, y, (6, 2, 2, 2), 1, n_mr=2, colours=1)  # one block spans x


def _hierarchy(dense, ntv, seed, **kw):
    h = mg.Hierarchy(dense.U, dense.C, H.M0, dense.L, dense.Bs, **kw)
    h.build_coarse(H.tv_field(seed, ntv, dense.L))
    return h


def test_cgc_with_exact_coarse_solve_is_P_Dc_inverse_R(dense):
    h = _hierarchy(dense, 6, 41, coarse_tol=1e-13, coarse_max_applies=2000)
    R = coarse.dense_restriction(h.Q, dense.L, dense.Bs)
    y = _vec(11, dense.D.shape[0])
    want = R.conj().T @ np.linalg.solve(R @ dense.D @ R.conj().T, R @ y)
    assert np.abs(h.cgc(dense.field(y)).ravel() - want).max() < 1e-10 * np.abs(want).max()
    heo = _hierarchy(dense, 6, 41, coarse_tol=1e-13, coarse_max_applies=2000, eo=True)
    assert np.abs(heo.cgc(dense.field(y)).ravel() - want).max() < 1e-10 * np.abs(want).max()


def test_cgc_with_full_rank_aggregates_inverts_D():
    """N_tv = 6 V_block makes every R_i^h unitary, so P R = 1 and CGC = D^{-1}."""
    d = Dense((2, 2, 2, 2), (1, 1, 1, 1), 43)
    h = _hierarchy(d, 6, 44, coarse_tol=1e-13, coarse_max_applies=2000)
    y = _vec(12, d.D.shape[0])
    want = np.linalg.solve(d.D, y)
    assert np.abs(h.cgc(d.field(y)).ravel() - want).max() < 1e-10 * np.abs(want).max()


def test_vcycle_is_smoother_after_cgc(dense):
    h = _hierarchy(dense, 6, 45, n_smoother=2, coarse_tol=1e-13, coarse_max_applies=2000)
    R = coarse.dense_restriction(h.Q, dense.L, dense.Bs)
    P = R.conj().T
    K0, K1 = dense.K({0}), dense.K({1})
    y = _vec(13, dense.D.shape[0])
    x = P @ np.linalg.solve(R @ dense.D @ P, R @ y)
    for _ in range(2):
        x = x + K0 @ (y - dense.D @ x)
        x = x + K1 @ (y - dense.D @ x)
    got = h.vcycle(dense.field(y)).ravel()
    assert np.abs(got - x).max() < 1e-10 * np.abs(x).max()


def test_setup_follows_alg4_step_by_step(dense):
    """Alg. 4 redone with dense propagators and a dense coarse inverse."""
    ntv, nu = 4, 2
    h = mg.Hierarchy(dense.U, dense.C, H.M0, dense.L, dense.Bs, n_smoother=nu, coarse_tol=1e-13,
                     coarse_max_applies=2000)
    tv0 = H.tv_field(46, ntv, dense.L)
    v_final = mg.setup(h, tv0, n_setup=1)
    K0, K1 = dense.K({0}), dense.K({1})
    D = dense.D

    def smooth(y, x, n):
        for _ in range(n):
            x = x + K0 @ (y - D @ x)
            x = x + K1 @ (y - D @ x)
        return x

    v = [tv0[..., j].ravel().copy() for j in range(ntv)]
    for k in (1, 2, 3):
        v = [smooth(vj, np.zeros_like(vj), k) for vj in v]
    Q = coarse.orthonormalize(np.stack([dense.field(vj) for vj in v], axis=-1), dense.Bs)
    R = coarse.dense_restriction(Q, dense.L, dense.Bs)
    v = [vj / np.linalg.norm(vj) for vj in v]
    for j in range(ntv):
        x0 = R.conj().T @ np.linalg.solve(R @ D @ R.conj().T, R @ v[j])
        v[j] = smooth(v[j], x0, nu)
    Q = coarse.orthonormalize(np.stack([dense.field(vj) for vj in v], axis=-1), dense.Bs)
    R = coarse.dense_restriction(Q, dense.L, dense.Bs)
    for j in range(ntv):
        assert np.abs(v_final[..., j].ravel() - v[j]).max() < 1e-9 * np.abs(v[j]).max()
    assert np.abs(h.Q - Q).max() < 1e-9
    Dc = coarse.dense_coarse(h.Dc, lat.coarse_dims(dense.L, dense.Bs))
    assert np.abs(Dc - R @ D @ R.conj().T).max() < 1e-9 * np.abs(Dc).max()


def test_fgmres_with_a_varying_preconditioner_minimises_over_its_search_space(dense):
    """Flexible GMRES (Saad, Prop. 9.2): after k steps x minimises ||b - D x|| over
    span{z_1..z_k}, the preconditioned vectors it actually used."""
    rng = np.random.default_rng(14)
    Z = []

    def precond(v):  # a different (random diagonal) preconditioner every call
        z = v * (1.0 + 0.5 * rng.uniform(size=v.shape))
        Z.append(z.ravel())
        return z

    b = _vec(15, dense.D.shape[0])
    x, hist, n = krylov.fgmres(lambda v: dense.D @ v, b, tol=1e-30, restart=6, max_applies=6, precond=precond)
    Zm = np.stack(Z, axis=1)
    c, *_ = np.linalg.lstsq(dense.D @ Zm, b, rcond=None)
    assert np.abs(x - Zm @ c).max() < 1e-10 * np.abs(x).max()
    assert abs(hist[-1] - np.linalg.norm(b - dense.D @ x) / np.linalg.norm(b)) < 1e-10


def test_mg_preconditioned_solve(dense):
    h = mg.Hierarchy(dense.U, dense.C, H.M0, dense.L, dense.Bs, n_smoother=2, n_mr=4)
    mg.setup(h, H.tv_field(47, 8, dense.L), n_setup=1)
    f = H.rhs_field(48, 1, dense.L)[..., 0]
    u, hist, n = mg.solve(h, f, tol=1e-10)
    want = np.linalg.solve(dense.D, f.ravel())
    assert np.abs(u.ravel() - want).max() < 1e-8 * np.abs(want).max()
    assert np.linalg.norm(f.ravel() - dense.D @ u.ravel()) / np.linalg.norm(f) < 2e-10
    # the two-level preconditioner does the work: far fewer D applications than plain GMRES
    _, _, n_plain = krylov.fgmres(lambda v: dense.D @ v, f.ravel(), tol=1e-10, restart=30, max_applies=5000)
    assert n * 10 < n_plain
