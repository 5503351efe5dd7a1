"""Restriction, Galerkin coarse operator and prolongation (oracle, complex128).

Notation of the paper (Sec. 2, Alg. 2, Alg. 5): N_tv test vectors v_j; for
block i and chirality h in {l, r} the matrix R_i^h (N_tv x 6 V_block) has in
its rows the vectors v_j^dagger restricted to aggregate A_i^h after
Gram-Schmidt; R = diag(R_1^l, R_1^r, ...), P = R^dagger (Eq. R) and
D_c = R D P (Eq. cgo).

Array conventions used throughout the oracle:

* ``Q``  (Vc, 2, 6 V_block, N_tv): column j of Q[i, h] is the orthonormal
  vector q_j on aggregate A_i^h, so R_i^h = Q[i, h]^dagger;
* coarse vectors (Vc, 2, N_tv[, k]) -- per coarse site the l block then the
  r block (2 N_tv components);
* ``Dc`` (Vc, 9, 2 N_tv, 2 N_tv): Dc[i, d] couples coarse site i to
  nbr(i, d) in stencil direction d = 0, +x, -x, +y, -y, +z, -z, +t, -t, so
  (D_c x_c)(i) = sum_d Dc[i, d] x_c(nbr(i, d)).
"""
import numpy as np

from . import dirac
from . import lattice as lat


class RankDeficient(ArithmeticError):
    pass


def gram_schmidt(W, passes=2):
    """Classical Gram-Schmidt on the columns of W, in order j = 1..N_tv.

    Alg. 5 ("run Gram-Schmidt on the rows of R_i^h") with the classical
    variant that Sec. 3 ("Gram-Schmidt on aggregates") chooses:
    q_j = (w_j - sum_{k<j} q_k <q_k, w_j>) / norm, all projections of one
    pass taken from the same vector.  The projection is repeated ``passes``
    times (re-orthogonalisation, which leaves the exact result unchanged).
    The result is the unique orthonormal Q with W = Q T, T upper triangular
    with a real positive diagonal.  A norm below 1e-12 |w_j| is rank
    deficiency.
    """
    n, N = W.shape
    Q = np.zeros_like(W)
    for j in range(N):
        w = W[:, j].copy()
        w_norm = np.linalg.norm(w)
        for _ in range(passes):
            c = Q[:, :j].conj().T @ w
            w = w - Q[:, :j] @ c
        nrm = np.linalg.norm(w)
        if not nrm > 1e-12 * w_norm:
            raise RankDeficient("test vector %d is (nearly) dependent on the previous ones" % j)
        Q[:, j] = w / nrm
    return Q


def orthonormalize(tv, B):
    """Q for every aggregate from the fine test vectors tv (t,z,y,x,4,3,N_tv)."""
    W = lat.to_aggregates(tv, B)
    Vc, _, n, N = W.shape
    Q = np.empty_like(W)
    for i in range(Vc):
        for h in range(2):
            Q[i, h] = gram_schmidt(W[i, h])
    return Q


def restrict(Q, y, B):
    """y_c = R y (Eq. R): (y_c)_i^h = R_i^h y|_{A_i^h}."""
    ya = lat.to_aggregates(y, B)
    if ya.ndim == 3:
        return np.einsum("ihnj,ihn->ihj", Q.conj(), ya)
    return np.einsum("ihnj,ihnk->ihjk", Q.conj(), ya)


def prolong(Q, xc, L, B):
    """x = P x_c with P = R^dagger (Alg. 2): x|_{A_i^h} = Q[i, h] (x_c)_i^h."""
    if xc.ndim == 3:
        xa = np.einsum("ihnj,ihj->ihn", Q, xc)
    else:
        xa = np.einsum("ihnj,ihjk->ihnk", Q, xc)
    return lat.from_aggregates(xa, L, B)


def _column_fields(Q, L, B):
    """The 2 N_tv columns of P as fine fields (t,z,y,x,4,3,2 N_tv).

    Column c < N_tv is q_c of the l aggregate of every block, column
    N_tv + j is q_j of the r aggregate; each block carries its own columns.
    """
    Vc, _, n, N = Q.shape
    cols = np.zeros((Vc, 2, n, 2 * N), dtype=np.complex128)
    cols[:, 0, :, :N] = Q[:, 0]
    cols[:, 1, :, N:] = Q[:, 1]
    return lat.from_aggregates(cols, L, B)


def coarse_operator(U, C, m0, Q, L, B, sites=None):
    """(D_c)_{i,d} = R_i H_d P_{nbr(i,d)} for every stencil direction d.

    Eq. cgo, (D_c)_ij^{hh'} = R_i^h D_ij^{hh'} P_j^{h'}, evaluated directly
    for d = 0 and all eight neighbours (no use of Eq. dagger), with H_d the
    block part of D (dirac.apply_block_part).  When the coarse extent is 2
    the +mu and -mu neighbours coincide; the two faces stay separate blocks
    whose sum is the full coupling.  ``sites`` restricts the output to the
    listed coarse sites.
    """
    Vc, _, n, N = Q.shape
    if sites is None:
        sites = np.arange(Vc)
    sites = np.asarray(sites)
    Psi = _column_fields(Q, L, B)
    Dc = np.empty((len(sites), lat.NDIR, 2 * N, 2 * N), dtype=np.complex128)
    for d in range(lat.NDIR):
        Phi = lat.to_aggregates(dirac.apply_block_part(U, C, m0, Psi, B, d), B)
        for h in range(2):
            Dc[:, d, h * N:(h + 1) * N, :] = np.einsum(
                "inj,inc->ijc", Q[sites, h].conj(), Phi[sites, h])
    return Dc


def coarse_apply(Dc, xc, Lc):
    """y_c = D_c x_c: y_c(i) = sum_d Dc[i, d] x_c(nbr(i, d)) (Alg. 2)."""
    Vc = Dc.shape[0]
    nc = Dc.shape[2]
    nbr = lat.coarse_neighbours(Lc)
    x = xc.reshape((Vc, nc) + xc.shape[3:])
    y = np.zeros_like(x)
    for d in range(lat.NDIR):
        y += np.einsum("iac,ic...->ia...", Dc[:, d], x[nbr[:, d]])
    return y.reshape(xc.shape)


def abs_apply(Dc, xc, Lc):
    """|D_c| |x_c| entrywise (for the reduced-precision error bound)."""
    return coarse_apply(np.abs(Dc).astype(np.complex128),
                        np.abs(xc).astype(np.complex128), Lc).real


def gamma5_coarse(N):
    """Coarse gamma_5: +1 on the l block, -1 on the r block of a site."""
    return np.concatenate([np.ones(N), -np.ones(N)])


def aggregate_dof_indices(L, B):
    """Fine dof index (s*12 + spin*3 + colour) of every aggregate dof."""
    V = int(np.prod(L))
    idx = np.arange(12 * V).reshape(L[3], L[2], L[1], L[0], 4, 3)
    return lat.to_aggregates(idx, B)


def dense_restriction(Q, L, B):
    """R as a dense (2 N_tv Vc x 12 V) matrix; row i*2N_tv + h*N_tv + j."""
    Vc, _, n, N = Q.shape
    V = int(np.prod(L))
    idx = aggregate_dof_indices(L, B)
    R = np.zeros((2 * N * Vc, 12 * V), dtype=np.complex128)
    for i in range(Vc):
        for h in range(2):
            rows = i * 2 * N + h * N + np.arange(N)
            R[np.ix_(rows, idx[i, h])] = Q[i, h].conj().T
    return R


def dense_coarse(Dc, Lc):
    """D_c assembled as a dense (2 N_tv Vc)^2 matrix from its stencil blocks."""
    Vc, _, nc, _ = Dc.shape
    nbr = lat.coarse_neighbours(Lc)
    M = np.zeros((nc * Vc, nc * Vc), dtype=np.complex128)
    for i in range(Vc):
        for d in range(lat.NDIR):
            j = nbr[i, d]
            M[i * nc:(i + 1) * nc, j * nc:(j + 1) * nc] += Dc[i, d]
    return M


def reduced_precision_bound(Dc, xc, Lc, u_store, u_acc=2.0 ** -24):
    """Relative error bound of one D_c application with rounded D_c entries.

    Each stored entry carries a relative error of at most u_store (rounding
    to nearest), and a length-K FP32 sum adds at most K u_acc, K = 9 * 2N:
    |dy| <= (u_store + (K + 2) u_acc) |D_c| |x|, hence
    ||dy|| / ||y|| <= (u_store + (K + 2) u_acc) || |D_c||x| || / ||D_c x||.
    """
    nc = Dc.shape[2]
    K = lat.NDIR * nc
    y = coarse_apply(Dc, xc, Lc)
    ay = abs_apply(Dc, xc, Lc)
    return (u_store + (K + 2) * u_acc) * np.linalg.norm(ay) / np.linalg.norm(y)
