"""A third level: the coarse grid coarsened once more (oracle, complex128).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3 describes two levels and notes that most of it carries over to three or
more, except a domain-decomposition smoother on a coarse grid, which the paper
does not have.  The readings fixed here:

* Level-2 aggregates.  The coarse lattice (level 1, Lc) is divided into blocks
  B2 of coarse sites; each block carries two aggregates, one per chirality
  (the l and r halves of a coarse site's 2 N_tv components, the split that
  makes D_c gamma_5-compatible, Sec. 2), each of N_tv1 V_block2 degrees of
  freedom, enumerated (site in block, lexicographic x fastest; component)
  slowest first -- the order lattice.to_aggregates uses on the fine grid.
* The level-2 test vectors are level-1 vectors (Vc1, 2, N_tv1, N_tv2), given as
  input; Q2 is their per-aggregate Gram-Schmidt (coarse.gram_schmidt, the same
  classical variant as Alg. 5).  R2 = Q2^dagger, P2 = Q2, D_cc = R2 D_c P2
  (Eq. cgo one level down).
* The coarse-grid smoother is n_mr minimal-residual steps on D_c from 0
  (x += alpha r, r -= alpha D_c r with alpha = <D_c r, r> / <D_c r, D_c r>),
  the one-vector case of the GMRES that Alg. 2 already uses.
* One two-grid cycle on level 1 (two_grid): x = MR(y); x += P2 x_cc with x_cc
  the FGMRES solution of D_cc x_cc = R2 (y - D_c x); x += MR(y - D_c x).
* The three-level V-cycle replaces the coarse solve of Alg. 2 in the
  two-level V-cycle (mg.Hierarchy.vcycle) by one two-grid cycle on level 1.
"""
import numpy as np

from . import coarse, krylov
from . import lattice as lat


def to_aggregates2(v, Lc, B2):
    """Level-1 vector (Vc1, 2, N_tv1, *rest) -> (Vc2, 2, V_block2 N_tv1, *rest)."""
    Lx, Ly, Lz, Lt = Lc
    Bx, By, Bz, Bt = B2
    ntv1 = v.shape[2]
    rest = v.shape[3:]
    a = v.reshape(Lt // Bt, Bt, Lz // Bz, Bz, Ly // By, By, Lx // Bx, Bx, 2, ntv1, *rest)
    nrest = len(rest)
    a = a.transpose(0, 2, 4, 6, 8, 1, 3, 5, 7, 9, *range(10, 10 + nrest))
    Vc2 = (Lt // Bt) * (Lz // Bz) * (Ly // By) * (Lx // Bx)
    return a.reshape(Vc2, 2, Bx * By * Bz * Bt * ntv1, *rest)


def from_aggregates2(a, Lc, B2):
    """Inverse of to_aggregates2."""
    Lx, Ly, Lz, Lt = Lc
    Bx, By, Bz, Bt = B2
    Vb2 = Bx * By * Bz * Bt
    ntv1 = a.shape[2] // Vb2
    rest = a.shape[3:]
    nrest = len(rest)
    v = a.reshape(Lt // Bt, Lz // Bz, Ly // By, Lx // Bx, 2, Bt, Bz, By, Bx, ntv1, *rest)
    v = v.transpose(0, 5, 1, 6, 2, 7, 3, 8, 4, 9, *range(10, 10 + nrest))
    return v.reshape(Lt * Lz * Ly * Lx, 2, ntv1, *rest)


def orthonormalize2(tv2, Lc, B2):
    """Q2 (Vc2, 2, V_block2 N_tv1, N_tv2) from the level-1 test vectors."""
    W = to_aggregates2(tv2, Lc, B2)
    Q = np.empty_like(W)
    for i in range(W.shape[0]):
        for h in range(2):
            Q[i, h] = coarse.gram_schmidt(W[i, h])
    return Q


def restrict2(Q2, v, Lc, B2):
    """y_cc = R2 y_c: (y_cc)_i^h = Q2[i, h]^dagger y_c|_{A_i^h}."""
    a = to_aggregates2(v, Lc, B2)
    return np.einsum("ihnj,ihn...->ihj...", Q2.conj(), a)


def prolong2(Q2, xcc, Lc, B2):
    """x_c = P2 x_cc with P2 = R2^dagger."""
    return from_aggregates2(np.einsum("ihnj,ihj...->ihn...", Q2, xcc), Lc, B2)


def hop_class(Lc, B2):
    """cls[s, e]: the level-2 stencil direction of the coupling D_c[s, e].

    0 when the site D_c[s, e] reaches lies in the block of s (the self part of
    the level-2 operator), 1 + 2 mu when e = +mu leaves the block through its
    +mu face, 2 + 2 mu when e = -mu leaves through its -mu face (a block of
    extent 1 is left by both).
    """
    Vc1 = int(np.prod(Lc))
    c = lat.coarse_coords(np.arange(Vc1), Lc)
    cls = np.zeros((Vc1, lat.NDIR), dtype=np.int64)
    for mu in range(4):
        lc = c[:, mu] % B2[mu]
        cls[:, 1 + 2 * mu] = np.where(lc == B2[mu] - 1, 1 + 2 * mu, 0)
        cls[:, 2 + 2 * mu] = np.where(lc == 0, 2 + 2 * mu, 0)
    return cls


def coarse2_operator(Dc, Q2, Lc, B2):
    """(D_cc)_{i,d} = R2_i H_d P2_{nbr(i,d)}, the part of D_c of hop class d
    between aggregate i and its level-2 neighbour in direction d.

    All columns of P2 are placed at once (every block carries its own, as in
    coarse._column_fields); H_d keeps the couplings D_c[s, e] of class d."""
    Vc1, _, nc1, _ = Dc.shape
    ntv1 = nc1 // 2
    Vc2, _, n2, ntv2 = Q2.shape
    cols = np.zeros((Vc2, 2, n2, 2 * ntv2), dtype=np.complex128)
    cols[:, 0, :, :ntv2] = Q2[:, 0]
    cols[:, 1, :, ntv2:] = Q2[:, 1]
    Psi = from_aggregates2(cols, Lc, B2).reshape(Vc1, nc1, 2 * ntv2)
    nbr = lat.coarse_neighbours(Lc)
    cls = hop_class(Lc, B2)
    Dcc = np.empty((Vc2, lat.NDIR, 2 * ntv2, 2 * ntv2), dtype=np.complex128)
    for d in range(lat.NDIR):
        Phi = np.zeros((Vc1, nc1, 2 * ntv2), dtype=np.complex128)
        for e in range(lat.NDIR):
            m = cls[:, e] == d
            Phi[m] += np.einsum("sab,sbc->sac", Dc[m, e], Psi[nbr[m, e]])
        Pa = to_aggregates2(Phi.reshape(Vc1, 2, ntv1, 2 * ntv2), Lc, B2)
        for h in range(2):
            Dcc[:, d, h * ntv2:(h + 1) * ntv2, :] = np.einsum("inj,inc->ijc", Q2[:, h].conj(), Pa[:, h])
    return Dcc


def mr(apply, b, n):
    """n minimal-residual steps on apply(x) = b from x = 0 (the smoother of level 1)."""
    x = np.zeros_like(b)
    r = np.array(b, dtype=np.complex128)
    for _ in range(n):
        w = apply(r)
        ww = np.vdot(w.ravel(), w.ravel()).real
        if ww == 0:
            break
        alpha = np.vdot(w.ravel(), r.ravel()) / ww
        x = x + alpha * r
        r = r - alpha * w
    return x


class Level2:
    """The level-2 operator of a two-level hierarchy and the two-grid cycle on level 1."""

    def __init__(self, Dc, Lc, B2, tv2, n_mr=2, tol=0.05, restart=30, max_applies=200):
        self.Dc, self.Lc, self.B2 = Dc, tuple(Lc), tuple(B2)
        self.Lc2 = lat.coarse_dims(self.Lc, self.B2)
        self.Q2 = orthonormalize2(tv2, self.Lc, self.B2)
        self.Dcc = coarse2_operator(Dc, self.Q2, self.Lc, self.B2)
        self.n_mr, self.tol, self.restart, self.max_applies = n_mr, tol, restart, max_applies

    def apply_Dc(self, v):
        return coarse.coarse_apply(self.Dc, v, self.Lc)

    def apply_Dcc(self, v):
        return coarse.coarse_apply(self.Dcc, v, self.Lc2)

    def two_grid(self, y):
        """One two-grid cycle on level 1 for D_c x = y (y: (Vc1, 2, N_tv1[, k]))."""
        x = self.mr_cols(y)
        r = y - self.apply_Dc(x)
        ycc = restrict2(self.Q2, r, self.Lc, self.B2)
        xcc = self.solve_cols(ycc)
        x = x + prolong2(self.Q2, xcc, self.Lc, self.B2)
        r = y - self.apply_Dc(x)
        return x + self.mr_cols(r)

    def mr_cols(self, b):
        if b.ndim == 3:
            return mr(self.apply_Dc, b, self.n_mr)
        return np.stack([mr(self.apply_Dc, b[..., k], self.n_mr) for k in range(b.shape[-1])], axis=-1)

    def solve_cols(self, b):
        def one(v):
            x, _, _ = krylov.fgmres(self.apply_Dcc, v, tol=self.tol, restart=self.restart,
                                    max_applies=self.max_applies)
            return x
        if b.ndim == 3:
            return one(b)
        return np.stack([one(b[..., k]) for k in range(b.shape[-1])], axis=-1)


def vcycle3(h, l2, y):
    """The three-level V-cycle: Alg. 1 with the coarse solve of Alg. 2 replaced by one
    two-grid cycle on level 1 (h: mg.Hierarchy, l2: Level2 built on h.Dc)."""
    yc = coarse.restrict(h.Q, y, h.B)
    return h.smooth(y, coarse.prolong(h.Q, l2.two_grid(yc), h.L, h.B))


def solve3(h, l2, f, tol=1e-10, restart=30, max_applies=500):
    """D u = f by FGMRES right-preconditioned with the three-level V-cycle."""
    return krylov.fgmres(h.apply_D, f, tol=tol, restart=restart, max_applies=max_applies,
                         precond=lambda v: vcycle3(h, l2, v))
