"""Two-level MG: coarse-grid correction (Alg. 2), the V-cycle preconditioner
(Alg. 1), the adaptive setup (Alg. 4) and the outer FGMRES solve (Sec. 1)
(oracle, complex128).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings fixed here where the paper prints no more:

* The V-cycle returns x = S(y; x0) with x0 = CGC(y) and S the smoother of
  Alg. 3 (SAP, smoother.sap) run for n_smoother cycles.
* CGC(y) = P x_c with x_c the coarse FGMRES solution of D_c x_c = R y to the
  relative residual coarse_tol (Alg. 2; 0.05 in the paper), either on D_c
  itself or on its even/odd Schur complement (evenodd.eo_solve).
* Alg. 4.  The random starting test vectors are an input.  The initial phase
  replaces v_j by S_k(v_j; 0) for k = 1, 2, 3 (the smoother with N_smoother = k,
  right-hand side v_j, start 0), builds R and D_c (Alg. 5), then divides each
  v_j by its norm.  Each of the n_setup iterative passes replaces every v_j, in
  order j = 1..N_tv, by S(v_j; CGC(v_j)) with the current R and D_c and the
  V-cycle's n_smoother, and rebuilds R and D_c once all N_tv vectors are
  updated.  Only the initial phase normalises (the aggregates' Gram-Schmidt
  makes the scale of v_j irrelevant to R).
* The outer solver of D u = f is right-preconditioned FGMRES (krylov.fgmres)
  with the V-cycle as its variable preconditioner.
"""
import numpy as np

from . import coarse, dirac, evenodd, krylov, smoother
from . import lattice as lat


class Hierarchy:
    """The two-level method on one gauge field: fine operator, smoother
    parameters, and the restriction (Q) and coarse operator (Dc) of Alg. 5."""

    def __init__(self, U, C, m0, L, B, Bs=None, n_smoother=4, n_mr=None, coarse_tol=0.05,
                 coarse_restart=30, coarse_max_applies=200, eo=False):
        self.U, self.C, self.m0 = U, C, m0
        self.L, self.B = tuple(L), tuple(B)
        self.Bs = tuple(B) if Bs is None else tuple(Bs)
        self.Lc = lat.coarse_dims(self.L, self.B)
        self.n_smoother, self.n_mr = n_smoother, n_mr
        self.coarse_tol, self.coarse_restart, self.coarse_max_applies = \
            coarse_tol, coarse_restart, coarse_max_applies
        self.eo = eo
        self.Bm = smoother.block_matrices(U, C, m0, self.L, self.Bs) if n_mr is None else None
        self.Q = None
        self.Dc = None

    def apply_D(self, psi):
        return dirac.apply_dirac(self.U, self.C, self.m0, psi)

    def build_coarse(self, tv):
        """Alg. 5: R from the test vectors (t,z,y,x,4,3,N_tv) and D_c = R D P."""
        self.Q = coarse.orthonormalize(tv, self.B)
        self.Dc = coarse.coarse_operator(self.U, self.C, self.m0, self.Q, self.L, self.B)

    def smooth(self, y, x0, n_cycles=None):
        n = self.n_smoother if n_cycles is None else n_cycles
        return smoother.sap(self.U, self.C, self.m0, y, x0, self.Bs, n, n_mr=self.n_mr, Bm=self.Bm)

    def coarse_solve(self, yc):
        """x_c ~ D_c^{-1} y_c to the relative residual coarse_tol (Alg. 2)."""
        if self.eo:
            Vc = self.Dc.shape[0]
            x, _, _ = evenodd.eo_solve(self.Dc, yc.reshape(Vc, -1), self.Lc, tol=self.coarse_tol,
                                       restart=self.coarse_restart, max_applies=self.coarse_max_applies)
            return x.reshape(yc.shape)
        x, _, _ = krylov.fgmres(lambda v: coarse.coarse_apply(self.Dc, v, self.Lc), yc, tol=self.coarse_tol,
                                restart=self.coarse_restart, max_applies=self.coarse_max_applies)
        return x

    def cgc(self, y):
        """Alg. 2: x = P x_c, x_c the coarse solve of R y."""
        yc = coarse.restrict(self.Q, y, self.B)
        return coarse.prolong(self.Q, self.coarse_solve(yc), self.L, self.B)

    def vcycle(self, y):
        """Alg. 1: the smoother on D x = y started from the coarse-grid correction."""
        return self.smooth(y, self.cgc(y))


def setup(h, tv0, n_setup):
    """Alg. 4 on Hierarchy h from the random test vectors tv0 (t,z,y,x,4,3,N_tv).

    Leaves R and D_c of the final test vectors in h and returns those vectors.
    """
    ntv = tv0.shape[-1]
    v = [np.array(tv0[..., j], dtype=np.complex128) for j in range(ntv)]
    zero = np.zeros_like(v[0])
    for k in (1, 2, 3):
        v = [h.smooth(vj, zero, n_cycles=k) for vj in v]
    h.build_coarse(np.stack(v, axis=-1))
    v = [vj / np.linalg.norm(vj) for vj in v]
    for _ in range(n_setup):
        for j in range(ntv):
            v[j] = h.smooth(v[j], h.cgc(v[j]))
        h.build_coarse(np.stack(v, axis=-1))
    return np.stack(v, axis=-1)


def solve(h, f, tol=1e-10, restart=30, max_applies=500):
    """D u = f by FGMRES right-preconditioned with the V-cycle (Sec. 1).
    Returns (u, relres_history, n_applies of D)."""
    return krylov.fgmres(h.apply_D, f, tol=tol, restart=restart, max_applies=max_applies, precond=h.vcycle)
