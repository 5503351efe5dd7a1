"""Even/odd (red-black) reduction of the coarse system (oracle, complex128).

Alg. 2 solves the coarse system by FGMRES "with even/odd preconditioning".
The coarse operator couples a site only to itself and to its eight nearest
neighbours, so on a coarse lattice whose extents are all even the sites split
into two checkerboard halves (parity (x + y + z + t) mod 2) with no hop inside
a half.  Ordering the unknowns even-then-odd,

    D_c = [[D_ee, D_eo], [D_oe, D_oo]],   D_ee, D_oo block diagonal (self blocks),

and block elimination of the odd half gives the Schur complement
S = D_ee - D_eo D_oo^{-1} D_oe on the even half.  The reading fixed here: the
coarse solve runs FGMRES on S x_e = b_e - D_eo D_oo^{-1} b_o and then recovers
x_o = D_oo^{-1} (b_o - D_oe x_e) (the standard even/odd reduction; the paper
names the method without writing it out).

Half vectors list the sites of one parity in lexicographic order; on a lattice
with even L_x the site i of either parity is entry i // 2 of its half.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np

from . import coarse, krylov, lattice as lat


def check_even(Lc):
    if any(int(l) % 2 for l in Lc):
        raise ValueError("even/odd reduction needs every coarse extent even: %s" % (tuple(Lc),))


def parity(Lc):
    """Checkerboard parity of every coarse site (lexicographic, x fastest)."""
    c = lat.coarse_coords(np.arange(int(np.prod(Lc))), Lc)
    return c.sum(axis=-1) % 2


def split(v, Lc):
    """Full coarse vector [Vc, nc, ...] -> (even half, odd half)."""
    check_even(Lc)
    p = parity(Lc)
    return v[p == 0], v[p == 1]


def merge(ve, vo, Lc):
    check_even(Lc)
    p = parity(Lc)
    v = np.zeros((len(p),) + ve.shape[1:], dtype=np.complex128)
    v[p == 0] = ve
    v[p == 1] = vo
    return v


def self_inverses(Dc, Lc):
    """D_oo^{-1}: the inverse of the self block D_c[i, 0] of every odd site i."""
    p = parity(Lc)
    return np.linalg.inv(Dc[p == 1, 0])


def _apply_full(Dc, ve, vo, Lc):
    """(D_c (v_e, v_o)) split into halves, by the stencil definition (vectors [.., nc, ...])."""
    v = merge(ve, vo, Lc)
    nc = v.shape[1]
    y = coarse.coarse_apply(Dc, v.reshape((v.shape[0], 2, nc // 2) + v.shape[2:]), Lc)
    return split(y.reshape(v.shape), Lc)


def schur_apply(Dc, xe, Lc, Dinv=None):
    """S x_e = D_ee x_e - D_eo D_oo^{-1} D_oe x_e (x_e: [Vc/2, nc, ...])."""
    if Dinv is None:
        Dinv = self_inverses(Dc, Lc)
    zero_o = np.zeros_like(xe)
    ye, zo = _apply_full(Dc, xe, zero_o, Lc)       # D_ee x_e, D_oe x_e
    wo = np.einsum("iac,ic...->ia...", Dinv, zo)   # D_oo^{-1} D_oe x_e
    zero_e = np.zeros_like(xe)
    de, _ = _apply_full(Dc, zero_e, wo, Lc)        # D_eo w_o
    return ye - de


def reduced_rhs(Dc, b, Lc, Dinv=None):
    """b_e - D_eo D_oo^{-1} b_o, and b_o, for a full right-hand side b."""
    if Dinv is None:
        Dinv = self_inverses(Dc, Lc)
    be, bo = split(b, Lc)
    wo = np.einsum("iac,ic...->ia...", Dinv, bo)
    de, _ = _apply_full(Dc, np.zeros_like(be), wo, Lc)
    return be - de, bo


def reconstruct_odd(Dc, xe, bo, Lc, Dinv=None):
    """x_o = D_oo^{-1} (b_o - D_oe x_e)."""
    if Dinv is None:
        Dinv = self_inverses(Dc, Lc)
    _, zo = _apply_full(Dc, xe, np.zeros_like(xe), Lc)
    return np.einsum("iac,ic...->ia...", Dinv, bo - zo)


def eo_solve(Dc, b, Lc, tol=0.05, restart=30, max_applies=200):
    """Even/odd-reduced coarse solve of D_c x = b for one right-hand side b [Vc, nc].

    Returns (x, relres_history, n_applies) where the history and the count are
    FGMRES's on S (each application of S streams D_c once)."""
    Dinv = self_inverses(Dc, Lc)
    rhs, bo = reduced_rhs(Dc, b, Lc, Dinv)
    xe, hist, n = krylov.fgmres(lambda v: schur_apply(Dc, v, Lc, Dinv), rhs, tol=tol, restart=restart,
                                max_applies=max_applies)
    xo = reconstruct_odd(Dc, xe, bo, Lc, Dinv)
    return merge(xe, xo, Lc), hist, n
