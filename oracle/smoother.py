"""Domain-decomposition smoother of Alg. 3 (oracle, complex128).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Alg. 3 splits D = B + Z, B the couplings inside the smoother's blocks and Z
the couplings between blocks, and iterates x <- x + B^{-1} (y - D x); the
paper adds that the Schwarz alternating procedure (SAP, Luescher 2003) is the
form used in practice.  Readings fixed here (the paper prints no more):

* B is D with every hop across a block face removed (the d = 0 part of
  dirac.apply_block_part); the smoother blocks are the aggregation blocks
  unless a caller passes others.
* SAP is the multiplicative Schwarz method over a two-colouring of the
  blocks.  A block's colour is the parity of the sum of its block
  coordinates; every extent of the block lattice must be even (and at least
  2), so that neighbouring blocks differ in colour across the periodic
  boundary too.  One SAP cycle solves on the colour-0 blocks with the current
  residual, then on the colour-1 blocks with the residual left after that.
* ``colours=1`` is the additive form Alg. 3 prints: all blocks from one
  residual (block Jacobi); the block lattice needs extents >= 2 (a block
  that spans a whole periodic direction would couple to itself across its
  face).
* Each block system B_b e = r_b is solved exactly (``n_mr=None``) or by n_mr
  minimal-residual (MR) steps from e = 0 (Saad, Iterative Methods for Sparse
  Linear Systems, Sec. 5.3.2), each block with its own step length:
  p = B rho, alpha = <p, rho> / <p, p>, e += alpha rho, rho -= alpha p.
* The residual y - D x is recomputed from x before every colour (the plain
  definition; an implementation may update it incrementally).
"""
import numpy as np

from . import dirac
from . import lattice as lat


def check_colourable(L, Bs):
    """The block lattice L / Bs must have even extents >= 2 for two colours."""
    Lb = lat.coarse_dims(L, Bs)
    if any(n % 2 or n < 2 for n in Lb):
        raise ValueError("SAP needs an even number (>= 2) of blocks in every direction")
    return Lb


def block_colour(L, Bs):
    """Colour (0 or 1) of the block holding each site, as a (t, z, y, x) array."""
    x = lat.coords_fields(L)
    return sum(x[mu] // Bs[mu] for mu in range(4)) % 2


def _site_mask(mask, psi):
    return mask.reshape(mask.shape + (1,) * (psi.ndim - 4))


def block_apply(U, C, m0, psi, Bs):
    """B psi: D psi without the hops that cross a block face (Alg. 3)."""
    return dirac.apply_block_part(U, C, m0, psi, Bs, 0)


def block_dot(a, b, Bs):
    """<a, b>_blk = sum over block blk of conj(a) b, for every block (Vb order of
    lattice.to_aggregates)."""
    A = lat.to_aggregates(a, Bs)
    Bv = lat.to_aggregates(b, Bs)
    return np.einsum("ihn,ihn->i", A.conj(), Bv)


def _per_block(values, L, Bs):
    """A field that holds values[blk] at every degree of freedom of block blk."""
    nb = values.shape[0]
    n = 6 * int(np.prod(Bs))
    agg = np.broadcast_to(values[:, None, None], (nb, 2, n))
    return lat.from_aggregates(np.ascontiguousarray(agg), L, Bs)


def block_matrices(U, C, m0, L, Bs):
    """B_b as dense (12 V_b x 12 V_b) matrices for every block, in the
    aggregate order of lattice.to_aggregates (l dofs, then r dofs).

    Column k of every block comes from one application of B to the field that
    is the k-th unit vector in every block at once (blocks do not couple
    through B).
    """
    nb = int(np.prod(lat.coarse_dims(L, Bs)))
    n = 12 * int(np.prod(Bs))
    M = np.empty((nb, n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros((nb, n), dtype=np.complex128)
        e[:, k] = 1.0
        psi = lat.from_aggregates(e.reshape(nb, 2, n // 2), L, Bs)
        M[:, :, k] = lat.to_aggregates(block_apply(U, C, m0, psi, Bs), Bs).reshape(nb, n)
    return M


def block_solve_exact(Bm, r, mask, L, Bs):
    """e with B_b e_b = r_b on the blocks where ``mask`` holds, e = 0 elsewhere."""
    nb, n, _ = Bm.shape
    R = lat.to_aggregates(r * _site_mask(mask, r), Bs).reshape(nb, n)
    E = np.linalg.solve(Bm, R[:, :, None])[:, :, 0]
    return lat.from_aggregates(E.reshape(nb, 2, n // 2), L, Bs)


def block_solve_mr(U, C, m0, r, mask, Bs, n_mr):
    """n_mr MR steps from e = 0 on B_b e_b = r_b, every block where ``mask``
    holds at once with its own step length; e = 0 elsewhere."""
    L = (r.shape[3], r.shape[2], r.shape[1], r.shape[0])
    rho = r * _site_mask(mask, r)
    e = np.zeros_like(rho)
    for _ in range(n_mr):
        p = block_apply(U, C, m0, rho, Bs)
        pp = block_dot(p, p, Bs).real
        pr = block_dot(p, rho, Bs)
        alpha = np.where(pp > 0, pr / np.where(pp > 0, pp, 1.0), 0.0)
        a = _per_block(alpha, L, Bs)
        e = e + a * rho
        rho = rho - a * p
    return e


def sap(U, C, m0, y, x0, Bs, n_cycles, n_mr=None, colours=2, Bm=None):
    """N_smoother = n_cycles cycles of the smoother of Alg. 3 on D x = y from x0.

    colours=2: SAP (colour-0 blocks, then colour-1 blocks, per cycle);
    colours=1: the additive iteration x <- x + B^{-1} (y - D x).
    n_mr=None solves each block exactly (Bm, the block_matrices, may be passed
    in to save rebuilding them); otherwise n_mr MR steps per block solve.
    """
    L = (y.shape[3], y.shape[2], y.shape[1], y.shape[0])
    if colours == 2:
        check_colourable(L, Bs)
        col = block_colour(L, Bs)
        masks = [col == 0, col == 1]
    elif colours == 1:
        if min(lat.coarse_dims(L, Bs)) < 2:
            raise ValueError("the smoother needs at least 2 blocks in every direction")
        masks = [np.ones(lat.coords_fields(L)[0].shape, dtype=bool)]
    else:
        raise ValueError("colours must be 1 or 2")
    if n_mr is None and Bm is None:
        Bm = block_matrices(U, C, m0, L, Bs)
    x = np.array(x0, dtype=np.complex128, copy=True)
    for _ in range(n_cycles):
        for mask in masks:
            r = y - dirac.apply_dirac(U, C, m0, x)
            if n_mr is None:
                x = x + block_solve_exact(Bm, r, mask, L, Bs)
            else:
                x = x + block_solve_mr(U, C, m0, r, mask, Bs, n_mr)
    return x
