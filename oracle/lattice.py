"""Lattice geometry: blocks, aggregates and the coarse lattice (oracle).

Field arrays have axes (t, z, y, x, spin, colour, ...) so that the C-order
flattening of the site axes is lexicographic with x fastest.  Direction mu =
0, 1, 2, 3 is x, y, z, t and lives on array axis 3 - mu.

Sec. 2 of the paper divides the lattice into N_block blocks of V_block sites;
each block carries two aggregates A_i^l (spins 0, 1: gamma_5 = +1 in the
chiral basis) and A_i^r (spins 2, 3: gamma_5 = -1), each of 6 V_block degrees
of freedom.  The reading fixed here: aggregate dof n enumerates (site in block,
lexicographic x fastest; spin within the chirality, 2; colour, 3) in that
order, slowest first.
"""
import numpy as np


def axis(mu):
    return 3 - mu


def shift(f, mu, step):
    """f(x + step * mu_hat) on the periodic lattice."""
    return np.roll(f, -step, axis=axis(mu))


def coarse_dims(L, B):
    for mu in range(4):
        if L[mu] % B[mu]:
            raise ValueError("block size must divide the lattice size")
    return tuple(L[mu] // B[mu] for mu in range(4))


def coords_fields(L):
    """Integer coordinate arrays x_mu on the (t, z, y, x) grid."""
    t, z, y, x = np.meshgrid(*(np.arange(L[m]) for m in (3, 2, 1, 0)), indexing="ij")
    return (x, y, z, t)


def to_aggregates(psi, B):
    """Fine field (t,z,y,x,4,3,*rest) -> (Vc, 2, 6 V_block, *rest)."""
    Lt, Lz, Ly, Lx = psi.shape[:4]
    rest = psi.shape[6:]
    Bx, By, Bz, Bt = B
    a = psi.reshape(Lt // Bt, Bt, Lz // Bz, Bz, Ly // By, By, Lx // Bx, Bx, 2, 2, 3, *rest)
    nrest = len(rest)
    a = a.transpose(0, 2, 4, 6, 8, 1, 3, 5, 7, 9, 10, *range(11, 11 + nrest))
    Vc = (Lt // Bt) * (Lz // Bz) * (Ly // By) * (Lx // Bx)
    Vb = Bx * By * Bz * Bt
    return a.reshape(Vc, 2, 6 * Vb, *rest)


def from_aggregates(agg, L, B):
    """Inverse of to_aggregates: (Vc, 2, 6 V_block, *rest) -> fine field."""
    Lx, Ly, Lz, Lt = L
    Bx, By, Bz, Bt = B
    rest = agg.shape[3:]
    nrest = len(rest)
    a = agg.reshape(Lt // Bt, Lz // Bz, Ly // By, Lx // Bx, 2, Bt, Bz, By, Bx, 2, 3, *rest)
    a = a.transpose(0, 5, 1, 6, 2, 7, 3, 8, 4, 9, 10, *range(11, 11 + nrest))
    return a.reshape(Lt, Lz, Ly, Lx, 4, 3, *rest)


def coarse_coords(i, Lc):
    i = np.asarray(i)
    x = i % Lc[0]
    y = (i // Lc[0]) % Lc[1]
    z = (i // (Lc[0] * Lc[1])) % Lc[2]
    t = i // (Lc[0] * Lc[1] * Lc[2])
    return np.stack([x, y, z, t], axis=-1)


def coarse_index(c, Lc):
    c = np.asarray(c)
    return ((c[..., 3] * Lc[2] + c[..., 2]) * Lc[1] + c[..., 1]) * Lc[0] + c[..., 0]


# Stencil directions of the coarse operator: 0 = self, 1 + 2 mu = +mu,
# 2 + 2 mu = -mu (order 0, +x, -x, +y, -y, +z, -z, +t, -t).
NDIR = 9


def direction_offset(d):
    off = np.zeros(4, dtype=np.int64)
    if d > 0:
        mu = (d - 1) // 2
        off[mu] = 1 if d % 2 == 1 else -1
    return off


def coarse_neighbours(Lc):
    """nbr[i, d]: coarse site reached from i in stencil direction d."""
    Vc = int(np.prod(Lc))
    c = coarse_coords(np.arange(Vc), Lc)
    nbr = np.empty((Vc, NDIR), dtype=np.int64)
    for d in range(NDIR):
        nbr[:, d] = coarse_index((c + direction_offset(d)) % np.asarray(Lc), Lc)
    return nbr
