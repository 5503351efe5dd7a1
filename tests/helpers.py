"""Shared test helpers: synthetic inputs in the oracle's array layout.

Workloads (WORKLOADS below): each has a fine lattice L (x, y, z, t), block B,
number of test vectors, link spread eps and a seed offset; the mass m0 and c_sw
are shared (M0, CSW).
"""
import numpy as np

from synth import inputs as si

M0 = -0.3
CSW = 1.0

# name: (L, B, ntv, eps, seed offset)
WORKLOADS = {
    "tiny_4^4_b2_ntv8": ((4, 4, 4, 4), (2, 2, 2, 2), 8, 0.3, 1),
    "fp32_32^4_b4_ntv20": ((32, 32, 32, 32), (4, 4, 4, 4), 20, 0.3, 2),
    "fp16_32^3x64_b4_ntv24": ((32, 32, 32, 64), (4, 4, 4, 4), 24, 0.3, 3),
    "bf16_48^3x96_b4_ntv24": ((48, 48, 48, 96), (4, 4, 4, 4), 24, 0.3, 4),
}


def field_shape(L):
    return (L[3], L[2], L[1], L[0])


def links_field(seed, eps, L, origin=(0, 0, 0, 0), shape=None):
    """U as (4, t, z, y, x, 3, 3) on a box of the lattice (whole lattice by default)."""
    shape = tuple(L) if shape is None else tuple(shape)
    sites = si.box_sites(L, origin, shape).reshape(-1)
    U = si.links(seed, eps, sites).reshape(field_shape(shape) + (4, 3, 3))
    return np.ascontiguousarray(np.moveaxis(U, 4, 0))


def tv_field(seed, ntv, L, origin=(0, 0, 0, 0), shape=None):
    shape = tuple(L) if shape is None else tuple(shape)
    sites = si.box_sites(L, origin, shape).reshape(-1)
    return si.test_vectors(seed, ntv, sites).reshape(field_shape(shape) + (4, 3, ntv))


def rhs_field(seed, nrhs, L, origin=(0, 0, 0, 0), shape=None):
    shape = tuple(L) if shape is None else tuple(shape)
    sites = si.box_sites(L, origin, shape).reshape(-1)
    return si.fine_rhs(seed, nrhs, sites).reshape(field_shape(shape) + (4, 3, nrhs))


def identity_links(L):
    U = np.zeros((4,) + field_shape(L) + (3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


# ---------------------------------------------------------------- layout conversions
def clover_to_lib(C):
    """Oracle clover (t,z,y,x,4,3,4,3) -> library layout [V][2][6][6]."""
    V = int(np.prod(C.shape[:4]))
    Cf = C.reshape(V, 4, 3, 4, 3)
    out = np.empty((V, 2, 6, 6), dtype=np.complex128)
    for h in range(2):
        out[:, h] = Cf[:, 2 * h:2 * h + 2, :, 2 * h:2 * h + 2, :].reshape(V, 6, 6)
    return out


def q_to_lib_R(Q):
    """Oracle Q (Vc, 2, 6Vb, N) -> library R [Vc][2][N][6Vb] = conj(q_j) rows."""
    return np.conj(np.swapaxes(Q, -1, -2))


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def patch_box(seed, eps, L, B, ntv, X, m0=M0, csw=CSW):
    """Oracle Q of every block of the 3x3x3x3-block box around coarse site X, and the D_c row of X.

    Returns (Q (81, 2, 6Vb, N) in box-lexicographic block order, Dc row (9, 2N, 2N), box origin,
    box shape); the box's centre block is X and box block nbr_box[d] is X's neighbour in stencil
    direction d.  Every input is regenerated from the counter-based generator at the box's global
    sites, so this works for lattices far too large for the host.
    """
    from oracle import coarse, dirac, lattice as lat
    origin = [(X[mu] - 1) * B[mu] for mu in range(4)]
    shape = tuple(3 * B[mu] for mu in range(4))
    U = links_field(seed, eps, L, origin, shape)
    C = dirac.clover_field(U, csw)
    tv = tv_field(seed, ntv, L, origin, shape)
    Q = coarse.orthonormalize(tv, B)
    Dc = coarse.coarse_operator(U, C, m0, Q, shape, B, sites=[BOX_CENTRE])
    return Q, Dc[0], origin, shape


def patch_neighbourhood(seed, eps, L, B, ntv, X):
    """(Q of block X and of its 8 neighbours (9, 2, 6Vb, N) in stencil order, D_c row of X (9, 2N, 2N));
    a module-level function so that a process pool can run it."""
    Q, Dc, _, _ = patch_box(seed, eps, L, B, ntv, X)
    return Q[BOX_NBR], Dc


def patch_reference(seed, eps, L, B, ntv, X, m0=M0, csw=CSW):
    """Oracle R rows and D_c row of coarse site X (patch_box's centre block).

    Returns (Q of the block (2, 6Vb, N), Dc row (9, 2N, 2N), box origin, box shape).
    """
    Q, Dc, origin, shape = patch_box(seed, eps, L, B, ntv, X, m0, csw)
    return Q[BOX_CENTRE], Dc, origin, shape


def _box_neighbours():
    from oracle import lattice as lat
    centre = int(lat.coarse_index(np.array([1, 1, 1, 1]), (3, 3, 3, 3)))
    return centre, lat.coarse_neighbours((3, 3, 3, 3))[centre]


BOX_CENTRE, BOX_NBR = _box_neighbours()


def block_sites(L, B, X):
    """Global site indices of block X in the library's aggregate order (site in block, x fastest)."""
    bt, bz, by, bx = np.meshgrid(*(np.arange(B[m]) for m in (3, 2, 1, 0)), indexing="ij")
    c = np.stack([X[0] * B[0] + bx, X[1] * B[1] + by, X[2] * B[2] + bz, X[3] * B[3] + bt], axis=-1)
    return si.site_index(L, c.reshape(-1, 4))


def coarse_coords(Lc, i):
    """Coordinates (x, y, z, t) of coarse site i (lexicographic, x fastest)."""
    c = []
    for mu in range(4):
        c.append(i % Lc[mu])
        i //= Lc[mu]
    return tuple(int(v) for v in c)


def to_aggregates_block(yb):
    """One block's fine values (Vb, 4, 3[, k]) -> its two aggregates (2, 6 Vb[, k]), dof order
    (site in block, spin within the chirality, colour)."""
    k = yb.shape[3:]
    a = yb.reshape((-1, 2, 2, 3) + k)
    return np.moveaxis(a, 1, 0).reshape((2, -1) + k)


def from_aggregates_block(xa):
    """Inverse of to_aggregates_block: (2, 6 Vb[, k]) -> (Vb, 4, 3[, k])."""
    k = xa.shape[2:]
    a = xa.reshape((2, -1, 2, 3) + k)
    return np.moveaxis(a, 0, 1).reshape((-1, 4, 3) + k)


def worst_ratio(got, ref, absref, c, floor=0.0):
    """max over elements of |got - ref| / (c |absref| + floor): <= 1 when every element is inside
    its own bound."""
    den = c * np.abs(absref) + floor
    return float(np.max(np.abs(np.asarray(got) - np.asarray(ref)) / den))


U_BF16 = 2.0 ** -8
U_FP16 = 2.0 ** -11
U_FP32 = 2.0 ** -24


def bf16_round(z):
    """Complex array -> the nearest BF16 Re/Im values (torch's round-to-nearest-even), complex128."""
    import torch
    f = torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], -1)).astype(np.float32))
    b = f.to(torch.bfloat16).to(torch.float64).numpy()
    return b[..., 0] + 1j * b[..., 1]
