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


def patch_reference(seed, eps, L, B, ntv, X, m0=M0, csw=CSW):
    """Oracle R rows and D_c row of coarse site X, from a 3x3x3x3-block box around it.

    Returns (Q of the block (2, 6Vb, N), Dc row (9, 2N, 2N), box origin, box shape).
    Every input is regenerated from the counter-based generator at the box's
    global sites, so this works for lattices far too large for the host.
    """
    from oracle import coarse, dirac, lattice as lat
    origin = [(X[mu] - 1) * B[mu] for mu in range(4)]
    shape = tuple(3 * B[mu] for mu in range(4))
    U = links_field(seed, eps, L, origin, shape)
    C = dirac.clover_field(U, csw)
    tv = tv_field(seed, ntv, L, origin, shape)
    Q = coarse.orthonormalize(tv, B)
    centre = int(lat.coarse_index(np.array([1, 1, 1, 1]), (3, 3, 3, 3)))
    Dc = coarse.coarse_operator(U, C, m0, Q, shape, B, sites=[centre])
    return Q[centre], Dc[0], origin, shape
