"""Wilson-clover Dirac operator D on the fine lattice (oracle, complex128).

The paper uses D through Alg. 7, where one hop of D contributes
(1 +- gamma_mu) U^(dagger) P(x + mu) and the clover term C^{hh}(x) is
chirality-diagonal; it does not print D.  Reading fixed here (standard form):

    D psi(x) = (4 + m0) psi(x) + C(x) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                            + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]

    C(x) = c_sw (i/4) sum_{mu != nu} sigma_{mu nu} F_{mu nu}(x),
    sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu],
    F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger) / 8,

with Q_{mu nu}(x) the sum of the four plaquettes in the (mu, nu) plane that
start and end at x, each traversed counter-clockwise, and periodic boundary
conditions in all four directions.  Gamma matrices are in the chiral basis,
gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]], so
gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).
"""
import numpy as np

from . import lattice as lat

_PAULI = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def gammas():
    """gamma_mu, mu = 0..3 (x, y, z, t), chiral basis, 4x4 complex."""
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = [np.block([[z, -1j * s], [1j * s, z]]) for s in _PAULI]
    g.append(np.block([[z, one], [one, z]]))
    return np.array(g)


def gamma5():
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def sigma(mu, nu):
    g = gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def _mm(a, b):
    return np.einsum("...ij,...jk->...ik", a, b)


def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def clover_leaves(U, mu, nu):
    """Q_{mu nu}(x): the four counter-clockwise plaquettes at x, summed.

    U has shape (4, t, z, y, x, 3, 3) with U[mu] the link from x to x + mu.
    """
    Um, Un = U[mu], U[nu]
    s = lat.shift
    q = _mm(_mm(Um, s(Un, mu, 1)), _mm(_dag(s(Um, nu, 1)), _dag(Un)))
    q = q + _mm(_mm(Un, _dag(s(s(Um, nu, 1), mu, -1))),
                _mm(_dag(s(Un, mu, -1)), s(Um, mu, -1)))
    q = q + _mm(_mm(_dag(s(Um, mu, -1)), _dag(s(s(Un, mu, -1), nu, -1))),
                _mm(s(s(Um, mu, -1), nu, -1), s(Un, nu, -1)))
    q = q + _mm(_mm(_dag(s(Un, nu, -1)), s(Um, nu, -1)),
                _mm(s(s(Un, nu, -1), mu, 1), _dag(Um)))
    return q


def clover_field(U, csw):
    """C(x) as a (t, z, y, x, 4, 3, 4, 3) array: c_sw (i/4) sum sigma F."""
    shape = U.shape[1:5]
    C = np.zeros(shape + (4, 3, 4, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            Q = clover_leaves(U, mu, nu)
            F = (Q - _dag(Q)) / 8.0
            C += np.einsum("ab,...ij->...aibj", sigma(mu, nu), F)
    return csw * 0.25j * C


def apply_site_term(C, m0, psi):
    """(4 + m0) psi(x) + C(x) psi(x)."""
    if psi.ndim == 6:
        cpsi = np.einsum("...aibj,...bj->...ai", C, psi)
    else:
        cpsi = np.einsum("...aibj,...bjk->...aik", C, psi)
    return (4.0 + m0) * psi + cpsi


def _colour(Ux, psi):
    # U acting on the colour index of psi (t,z,y,x,4,3[,k])
    if psi.ndim == 6:
        return np.einsum("...ij,...aj->...ai", Ux, psi)
    return np.einsum("...ij,...ajk->...aik", Ux, psi)


def _spin(G, psi):
    if psi.ndim == 6:
        return np.einsum("ab,...bi->...ai", G, psi)
    return np.einsum("ab,...bik->...aik", G, psi)


def hop_forward(U, psi, mu):
    """-1/2 (1 - gamma_mu) U_mu(x) psi(x + mu) at every x."""
    g = gammas()[mu]
    t = _colour(U[mu], lat.shift(psi, mu, 1))
    return -0.5 * (t - _spin(g, t))


def hop_backward(U, psi, mu):
    """-1/2 (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) at every x."""
    g = gammas()[mu]
    t = _colour(_dag(lat.shift(U[mu], mu, -1)), lat.shift(psi, mu, -1))
    return -0.5 * (t + _spin(g, t))


def apply_dirac(U, C, m0, psi):
    """D psi on the whole periodic lattice (psi: (t,z,y,x,4,3[,k]))."""
    out = apply_site_term(C, m0, psi)
    for mu in range(4):
        out = out + hop_forward(U, psi, mu) + hop_backward(U, psi, mu)
    return out


def _bcast(mask, psi):
    return mask.reshape(mask.shape + (1,) * (psi.ndim - 4))


def apply_block_part(U, C, m0, psi, B, d):
    """One stencil part H_d of D with respect to the block decomposition.

    H_0 holds the site term and every hop whose two ends lie in one block;
    H_{+mu} (d = 1 + 2 mu) holds the forward hops from a site on the +mu face
    of its block into the next block; H_{-mu} (d = 2 + 2 mu) the backward
    hops from a site on the -mu face.  D = H_0 + sum_mu (H_{+mu} + H_{-mu}),
    and the coupling of block i to its neighbour in direction d is
    D_{i, nbr(i,d)} restricted to H_d (Eq. cgo).
    """
    L = (psi.shape[3], psi.shape[2], psi.shape[1], psi.shape[0])
    x = lat.coords_fields(L)
    if d == 0:
        out = apply_site_term(C, m0, psi)
        for mu in range(4):
            inner_f = (x[mu] % B[mu]) != B[mu] - 1
            inner_b = (x[mu] % B[mu]) != 0
            out = out + _bcast(inner_f, psi) * hop_forward(U, psi, mu) \
                + _bcast(inner_b, psi) * hop_backward(U, psi, mu)
        return out
    mu = (d - 1) // 2
    if d % 2 == 1:
        face = (x[mu] % B[mu]) == B[mu] - 1
        return _bcast(face, psi) * hop_forward(U, psi, mu)
    face = (x[mu] % B[mu]) == 0
    return _bcast(face, psi) * hop_backward(U, psi, mu)


def dense_dirac(U, C, m0):
    """D as a dense (12V x 12V) matrix built entry by entry (tiny lattices).

    Row/column index s*12 + spin*3 + colour with s the lexicographic site
    index.  Written with explicit site loops, independently of apply_dirac.
    """
    Lt, Lz, Ly, Lx = U.shape[1:5]
    L = (Lx, Ly, Lz, Lt)
    V = Lx * Ly * Lz * Lt
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    for t in range(Lt):
        for z in range(Lz):
            for y in range(Ly):
                for xx in range(Lx):
                    c = [xx, y, z, t]
                    s = ((t * Lz + z) * Ly + y) * Lx + xx
                    D[12 * s:12 * s + 12, 12 * s:12 * s + 12] += \
                        (4.0 + m0) * np.eye(12) + C[t, z, y, xx].reshape(12, 12)
                    for mu in range(4):
                        cp = list(c)
                        cp[mu] = (cp[mu] + 1) % L[mu]
                        sp = ((cp[3] * Lz + cp[2]) * Ly + cp[1]) * Lx + cp[0]
                        Ul = U[mu, t, z, y, xx]
                        # row s, column s+mu: -1/2 (1 - gamma_mu) (x) U_mu(s)
                        D[12 * s:12 * s + 12, 12 * sp:12 * sp + 12] += \
                            -0.5 * np.kron(one - g[mu], Ul)
                        # row s+mu, column s: -1/2 (1 + gamma_mu) (x) U_mu(s)^dagger
                        D[12 * sp:12 * sp + 12, 12 * s:12 * s + 12] += \
                            -0.5 * np.kron(one + g[mu], Ul.conj().T)
    return D


def flatten_field(psi):
    """(t,z,y,x,4,3[,k]) -> (12V[,k]) with index s*12 + spin*3 + colour."""
    V = int(np.prod(psi.shape[:4]))
    return psi.reshape((12 * V,) + psi.shape[6:])


def gauge_transform(U, G):
    """U_mu(x) -> G(x) U_mu(x) G(x + mu)^dagger."""
    return np.stack([_mm(_mm(G, U[mu]), _dag(lat.shift(G, mu, 1))) for mu in range(4)])
