"""Seeded synthetic lattice inputs (host side, numpy, complex128).

Every value is addressed by a global index, so the inputs of any set of sites
can be regenerated without generating the whole lattice.

Site index: lexicographic on the fine lattice L = (Lx, Ly, Lz, Lt), x fastest.
Streams of the counter generator in ``synth.rng``:

* 0   -- gauge links: real normal ``(s*4 + mu)*8 + a`` is the coefficient h_a
         of the Gell-Mann matrix lambda_{a+1} in H_mu(s);
* 1   -- test vectors: complex Gaussian ``n*64 + j`` is component n of test
         vector j, with n = s*12 + spin*3 + colour (so test vector j does not
         depend on how many test vectors are drawn);
* 2+r -- fine right-hand side r: complex Gaussian n (same n);
* 1000+r -- coarse vector r: complex Gaussian ``i*128 + h*64 + j`` for coarse
         site i, chirality h and test-vector index j.

Links are U = exp(i eps H) with H = sum_a h_a lambda_a / 2 (traceless
Hermitian), evaluated here through the eigen-decomposition of H.
Seeds: 20151204 + workload number (the offset listed with each workload in
tests/helpers.py WORKLOADS).

This module holds none of the multigrid method's arithmetic.
"""
import numpy as np

from . import rng

SEED_BASE = 20151204
STREAM_LINKS = 0
STREAM_TV = 1
STREAM_RHS = 2
STREAM_COARSE = 1000
MAX_NTV = 64


def gell_mann():
    """The eight Gell-Mann matrices lambda_1..lambda_8 (3x3 complex)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


def volume(L):
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def all_sites(L):
    return np.arange(volume(L), dtype=np.int64)


def link_generators(seed, sites):
    """H_mu(s) = sum_a h_a lambda_a / 2 for the given sites: (n, 4, 3, 3)."""
    sites = np.asarray(sites, dtype=np.int64)
    k = (sites[:, None, None] * 4 + np.arange(4)[None, :, None]) * 8 + np.arange(8)[None, None, :]
    h = rng.normal(seed, STREAM_LINKS, k)                       # (n, 4, 8)
    return 0.5 * np.einsum("nma,aij->nmij", h, gell_mann())


def links(seed, eps, sites):
    """SU(3) links U_mu(s) = exp(i eps H_mu(s)) for the given sites: (n, 4, 3, 3)."""
    H = link_generators(seed, sites)
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("nmik,nmk,nmjk->nmij", v, ph, v.conj())


def test_vectors(seed, ntv, sites):
    """Test vectors at the given sites, layout (n, 4, 3, ntv) complex128."""
    if ntv > MAX_NTV:
        raise ValueError("ntv > %d" % MAX_NTV)
    sites = np.asarray(sites, dtype=np.int64)
    n = sites[:, None] * 12 + np.arange(12)[None, :]
    m = n[:, :, None] * MAX_NTV + np.arange(ntv)[None, None, :]
    return rng.complex_gaussian(seed, STREAM_TV, m).reshape(len(sites), 4, 3, ntv)


def fine_rhs(seed, nrhs, sites):
    """Fine right-hand sides at the given sites, layout (n, 4, 3, nrhs)."""
    sites = np.asarray(sites, dtype=np.int64)
    n = (sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
    out = np.empty((len(sites) * 12, nrhs), dtype=np.complex128)
    for r in range(nrhs):
        out[:, r] = rng.complex_gaussian(seed, STREAM_RHS + r, n)
    return out.reshape(len(sites), 4, 3, nrhs)


def coarse_vector(seed, ntv, nrhs, coarse_sites):
    """Coarse vectors at the given coarse sites, layout (n, 2, ntv, nrhs)."""
    cs = np.asarray(coarse_sites, dtype=np.int64)
    idx = (cs[:, None, None] * 128 + np.arange(2)[None, :, None] * 64
           + np.arange(ntv)[None, None, :])
    out = np.empty((len(cs), 2, ntv, nrhs), dtype=np.complex128)
    for r in range(nrhs):
        out[..., r] = rng.complex_gaussian(seed, STREAM_COARSE + r, idx)
    return out


def site_index(L, coords):
    """Lexicographic index (x fastest) of integer coordinates (..., 4)."""
    c = np.asarray(coords, dtype=np.int64)
    return ((c[..., 3] * L[2] + c[..., 2]) * L[1] + c[..., 1]) * L[0] + c[..., 0]


def box_sites(L, origin, shape):
    """Global site indices of a box of the periodic lattice.

    Returns an int64 array of shape (shape[3], shape[2], shape[1], shape[0]),
    i.e. the same (t, z, y, x) axis order as the field arrays of the oracle.
    """
    ax = [(origin[mu] + np.arange(shape[mu])) % L[mu] for mu in range(4)]
    t, z, y, x = np.meshgrid(ax[3], ax[2], ax[1], ax[0], indexing="ij")
    return site_index(L, np.stack([x, y, z, t], axis=-1))
