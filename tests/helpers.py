"""Shared test helpers: synthetic inputs in the oracle's array layout.

Workloads (input recipe): each has a fine lattice L (x, y, z,
t), block B, number of test vectors, link spread eps, mass m0 and c_sw.
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
