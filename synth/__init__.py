"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

``synth.inputs`` / ``synth.rng`` generate inputs on the host (numpy);
``synth.device`` generates the same values on a GPU from an independent CUDA
implementation of the same published generator (used where a lattice is too
large to generate on the host).  Nothing here computes any part of the
multigrid method.
"""
from . import rng, inputs  # noqa: F401
