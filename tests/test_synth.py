"""Pins of the counter-based input generator against its published definition."""
import os

import numpy as np

from synth import rng, inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    state = np.uint64(1234567)
    got = []
    for _ in vals:
        with np.errstate(over="ignore"):
            state = state + rng.GOLDEN
        got.append(int(rng.mix64(np.array([state], dtype=np.uint64))[0]))
    assert got == vals


def test_counter_addressing_and_distribution():
    # the counter-th draw is the counter-th output of SplitMix64 started at the stream key
    base = rng.stream_base(42, 3)
    s = base
    seq = []
    for _ in range(4):
        with np.errstate(over="ignore"):
            s = s + rng.GOLDEN
        seq.append(int(rng.mix64(np.array([s], dtype=np.uint64))[0]))
    assert [int(v) for v in rng.draw_u64(42, 3, np.arange(4))] == seq
    u = rng.uniform(1, 1, np.arange(200000))
    assert u.min() > 0 and u.max() <= 1
    z = rng.normal(1, 1, np.arange(400000))
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    c = rng.complex_gaussian(1, 1, np.arange(3))
    assert np.allclose(c.real, rng.normal(1, 1, 2 * np.arange(3)))
    assert np.allclose(c.imag, rng.normal(1, 1, 2 * np.arange(3) + 1))


def test_box_regeneration_matches_full_lattice():
    L = (4, 4, 2, 6)
    full = si.test_vectors(7, 5, si.all_sites(L)).reshape(L[3], L[2], L[1], L[0], 4, 3, 5)
    box = si.box_sites(L, (3, 1, 1, 4), (2, 4, 2, 3))
    part = si.test_vectors(7, 5, box.reshape(-1)).reshape(box.shape + (4, 3, 5))
    for t in range(3):
        for z in range(2):
            for y in range(4):
                for x in range(2):
                    g = ((3 + x) % 4, (1 + y) % 4, (1 + z) % 2, (4 + t) % 6)
                    assert np.array_equal(part[t, z, y, x], full[g[3], g[2], g[1], g[0]])
    # test vector j is the same whatever the number drawn
    a = si.test_vectors(7, 3, np.arange(5))
    b = si.test_vectors(7, 6, np.arange(5))
    assert np.array_equal(a, b[..., :3])
