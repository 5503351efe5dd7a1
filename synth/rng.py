"""Counter-based random numbers for the synthetic lattice inputs (host side).

The generator is defined so that any single value can be regenerated from
(seed, stream, counter) alone, which lets a test rebuild the inputs of one
block of a lattice far too large to generate on the host.

Definition (the device generator in ``synth/csrc/synth.cu`` implements the
same definition independently):

* ``mix64`` is the output function of SplitMix64 (Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014, with the
  multipliers of Vigna's reference ``splitmix64.c``)::

      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
      z = (z ^ (z >> 27)) * 0x94D049BB133111EB
      z =  z ^ (z >> 31)

* the stream key is ``base = mix64(mix64(seed) ^ (stream * 0xD1B54A32D192ED03))``;
* the counter-th 64-bit draw is ``mix64(base + (counter + 1) * 0x9E3779B97F4A7C15)``
  (SplitMix64's own state increment), all arithmetic modulo 2**64;
* a uniform in (0, 1] is ``((draw >> 11) + 1) * 2**-53``;
* normal number ``k`` is one half of the Box-Muller pair ``m = k >> 1`` built
  from uniforms ``u1 = U(2m)``, ``u2 = U(2m + 1)``:
  ``r = sqrt(-2 ln u1)``, even ``k`` -> ``r cos(2 pi u2)``, odd ``k`` ->
  ``r sin(2 pi u2)``;
* complex Gaussian ``m`` is ``normal(2m) + i normal(2m + 1)``, so its real and
  imaginary parts are each N(0, 1).

This module holds no arithmetic of the multigrid method itself.
"""
import numpy as np

_U64 = np.uint64
GOLDEN = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)
_STREAM_MUL = _U64(0xD1B54A32D192ED03)


def mix64(z):
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
    return z ^ (z >> _U64(31))


def stream_base(seed, stream):
    """Key of one stream: mix64(mix64(seed) ^ stream * 0xD1B54A32D192ED03)."""
    s = mix64(np.array([seed], dtype=np.uint64))
    with np.errstate(over="ignore"):
        t = np.array([stream], dtype=np.uint64) * _STREAM_MUL
    return mix64(s ^ t)[0]


def draw_u64(seed, stream, counter):
    """The counter-th 64-bit draw of a stream (counter: int array)."""
    c = np.asarray(counter, dtype=np.uint64)
    base = stream_base(seed, stream)
    with np.errstate(over="ignore"):
        z = base + (c + _U64(1)) * GOLDEN
    return mix64(z)


def uniform(seed, stream, counter):
    """Uniform doubles in (0, 1] from the top 53 bits of each draw."""
    d = draw_u64(seed, stream, counter)
    return ((d >> _U64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed, stream, k):
    """Standard normal number k of a stream (Box-Muller, see module doc)."""
    k = np.asarray(k, dtype=np.int64)
    m = k >> 1
    u1 = uniform(seed, stream, 2 * m)
    u2 = uniform(seed, stream, 2 * m + 1)
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return np.where((k & 1) == 0, r * np.cos(ang), r * np.sin(ang))


def complex_gaussian(seed, stream, m):
    """Complex Gaussian m of a stream: normal(2m) + i normal(2m+1)."""
    m = np.asarray(m, dtype=np.int64)
    u1 = uniform(seed, stream, 2 * m)
    u2 = uniform(seed, stream, 2 * m + 1)
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return r * np.cos(ang) + 1j * (r * np.sin(ang))
