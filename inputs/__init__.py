"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws random numbers. It holds none of the method's
arithmetic: the load vector, the matrices and the solve are computed
separately by each side from these parameters.

Right-hand sides follow the source of Sec. 6.1 in spirit (a smooth, localised
vector field F), but as a sum of Gaussian bumps whose parameters are drawn
here:

    F(x) = sum_b p_b * exp(-|x - c_b|^2 / w^2)

with centres c_b uniform in [0.2, 0.8]^3, width w, and complex polarisations
p_b in C^3 (independent standard complex Gaussians, scaled to unit 2-norm).

Generator: SplitMix64 (Steele, Lea, Flood 2014), one stream per
(seed, rhs index); doubles from the top 53 bits; Gaussians by Box-Muller.
"""
import math

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 counter-based generator (published constants)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def gauss(self) -> float:
        """Standard normal by Box-Muller (one value per call)."""
        u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)


def stream_seed(seed: int, index: int) -> int:
    """Seed of the stream for right-hand side `index` of a run seeded `seed`."""
    return ((seed & 0xFFFFFFFF) << 32) | (index & 0xFFFFFFFF)


def bumps(seed: int, index: int, nbumps: int = 3, lo: float = 0.2, hi: float = 0.8):
    """Bump parameters of one right-hand side.

    Returns (centres [nbumps,3] float64, pol [nbumps,3] complex128).
    """
    g = SplitMix64(stream_seed(seed, index))
    centres = np.empty((nbumps, 3))
    pol = np.empty((nbumps, 3), dtype=np.complex128)
    for b in range(nbumps):
        for a in range(3):
            centres[b, a] = lo + (hi - lo) * g.uniform()
        v = np.array([complex(g.gauss(), g.gauss()) for _ in range(3)])
        pol[b] = v / np.linalg.norm(v)
    return centres, pol


def bump_batch(seed: int, nrhs: int, nbumps: int = 3, first_index: int = 0):
    """Parameters of `nrhs` right-hand sides (stream indices first_index..).

    Returns centres [nrhs, nbumps, 3], pol [nrhs, nbumps, 3] complex128.
    """
    cs, ps = [], []
    for r in range(nrhs):
        c, p = bumps(seed, first_index + r, nbumps)
        cs.append(c)
        ps.append(p)
    return np.stack(cs), np.stack(ps)


def random_complex(seed: int, shape, index: int = 0) -> np.ndarray:
    """Seeded complex vector with independent standard normal parts.

    Uses numpy's PCG64 (test vectors only, e.g. for operator parity)."""
    rng = np.random.default_rng([seed & 0xFFFFFFFF, index & 0xFFFFFFFF])
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
