"""The seeded input generator shared by both sides: SplitMix64 against the known-answer
outputs of the published reference implementation (state 0), the uniform and Gaussian
transforms by their moments, and the bump parameters by their stated ranges."""
import math

import numpy as np

import inputs


def test_splitmix64_known_answers():
    g = inputs.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_uses_the_top_53_bits():
    g, h = inputs.SplitMix64(12345), inputs.SplitMix64(12345)
    for _ in range(100):
        u = g.uniform()
        assert 0.0 <= u < 1.0
        assert u == (h.next_u64() >> 11) / 2.0 ** 53


def test_gaussian_moments():
    """Box-Muller: mean 0, variance 1, fourth moment 3, within 5 standard errors (n = 40000)."""
    g = inputs.SplitMix64(7)
    x = np.array([g.gauss() for _ in range(40000)])
    n = len(x)
    assert abs(x.mean()) < 5 * math.sqrt(1 / n)
    assert abs(x.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs((x ** 4).mean() - 3) < 5 * math.sqrt(96 / n)


def test_bump_parameters():
    c, p = inputs.bump_batch(1, 16)
    assert c.shape == (16, 3, 3) and p.shape == (16, 3, 3)
    assert np.all((c >= 0.2) & (c < 0.8))
    assert np.allclose(np.linalg.norm(p, axis=2), 1.0, rtol=0, atol=1e-15)
    # one stream per (seed, right-hand side): batches are prefixes of each other, streams differ
    c2, p2 = inputs.bump_batch(1, 4)
    assert np.array_equal(c[:4], c2) and np.array_equal(p[:4], p2)
    assert len({tuple(ci.ravel()) for ci in c}) == 16
    c3, _ = inputs.bump_batch(2, 1)
    assert not np.array_equal(c3[0], c[0])
    assert inputs.stream_seed(1, 0) != inputs.stream_seed(0, 1)
