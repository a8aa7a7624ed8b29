"""Pins of the oracle's Philox-4x32-10 stream: published known-answer vectors
(tests/golden/philox4x32_10_kat.txt) and the moments of the normal draws."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden",
                      "philox4x32_10_kat.txt")


def test_known_answer_vectors():
    n = 0
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        out = philox.philox4x32_10(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10]
        n += 1
    assert n == 3


def test_normal_stream_moments_and_determinism():
    z = philox.normal(64, 4099, seed=3, it=7)
    assert z.shape == (64, 4099)
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / z.size)
    assert np.array_equal(z, philox.normal(64, 4099, seed=3, it=7))
    z2 = philox.normal(64, 4099, seed=3, it=8)
    assert abs(np.corrcoef(z.ravel(), z2.ravel())[0, 1]) < 4 / np.sqrt(z.size)
    # columns c and c + 4k in one row come from different counters
    assert abs(np.corrcoef(z[:, 0], z[:, 4])[0, 1]) < 0.5
