"""Pins for the oracle's counter-based Gaussian sketch generator.

* Philox4x32-10 against its published known-answer vectors (tests/golden);
* the uniform mapping's end points and the Box-Muller radius identity
  z1^2 + z2^2 = -2 ln u1;
* the output distribution against N(0, 1) (Kolmogorov-Smirnov).
"""

import os

import numpy as np
import scipy.stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(np.array([v[0:4]], dtype=np.uint64), (v[4], v[5]))[0]
        assert [int(x) for x in out] == v[6:10]


def test_uniform_end_points():
    u = philox.uniforms_from_words(np.array([0, 0xFFFFFFFF, 0x1FF, 0x200]))
    np.testing.assert_array_equal(u, [0.5 / 2**23, (2**23 - 0.5) / 2**23, 0.5 / 2**23, 1.5 / 2**23])
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_box_muller_radius_identity():
    seed = 12345
    z = philox.gaussian_matrix(1, 8, seed, 3).reshape(-1)
    words = philox.philox4x32_10(np.array([[0, 0, 3, 0], [1, 0, 3, 0]], dtype=np.uint64),
                                 (seed & 0xFFFFFFFF, seed >> 32))
    u = philox.uniforms_from_words(words)
    for g in range(2):
        np.testing.assert_allclose(z[4 * g] ** 2 + z[4 * g + 1] ** 2, -2 * np.log(u[g, 0]), rtol=1e-13)
        np.testing.assert_allclose(z[4 * g + 2] ** 2 + z[4 * g + 3] ** 2, -2 * np.log(u[g, 2]), rtol=1e-13)


def test_gaussian_distribution_and_streams():
    a = philox.gaussian_matrix(300, 333, 99, philox.STREAM_OMEGA_L).reshape(-1)
    b = philox.gaussian_matrix(300, 333, 99, philox.STREAM_OMEGA_R).reshape(-1)
    assert scipy.stats.kstest(a, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02
    # a ragged total (not a multiple of 4) is a prefix of the longer draw
    c = philox.gaussian_matrix(1, 7, 99, 0).reshape(-1)
    d = philox.gaussian_matrix(1, 8, 99, 0).reshape(-1)
    np.testing.assert_array_equal(c, d[:7])
