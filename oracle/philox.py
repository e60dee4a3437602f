"""Counter-based Gaussian sketch: Philox4x32-10 and Box-Muller, in numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Alg. 2 draws Gaussian Omega_L and Omega_R. Both the CUDA library and this
oracle derive them from one counter-based generator so that a seed fixes the
sketch on either side. Written from the published definitions:

  Philox4x32 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: as
  easy as 1, 2, 3"): state (c0, c1, c2, c3), key (k0, k1); one round is
      (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2     (64-bit products)
      c' = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
  with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl
  constants (0x9E3779B9, 0xBB67AE85) before every round but the first;
  10 rounds.

  Box-Muller (1958): u1, u2 in (0, 1) ->
      z1 = sqrt(-2 ln u1) cos(2 pi u2),  z2 = sqrt(-2 ln u1) sin(2 pi u2).

Sketch layout (the library's definition, restated in its header):
  element e of a row-major matrix belongs to group g = e // 4; group g is the
  Philox block at counter (g mod 2^32, g >> 32, stream, 0) and key
  (seed mod 2^32, seed >> 32); its words x0..x3 give
  u_j = ((x_j >> 9) + 0.5) / 2^23 (24 significant bits, exact in float32) and
      z[4g]   = sqrt(-2 ln u0) cos(2 pi u1),  z[4g+1] = sqrt(-2 ln u0) sin(2 pi u1),
      z[4g+2] = sqrt(-2 ln u2) cos(2 pi u3),  z[4g+3] = sqrt(-2 ln u2) sin(2 pi u3).
  Omega_L (m x nu) uses stream 0, Omega_R (nu x n) stream 1.
"""

from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

STREAM_OMEGA_L = 0
STREAM_OMEGA_R = 1


def _mulhilo(a: int, b: np.ndarray):
    prod = np.uint64(a) * b.astype(np.uint64)
    return (prod >> np.uint64(32)).astype(np.uint64), (prod & np.uint64(MASK32)).astype(np.uint64)


def philox4x32_10(counter: np.ndarray, key) -> np.ndarray:
    """Philox4x32 with 10 rounds. counter: (N, 4) integers < 2^32; key: (k0, k1)."""
    c = np.asarray(counter, dtype=np.uint64).reshape(-1, 4).copy()
    k0 = np.uint64(int(key[0]) & MASK32)
    k1 = np.uint64(int(key[1]) & MASK32)
    for r in range(10):
        if r > 0:
            k0 = np.uint64((int(k0) + W0) & MASK32)
            k1 = np.uint64((int(k1) + W1) & MASK32)
        hi0, lo0 = _mulhilo(M0, c[:, 0])
        hi1, lo1 = _mulhilo(M1, c[:, 2])
        c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
    return c.astype(np.uint32)


def uniforms_from_words(x: np.ndarray) -> np.ndarray:
    """u = ((x >> 9) + 0.5) / 2^23 in (0, 1), exactly representable in float32 and float64."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) / 8388608.0


def gaussian_matrix(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """rows x cols standard normal matrix from the counter layout above (float64)."""
    total = rows * cols
    groups = (total + 3) // 4
    g = np.arange(groups, dtype=np.uint64)
    ctr = np.stack([g & np.uint64(MASK32), g >> np.uint64(32),
                    np.full(groups, stream, dtype=np.uint64), np.zeros(groups, dtype=np.uint64)], axis=1)
    words = philox4x32_10(ctr, (seed & MASK32, (seed >> 32) & MASK32))
    u = uniforms_from_words(words)
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.stack([r01 * np.cos(2.0 * np.pi * u[:, 1]), r01 * np.sin(2.0 * np.pi * u[:, 1]),
                  r23 * np.cos(2.0 * np.pi * u[:, 3]), r23 * np.sin(2.0 * np.pi * u[:, 3])], axis=1)
    return z.reshape(-1)[:total].reshape(rows, cols)


def sketches(n: int, m: int, nu: int, seed: int):
    """(Omega_L m x nu, Omega_R nu x n) drawn as the library draws them from `seed`."""
    return (gaussian_matrix(m, nu, seed, STREAM_OMEGA_L), gaussian_matrix(nu, n, seed, STREAM_OMEGA_R))
