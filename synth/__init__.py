"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 4).

This module is shared by the CPU oracle, the tests and the benchmark. It holds
no arithmetic of the method itself: it only draws random nonnegative factors,
forms the observed matrix X = G0 F0 + noise, scales the noise to a requested
signal-to-noise ratio, and draws the initial factors and Gaussian sketches.

Every stream is derived from one integer seed through numpy's SeedSequence with
a fixed spawn key per purpose, so two calls with the same arguments return the
same bytes on any machine (numpy's PCG64 is platform independent).

Recipe (Sec. 4: nonnegative G, F drawn at random, X low-rank, noise such that
the SNR is about 30 dB):
  * G0 (n x p) and F0 (p x m) are iid Uniform[0, 1]; optionally a fraction of
    G0's entries is set to zero (sparse sources);
  * noise N = c |Z| with Z iid N(0, 1); c is chosen so that
    20 log10(||G0 F0||_F / ||N||_F) equals the requested SNR;
  * initial factors G, F are iid Uniform[0, 1] from a separate stream.
"""

from __future__ import annotations

import numpy as np

# Rows generated per block when X is assembled; a constant so that the random
# stream, and hence X, never depends on how the caller sizes its buffers.
_BLOCK_ROWS = 1024

_TAG_G0 = 1
_TAG_G0_ZERO = 2
_TAG_F0 = 3
_TAG_NOISE = 4
_TAG_INIT_G = 5
_TAG_INIT_F = 6
_TAG_OMEGA_L = 7
_TAG_OMEGA_R = 8
_TAG_SHAPES = 9
_TAG_DIRECTIONS = 10


def rng(seed: int, tag: int) -> np.random.Generator:
    """Independent PCG64 stream number `tag` of `seed`."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(int(seed), spawn_key=(int(tag),))))


def source_factors(n: int, m: int, p: int, seed: int, zero_frac: float = 0.0):
    """Ground-truth G0 (n x p) and F0 (p x m), iid Uniform[0,1], float64."""
    G0 = rng(seed, _TAG_G0).random((n, p))
    if zero_frac > 0.0:
        G0[rng(seed, _TAG_G0_ZERO).random((n, p)) < zero_frac] = 0.0
    F0 = rng(seed, _TAG_F0).random((p, m))
    return G0, F0


def lowrank_data(n: int, m: int, p: int, seed: int, snr_db: float | None = None,
                 zero_frac: float = 0.0, dtype=np.float64):
    """Observed X = G0 F0 (+ c|Z| at `snr_db`), returned with G0 and F0.

    X is assembled block by block in `dtype` so that a 1e4 x 1e4 float32 matrix
    never needs a float64 copy of the whole noise.
    """
    G0, F0 = source_factors(n, m, p, seed, zero_frac)
    X = np.empty((n, m), dtype=dtype)
    if snr_db is None:
        for r0 in range(0, n, _BLOCK_ROWS):
            X[r0:r0 + _BLOCK_ROWS] = G0[r0:r0 + _BLOCK_ROWS] @ F0
        return X, G0, F0
    # ||G0 F0||_F^2 = trace((G0^T G0)(F0 F0^T)) without forming G0 F0.
    signal_sq = float(np.sum((G0.T @ G0) * (F0 @ F0.T)))
    zr = rng(seed, _TAG_NOISE)
    noise_sq = 0.0
    for r0 in range(0, n, _BLOCK_ROWS):
        rows = min(_BLOCK_ROWS, n - r0)
        z = np.abs(zr.standard_normal((rows, m)))
        noise_sq += float(np.einsum("ij,ij->", z, z))
        X[r0:r0 + rows] = z
    c = np.sqrt(signal_sq / noise_sq) * 10.0 ** (-snr_db / 20.0)
    for r0 in range(0, n, _BLOCK_ROWS):
        blk = X[r0:r0 + _BLOCK_ROWS]
        blk[...] = G0[r0:r0 + _BLOCK_ROWS] @ F0 + c * blk.astype(np.float64)
    return X, G0, F0


def lowrank_data_device(n: int, m: int, p: int, seed: int, snr_db: float | None = None,
                        zero_frac: float = 0.0, device: str = "cuda"):
    """Device-resident float32 X with the recipe of lowrank_data, for batches too large to draw on the host.

    G0 and F0 are the host streams of source_factors (identical to
    lowrank_data's); the noise Z is drawn by torch's generator on `device`,
    seeded from (seed, noise tag), so X is reproducible but its noise is not
    lowrank_data's bytes. c is set from the float64 norms so that the SNR is
    exact. Returns (X, G0, F0) with X a torch tensor.
    """
    import torch
    G0, F0 = source_factors(n, m, p, seed, zero_frac)
    Gd = torch.from_numpy(G0).to(device)
    Fd = torch.from_numpy(F0).to(device)
    X = Gd @ Fd
    if snr_db is not None:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(rng(seed, _TAG_NOISE).integers(0, 2**63 - 1)))
        Z = torch.randn((n, m), generator=gen, device=device, dtype=torch.float32).abs_()
        signal_sq = float(np.sum((G0.T @ G0) * (F0 @ F0.T)))
        noise_sq = float(torch.sum(Z.double() ** 2))
        c = np.sqrt(signal_sq / noise_sq) * 10.0 ** (-snr_db / 20.0)
        X += c * Z.double()
        del Z
    return X.float().contiguous(), G0, F0


def initial_factors(n: int, m: int, p: int, seed: int):
    """Initial G (n x p) and F (p x m), iid Uniform[0,1], float64."""
    return rng(seed, _TAG_INIT_G).random((n, p)), rng(seed, _TAG_INIT_F).random((p, m))


def gaussian_sketches(n: int, m: int, nu: int, seed: int):
    """Host-drawn Gaussian Omega_L (m x nu) and Omega_R (nu x n), float64."""
    return (rng(seed, _TAG_OMEGA_L).standard_normal((m, nu)),
            rng(seed, _TAG_OMEGA_R).standard_normal((nu, n)))


def batched_shapes(count: int, seed: int, n_range=(1000, 8000), m_range=(500, 4000),
                   p_range=(4, 16), extra_sketch: int = 10):
    """Uneven instance shapes: n, m uniform integers, p uniform in p_range, nu = p + extra."""
    r = rng(seed, _TAG_SHAPES)
    n = r.integers(n_range[0], n_range[1] + 1, size=count)
    m = r.integers(m_range[0], m_range[1] + 1, size=count)
    p = r.integers(p_range[0], p_range[1] + 1, size=count)
    return [dict(n=int(a), m=int(b), p=int(c), nu=int(c) + extra_sketch) for a, b, c in zip(n, m, p)]


def random_directions(shape, count: int, seed: int):
    """`count` iid standard normal arrays of `shape` (finite-difference directions)."""
    r = rng(seed, _TAG_DIRECTIONS)
    return [r.standard_normal(shape) for _ in range(count)]
