"""Oracle sketch generator: Philox4x32-10 and Box-Muller, in numpy.

TEST INFRASTRUCTURE: see the package header.  Nothing in the product path
imports this file.

The paper draws the sketch G from the standard normal distribution with
i.i.d. entries (§3.1, construction of V-hat, step 1) and leaves the generator
unspecified.  Both sides of this project implement the same counter-based
generator from its published definition, so that the oracle and the GPU draw
the same G without passing it around:

* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC 2011): a round maps the counter
  (c0, c1, c2, c3) with key (k0, k1) to
  (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
  M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the
  Weyl constants (0x9E3779B9, 0xBB67AE85).
* key = (low 32 bits of the seed, high 32 bits of the seed).
* The sketch of step i is an rm x bi column-major matrix; element l = r + c*rm
  belongs to pair p = l >> 1, drawn from counter (p, i, matrix_id, stream).
* Two uniforms per counter, 53 bits each:
  j1 = (x0 >> 5) * 2^26 + (x1 >> 6),  u1 = (j1 + 1) * 2^-53  in (0, 1]
  j2 = (x2 >> 5) * 2^26 + (x3 >> 6),  u2 = j2 * 2^-53        in [0, 1)
* Box-Muller (Box & Muller 1958): rho = sqrt(-2 ln u1),
  G[2p] = rho cos(2 pi u2), G[2p+1] = rho sin(2 pi u2).

The batched form of the library (many small FP32 factorizations in one
launch) draws its sketch from the same words with 24-bit uniforms,
u1 = ((x0 >> 8) + 1) 2^-24 in (0, 1] and u2 = (x2 >> 8) 2^-24 in [0, 1)
(x1 and x3 unused), counter (p, step, matrix index, 0), and FP32 normals.
``box_muller_f32`` is that transform: the exact Box-Muller value of the two
FP32 uniforms, evaluated in FP64 and rounded once to FP32.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_SKETCH = 0


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` (shape (..., 4), uint32 values) under ``key``.

    Returns the four output words per counter, shape (..., 4), dtype uint32.
    """
    c = np.asarray(ctr, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.uint64(key[0]) & MASK32
    k1 = np.uint64(key[1]) & MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0          # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed: int) -> tuple[int, int]:
    s = int(seed) & 0xFFFF_FFFF_FFFF_FFFF
    return (s & 0xFFFFFFFF, s >> 32)


def uniforms(words: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(u1, u2) from Philox words (..., 4): u1 in (0,1], u2 in [0,1), 53 bits each."""
    w = words.astype(np.uint64)
    j1 = (w[..., 0] >> np.uint64(5)) * np.uint64(1 << 26) + (w[..., 1] >> np.uint64(6))
    j2 = (w[..., 2] >> np.uint64(5)) * np.uint64(1 << 26) + (w[..., 3] >> np.uint64(6))
    u1 = (j1 + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = j2.astype(np.float64) * 2.0 ** -53
    return u1, u2


def box_muller(words: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """The pair of normals (even element, odd element) of each word quadruple (..., 4)."""
    u1, u2 = uniforms(words)
    rho = np.sqrt(-2.0 * np.log(u1))
    return rho * np.cos(2.0 * np.pi * u2), rho * np.sin(2.0 * np.pi * u2)


def uniforms_f32(words: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(u1, u2) of the batched form: 24 bits each from x0 and x2, exact in FP32."""
    w = words.astype(np.uint64)
    u1 = ((w[..., 0] >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24
    u2 = (w[..., 2] >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    return u1, u2


def box_muller_f32(words: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """The batched form's FP32 pair of normals: Box-Muller of the 24-bit uniforms in FP64,
    rounded once to FP32."""
    u1, u2 = uniforms_f32(words)
    rho = np.sqrt(-2.0 * np.log(u1))
    return ((rho * np.cos(2.0 * np.pi * u2)).astype(np.float32),
            (rho * np.sin(2.0 * np.pi * u2)).astype(np.float32))


def _words(seed: int, step: int, matrix_id: int, stream: int, npairs: int) -> np.ndarray:
    p = np.arange(npairs, dtype=np.uint64)
    ctr = np.empty((npairs, 4), dtype=np.uint64)
    ctr[:, 0] = p & MASK32
    ctr[:, 1] = np.uint64(step) & MASK32
    ctr[:, 2] = np.uint64(matrix_id) & MASK32
    ctr[:, 3] = np.uint64(stream) & MASK32
    return philox4x32_10(ctr, seed_key(seed))


def normal_pairs(seed: int, step: int, matrix_id: int, stream: int,
                 npairs: int) -> np.ndarray:
    """Standard normals 2p, 2p+1 for pairs p = 0 .. npairs-1, as a flat array."""
    even, odd = box_muller(_words(seed, step, matrix_id, stream, npairs))
    out = np.empty(2 * npairs, dtype=np.float64)
    out[0::2] = even
    out[1::2] = odd
    return out


def normal_pairs_f32(seed: int, step: int, matrix_id: int, stream: int,
                     npairs: int) -> np.ndarray:
    """The batched form's FP32 normals 2p, 2p+1 for p = 0 .. npairs-1, as a flat array."""
    even, odd = box_muller_f32(_words(seed, step, matrix_id, stream, npairs))
    out = np.empty(2 * npairs, dtype=np.float32)
    out[0::2] = even
    out[1::2] = odd
    return out


def sketch(seed: int, step: int, rows: int, cols: int, matrix_id: int = 0,
           stream: int = STREAM_SKETCH) -> np.ndarray:
    """The rows x cols Gaussian sketch of one step, column-major element order."""
    count = rows * cols
    flat = normal_pairs(seed, step, matrix_id, stream, (count + 1) // 2)[:count]
    return flat.reshape(cols, rows).T.copy()


def sketch_f32(seed: int, step: int, rows: int, cols: int, matrix_id: int = 0,
               stream: int = STREAM_SKETCH) -> np.ndarray:
    """The batched form's FP32 sketch of one step (same element order as ``sketch``)."""
    count = rows * cols
    flat = normal_pairs_f32(seed, step, matrix_id, stream, (count + 1) // 2)[:count]
    return flat.reshape(cols, rows).T.copy()
