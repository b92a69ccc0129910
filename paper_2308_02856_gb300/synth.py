"""Seeded synthetic inputs for sampled sub-block hashing.

This module holds no arithmetic of the hashing method: it only draws the
weakly random input block and the uniform Toeplitz seed, which both the CUDA
path and the CPU oracle then receive as plain arrays.  Randomness comes from
numpy's Philox bit generator (Philox4x64-10); its raw 64-bit stream is split
into two little-endian 32-bit words, so a (seed, length) pair always yields the
same bits.

The paper measures on unpublished "simulated datasets" (Sec. IV.C); the
stand-ins here are i.i.d. Bernoulli(p) bits, the shape of a biased QRNG/QKD
raw key, with p from 0.55 to 0.9.
"""
from __future__ import annotations

import numpy as np

_CHUNK_BITS = 1 << 24  # 64 MiB of uint32 draws per chunk


def _raw_u32(rng: np.random.Generator, count: int) -> np.ndarray:
    """``count`` uniform uint32 words from the bit generator's raw stream."""
    raw = rng.bit_generator.random_raw((count + 1) // 2)
    return np.ascontiguousarray(raw.astype("<u8")).view("<u4")[:count]


def uniform_bits(nbits: int, seed: int) -> np.ndarray:
    """``ceil(nbits/32)`` uint32 words of uniform bits, LSB-first; bits past
    ``nbits`` are zero."""
    words = (nbits + 31) // 32
    rng = np.random.Generator(np.random.Philox(seed))
    out = _raw_u32(rng, words).copy()
    if nbits % 32:
        out[-1] &= np.uint32((1 << (nbits % 32)) - 1)
    return out


def bernoulli_bits(nbits: int, p: float, seed: int) -> np.ndarray:
    """i.i.d. Bernoulli(p) bits packed LSB-first into uint32 words.

    Bit i is 1 when the i-th uint32 draw is below floor(p * 2^32)."""
    thr = int(np.floor(p * 4294967296.0))
    words = (nbits + 31) // 32
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.empty(words, dtype="<u4")
    done = 0
    while done < nbits:
        cnt = min(_CHUNK_BITS, nbits - done)
        u = _raw_u32(rng, cnt)
        b = (u < np.uint32(thr)) if thr < 4294967296 else np.ones(cnt, dtype=bool)
        packed = np.packbits(b, bitorder="little")
        nb = (cnt + 31) // 32 * 4
        buf = np.zeros(nb, dtype=np.uint8)
        buf[:packed.shape[0]] = packed
        w0 = done // 32
        out[w0:w0 + nb // 4] = buf.view("<u4")
        done += cnt
    return out
