"""Seeded synthetic inputs for sampled sub-block hashing.

This module holds no arithmetic of the hashing method: it only draws the
weakly random input block, the uniform Toeplitz seed and the shapes of the
batch and serving workloads, which the CUDA path and the CPU oracle then
receive as plain arrays.

Randomness comes from numpy's Philox bit generator (Philox4x64-10).  Its raw
64-bit stream is split into two little-endian 32-bit draws, so draw t is half
(t & 1) of raw value t >> 1.  Long streams are filled in parallel chunks, each
positioned with ``advance`` (one step skips 4 raw values), so the bits do not
depend on the chunking.

The paper measures on unpublished "simulated datasets" (Sec. IV.C); the
stand-ins here are i.i.d. Bernoulli(p) bits, the shape of a biased QRNG/QKD
raw key, with p from 0.55 to 0.95.
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os

import numpy as np

_CHUNK_DRAWS = 1 << 24  # 32-bit draws per chunk (a multiple of 8)


def _draws(seed: int, start: int, count: int) -> np.ndarray:
    """32-bit draws [start, start + count) of the stream of ``seed``
    (start a multiple of 8)."""
    bg = np.random.Philox(seed)
    if start:
        bg.advance(start // 8)  # start/2 raw values, 4 per advance step
    raw = bg.random_raw((count + 1) // 2)
    return np.ascontiguousarray(raw.astype("<u8")).view("<u4")[:count]


def _parallel_chunks(nbits: int, fn) -> None:
    starts = list(range(0, nbits, _CHUNK_DRAWS))
    workers = min(len(starts), os.cpu_count() or 1, 32)
    if workers <= 1:
        for s in starts:
            fn(s, min(_CHUNK_DRAWS, nbits - s))
        return
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(lambda s: fn(s, min(_CHUNK_DRAWS, nbits - s)), starts))


def uniform_bits(nbits: int, seed: int) -> np.ndarray:
    """``ceil(nbits/32)`` uint32 words of uniform bits, LSB-first; bits past
    ``nbits`` are zero.  Word t is draw t of the stream."""
    words = (nbits + 31) // 32
    out = np.empty(max(words, 1), dtype="<u4")[:words]

    def fill(start, cnt):
        out[start:start + cnt] = _draws(seed, start, cnt)
    _parallel_chunks(words, fill)
    if nbits % 32:
        out[-1] &= np.uint32((1 << (nbits % 32)) - 1)
    return out


def bernoulli_bits(nbits: int, p: float, seed: int) -> np.ndarray:
    """i.i.d. Bernoulli(p) bits packed LSB-first into uint32 words: bit i is
    1 when draw i of the stream is below floor(p * 2^32)."""
    thr = int(np.floor(p * 4294967296.0))
    words = (nbits + 31) // 32
    out = np.zeros(max(words, 1), dtype="<u4")[:words]
    ob = out.view(np.uint8)

    def fill(start, cnt):
        u = _draws(seed, start, cnt)
        b = (u < np.uint32(thr)) if thr < 4294967296 else np.ones(cnt, dtype=bool)
        packed = np.packbits(b, bitorder="little")
        ob[start // 8:start // 8 + packed.shape[0]] = packed
    _parallel_chunks(nbits, fill)
    return out


# --------------------------------------------------------------------------
# workload shapes for batching and serving
# --------------------------------------------------------------------------
S_SET = (1 << 16, 1 << 18, 1 << 20)


def job_shapes(count: int, seed: int, n_lo: int, n_hi: int, s_set=S_SET, ratio=(0.05, 0.5),
               p=(0.55, 0.95)) -> list:
    """``count`` job shapes: n log-uniform in [n_lo, n_hi], s drawn from s_set
    and clamped to the largest member <= n, n rounded down to a multiple of
    s (m = n / s), k = max(1, floor(ratio * s)) with ratio uniform, Bernoulli
    p uniform; each job also gets its own input seed, Toeplitz seed and
    sampling key."""
    rng = np.random.Generator(np.random.Philox(seed))
    jobs = []
    lo, hi = math.log2(n_lo), math.log2(n_hi)
    for i in range(count):
        u = rng.random(4)
        n = int(2.0 ** (lo + (hi - lo) * u[0]))
        s = s_set[min(len(s_set) - 1, int(u[1] * len(s_set)))]
        fits = [x for x in s_set if x <= n]
        s = min(s, max(fits)) if fits else n
        n = (n // s) * s
        k = max(1, int((ratio[0] + (ratio[1] - ratio[0]) * u[2]) * s))
        jobs.append({"n": n, "m": n // s, "s": s, "k": k, "p": float(p[0] + (p[1] - p[0]) * u[3]),
                     "in_seed": seed * 100000 + 3 * i + 1, "seed_seed": seed * 100000 + 3 * i + 2,
                     "key": seed * 100000 + 3 * i + 3})
    return jobs


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of ``rate`` jobs/s: gaps
    -ln(1 - u) / rate."""
    rng = np.random.Generator(np.random.Philox(seed))
    u = rng.random(count)
    return np.cumsum(-np.log1p(-u) / rate)


def bernoulli_bits_device(nbits: int, p: float, seed: int, device="cuda"):
    """i.i.d. Bernoulli(p) bits drawn on the GPU with torch's seeded
    generator, packed LSB-first into an int32 tensor of ceil(nbits/32) words
    (bits past nbits zero).  For large benchmark inputs that no CPU check
    reads; CPU-checked inputs come from bernoulli_bits."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    words = (nbits + 31) // 32
    out = torch.empty(words, dtype=torch.int32, device=device)
    shifts = torch.arange(32, device=device, dtype=torch.int64)
    chunk = 1 << 21  # words per chunk
    for w0 in range(0, words, chunk):
        cw = min(chunk, words - w0)
        b = (torch.rand((cw, 32), generator=g, device=device) < p).to(torch.int64)
        lo = w0 * 32
        if lo + cw * 32 > nbits:  # clear bits past nbits
            idx = torch.arange(cw * 32, device=device).view(cw, 32) + lo
            b = b * (idx < nbits).to(torch.int64)
        v = (b << shifts).sum(1)
        out[w0:w0 + cw] = torch.where(v >= 2 ** 31, v - 2 ** 32, v).to(torch.int32)  # same 32 bits
    return out
