"""CPU oracle for sampled sub-block Toeplitz hashing (arXiv 2308.02856).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path (the CUDA library
and its binding) never imports this package.

The arithmetic lives in ``oracle.c`` (plain C, one bit at a time) and
``oracle_fast.c`` (the same Toeplitz sum on 64-bit words: AND, XOR and one
popcount parity per output bit, pinned to the bit loop); this module compiles
them with gcc and marshals numpy arrays through ctypes.  Definitions
(Sec. III.B steps 1, 3 and 4 of the paper, Sec. I for K = T . A'):

* sampling label of position i: ``(x0 << 32) | x1`` of Philox4x32-10 with
  counter ``(i_lo, i_hi, 0, 0)`` and key ``(K_lo, K_hi)``; the sampled order is
  the stable argsort of the labels; sub-block j = sorted ranks [j*s, (j+1)*s);
* ``K_j[i] = XOR_c seed_j[i - c + s - 1] AND A_j[c]`` for i < k;
* output bit ``j*k + i = K_j[i]``, LSB-first in uint32 words, tail bits 0.

With ``SAMPLING_IID`` the paper's own law replaces the sorted order: position
i joins sub-block ``V_i = floor(label_i * m / 2^64)``; sub-block j is the input
at ``{i : V_i = j}`` in increasing position order, zero-padded to s (the block
size limit L_S^UB of Eq. 7), and the run aborts when a sub-block exceeds s.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_FAST = os.path.join(_HERE, "oracle_fast.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SEED_PER_SUBBLOCK = 0x1
IDENTITY_PERM = 0x2
SAMPLING_IID = 0x10
NO_POS = 0xFFFFFFFF


class Abort(Exception):
    """The i.i.d. law aborts: some sub-block is larger than the limit s."""


def KEY_BITS(b: int) -> int:
    """Test hook: keep only the top ``b`` bits (1..63) of each sampling label."""
    return (int(b) & 0x3F) << 8


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` and ``oracle_fast.c`` into ``liboracle.so``
    (plain -O2, not tuned)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_FAST),
                                              os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, _SRC_FAST, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def load_library(path: str) -> ctypes.CDLL:
    """Open a compiled oracle library and declare its C signatures."""
    L = ctypes.CDLL(path)
    u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
    L.oracle_philox4x32_10.argtypes = [vp, vp, vp]
    L.oracle_philox4x32_10.restype = None
    L.oracle_sampling_key.argtypes = [u64, u64, u32]
    L.oracle_sampling_key.restype = u64
    L.oracle_sampling_keys.argtypes = [u64, u64, u32, vp, i32]
    L.oracle_sampling_keys.restype = None
    L.oracle_perm.argtypes = [u64, vp, vp]
    L.oracle_perm.restype = i32
    L.oracle_perm_range.argtypes = [u64, vp, u64, u64, vp]
    L.oracle_perm_range.restype = i32
    L.oracle_check_order.argtypes = [u64, vp, vp, i32]
    L.oracle_check_order.restype = ctypes.c_int64
    L.oracle_subblock.argtypes = [vp, vp, u64, vp]
    L.oracle_subblock.restype = None
    L.oracle_toeplitz_bit.argtypes = [vp, u64, u64, vp, u64]
    L.oracle_toeplitz_bit.restype = ctypes.c_uint8
    L.oracle_toeplitz.argtypes = [vp, u64, u64, vp, u64, u64, vp]
    L.oracle_toeplitz.restype = None
    L.oracle_extract.argtypes = [u64, u64, u64, u64, vp, vp, u64, u32, vp, i32]
    L.oracle_extract.restype = i32
    L.oracle_extract_window.argtypes = [vp, vp, u64, u64, vp, u32, u64, u64, u64, u64, vp, i32]
    L.oracle_extract_window.restype = None
    L.oracle_subblock_padded.argtypes = [vp, vp, u64, vp]
    L.oracle_subblock_padded.restype = None
    L.oracle_iid_label.argtypes = [u64, u64]
    L.oracle_iid_label.restype = u32
    L.oracle_iid_order.argtypes = [u64, vp, u64, u64, vp, vp]
    L.oracle_iid_order.restype = u64
    L.oracle_size_tail_bound.argtypes = [u64, u64, ctypes.c_double]
    L.oracle_size_tail_bound.restype = ctypes.c_double
    L.oracle_block_limit.argtypes = [u64, u64, ctypes.c_double, ctypes.c_double]
    L.oracle_block_limit.restype = u64
    if hasattr(L, "oracle_fast_window"):
        L.oracle_fast_window.argtypes = [vp, vp, u64, u64, vp, u64, u32, vp, u64, u64, u64, vp, i32]
        L.oracle_fast_window.restype = i32
        L.oracle_perm_ranges.argtypes = [u64, vp, u64, vp, vp, vp]
        L.oracle_perm_ranges.restype = i32
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(_LIB)
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sampling_key(i: int, sampling_key_: int, flags: int = 0) -> int:
    return int(lib().oracle_sampling_key(i, sampling_key_, flags))


def sampling_keys(n: int, sampling_key_: int, flags: int = 0, nthreads=None) -> np.ndarray:
    keys = np.empty(max(n, 1), dtype=np.uint64)
    lib().oracle_sampling_keys(n, sampling_key_, flags, _ptr(keys), _threads(nthreads))
    return keys[:n]


def perm_from_keys(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.shape[0]
    perm = np.empty(max(n, 1), dtype=np.uint32)
    rc = lib().oracle_perm(n, _ptr(keys) if n else 0, _ptr(perm))
    if rc:
        raise RuntimeError("oracle_perm failed: %d" % rc)
    return perm[:n]


def perm(n: int, sampling_key_: int, flags: int = 0, nthreads=None) -> np.ndarray:
    if flags & IDENTITY_PERM:
        return np.arange(n, dtype=np.uint32)
    return perm_from_keys(sampling_keys(n, sampling_key_, flags, nthreads))


def perm_range(keys: np.ndarray, lo: int, cnt: int) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(max(cnt, 1), dtype=np.uint32)
    rc = lib().oracle_perm_range(keys.shape[0], _ptr(keys), lo, cnt, _ptr(out))
    if rc:
        raise RuntimeError("oracle_perm_range failed: %d" % rc)
    return out[:cnt]


def check_order(keys: np.ndarray, perm_: np.ndarray, nthreads=None) -> int:
    """-1 if ``perm_`` is the stable argsort of ``keys`` (checked as strict
    increase in (label, position) order with every entry < n), else the first
    offending rank."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    perm_ = np.ascontiguousarray(perm_, dtype=np.uint32)
    assert keys.shape[0] == perm_.shape[0]
    return int(lib().oracle_check_order(keys.shape[0], _ptr(keys), _ptr(perm_), _threads(nthreads)))


def subblock(in_bits: np.ndarray, pos: np.ndarray) -> np.ndarray:
    in_bits = np.ascontiguousarray(in_bits, dtype=np.uint32)
    pos = np.ascontiguousarray(pos, dtype=np.uint32)
    A = np.empty(max(pos.shape[0], 1), dtype=np.uint8)
    lib().oracle_subblock(_ptr(in_bits), _ptr(pos), pos.shape[0], _ptr(A))
    return A[:pos.shape[0]]


def toeplitz(seed_bits: np.ndarray, s: int, A: np.ndarray, i0: int, cnt: int, off: int = 0) -> np.ndarray:
    seed_bits = np.ascontiguousarray(seed_bits, dtype=np.uint32)
    A = np.ascontiguousarray(A, dtype=np.uint8)
    assert A.shape[0] == s
    K = np.empty(max(cnt, 1), dtype=np.uint8)
    lib().oracle_toeplitz(_ptr(seed_bits), off, s, _ptr(A), i0, cnt, _ptr(K))
    return K[:cnt]


def toeplitz_bit(seed_bits: np.ndarray, s: int, A: np.ndarray, i: int, off: int = 0) -> int:
    seed_bits = np.ascontiguousarray(seed_bits, dtype=np.uint32)
    A = np.ascontiguousarray(A, dtype=np.uint8)
    return int(lib().oracle_toeplitz_bit(_ptr(seed_bits), off, s, _ptr(A), i))


def extract(n, m, s, k, in_bits, seed_bits, sampling_key_, flags=0, nthreads=None) -> np.ndarray:
    in_bits = np.ascontiguousarray(in_bits, dtype=np.uint32)
    seed_bits = np.ascontiguousarray(seed_bits, dtype=np.uint32)
    out = np.zeros((m * k + 31) // 32, dtype=np.uint32)
    rc = lib().oracle_extract(n, m, s, k, _ptr(in_bits), _ptr(seed_bits), sampling_key_, flags,
                              _ptr(out), _threads(nthreads))
    if rc == -3:
        raise Abort("a sub-block exceeds the limit s = %d" % s)
    if rc:
        raise ValueError("oracle_extract rejected the arguments (%d)" % rc)
    return out


def iid_label(key: int, m: int) -> int:
    """Sub-block of a position with sampling label ``key`` under the i.i.d. law."""
    return int(lib().oracle_iid_label(key, m))


def iid_order(keys: np.ndarray, m: int, s: int, with_order: bool = True):
    """(sizes, order, largest): sizes[j] = |S_j|; order (m*s entries, NO_POS
    padding) is None when the largest sub-block exceeds s (the abort case) or
    when with_order is False (sizes only, nothing of size m*s allocated)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    sizes = np.zeros(m, dtype=np.uint64)
    order = np.empty(max(m * s, 1), dtype=np.uint32) if with_order else None
    largest = int(lib().oracle_iid_order(keys.shape[0], _ptr(keys) if keys.shape[0] else 0, m, s,
                                         _ptr(sizes), _ptr(order) if with_order else 0))
    if largest == 2**64 - 1:
        raise MemoryError("oracle_iid_order")
    return sizes, (order[:m * s] if with_order and largest <= s else None), largest


def subblock_padded(in_bits: np.ndarray, pos: np.ndarray) -> np.ndarray:
    in_bits = np.ascontiguousarray(in_bits, dtype=np.uint32)
    pos = np.ascontiguousarray(pos, dtype=np.uint32)
    A = np.empty(max(pos.shape[0], 1), dtype=np.uint8)
    lib().oracle_subblock_padded(_ptr(in_bits), _ptr(pos), pos.shape[0], _ptr(A))
    return A[:pos.shape[0]]


def size_tail_bound(N: int, L: int, p: float) -> float:
    """Eq. 7's bound on P(a binomial(N, p) sub-block size exceeds L)."""
    return float(lib().oracle_size_tail_bound(N, L, p))


def block_limit(N: int, m: int, eps: float, p: float) -> int:
    """Eq. 7: the smallest L with m * size_tail_bound(N, L, p) <= eps."""
    return int(lib().oracle_block_limit(N, m, eps, p))


def extract_window(in_bits, pos, s, k, seed_bits, flags, j0, nj, i0, ni, nthreads=None) -> np.ndarray:
    """K_j[i] for j in [j0, j0+nj), i in [i0, i0+ni), one byte per bit, given
    ``pos`` = the sampled positions of those sub-blocks (nj*s entries)."""
    in_bits = np.ascontiguousarray(in_bits, dtype=np.uint32)
    pos = np.ascontiguousarray(pos, dtype=np.uint32)
    seed_bits = np.ascontiguousarray(seed_bits, dtype=np.uint32)
    assert pos.shape[0] == nj * s
    out = np.empty(max(nj * ni, 1), dtype=np.uint8)
    lib().oracle_extract_window(_ptr(in_bits), _ptr(pos), s, k, _ptr(seed_bits), flags,
                                j0, nj, i0, ni, _ptr(out), _threads(nthreads))
    return out[:nj * ni].reshape(nj, ni)


def bits_of(words: np.ndarray, nbits: int) -> np.ndarray:
    """Unpack LSB-first uint32 words into one uint8 per bit (first nbits)."""
    w = np.ascontiguousarray(words, dtype="<u4")
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:nbits]


# ---- word-packed restatement (oracle_fast.c) --------------------------------

def fast_window(in_bits, pos, s, k, seed_bits, flags, js, i0, ni, nthreads=None,
                seed_len_bits=None) -> np.ndarray:
    """K_j[i] for the sub-blocks ``js`` and rows i in [i0, i0+ni), one byte
    per bit (shape (len(js), ni)), computed on 64-bit words; ``pos`` holds the
    sampled positions of those sub-blocks (len(js)*s entries, in js order)."""
    in_bits = np.ascontiguousarray(in_bits, dtype=np.uint32)
    pos = np.ascontiguousarray(pos, dtype=np.uint32)
    seed_bits = np.ascontiguousarray(seed_bits, dtype=np.uint32)
    js = np.ascontiguousarray(js, dtype=np.uint64)
    nj = js.shape[0]
    assert pos.shape[0] == nj * s
    nbits = int(seed_len_bits) if seed_len_bits is not None else 32 * seed_bits.shape[0]
    assert nbits <= 32 * seed_bits.shape[0]
    out = np.empty(max(nj * ni, 1), dtype=np.uint8)
    rc = lib().oracle_fast_window(_ptr(in_bits), _ptr(pos), s, k, _ptr(seed_bits), nbits, flags,
                                  _ptr(js) if nj else 0, nj, i0, ni, _ptr(out), _threads(nthreads))
    if rc:
        raise ValueError("oracle_fast_window failed (%d)" % rc)
    return out[:nj * ni].reshape(nj, ni)


def perm_ranges(keys: np.ndarray, ranges) -> np.ndarray:
    """Ranks [lo, lo+cnt) of the stable argsort of ``keys`` for each (lo, cnt)
    in ``ranges``, concatenated, in one pass over the keys."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    lo = np.ascontiguousarray([r[0] for r in ranges], dtype=np.uint64)
    cnt = np.ascontiguousarray([r[1] for r in ranges], dtype=np.uint64)
    total = int(cnt.sum()) if len(ranges) else 0
    out = np.empty(max(total, 1), dtype=np.uint32)
    rc = lib().oracle_perm_ranges(keys.shape[0], _ptr(keys), len(ranges), _ptr(lo) if len(ranges) else 0,
                                  _ptr(cnt) if len(ranges) else 0, _ptr(out))
    if rc:
        raise RuntimeError("oracle_perm_ranges failed: %d" % rc)
    return out[:total]


def fast_extract(n, m, s, k, in_bits, seed_bits, sampling_key_, flags=0, nthreads=None) -> np.ndarray:
    """The whole method with the word-packed Toeplitz sum: the oracle's own
    order (sorted, identity or i.i.d.), every sub-block's rows, output words
    packed LSB-first with tail bits 0 (the same result as ``extract``)."""
    if flags & SAMPLING_IID:
        _, order, largest = iid_order(sampling_keys(n, sampling_key_, flags, nthreads), m, s)
        if order is None:
            raise Abort("a sub-block exceeds the limit s = %d" % s)
        pos = order
    else:
        pos = perm(n, sampling_key_, flags, nthreads)[:m * s]
    nseed = (m if flags & SEED_PER_SUBBLOCK else 1) * (s + k - 1)
    K = fast_window(in_bits, pos, s, k, seed_bits, flags, np.arange(m), 0, k, nthreads, seed_len_bits=nseed)
    bits = K.reshape(-1)
    pad = (-bits.shape[0]) % 32
    if pad:
        bits = np.concatenate([bits, np.zeros(pad, dtype=np.uint8)])
    return np.packbits(bits, bitorder="little").view("<u4").astype(np.uint32)
