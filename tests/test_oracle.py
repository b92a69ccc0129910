"""Pins for the CPU oracle, each against something other than the oracle itself.

* Philox4x32-10 and the sampling labels: ATen's open-source ``philox_engine``
  (an independent implementation of the same published generator).
* The sampled order: ``numpy.argsort(kind="stable")`` on the labels.
* The Toeplitz product K = T . A (Sec. I): an explicitly built T times A over
  GF(2) with numpy, the polynomial middle product via ``numpy.convolve``,
  closed forms for unit vectors, all-ones seeds and zero inputs, and
  bilinearity.
* The whole method (Sec. III.B steps 1, 3, 4): a numpy composition of those
  library routines.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

pytestmark = []

ATEN_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::philox_engine e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


@pytest.fixture(scope="session")
def aten_philox():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    if not os.path.exists(hdr):
        pytest.skip("ATen PhiloxRNGEngine.h not present")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "p.cpp")
    exe = os.path.join(d, "p")
    with open(src, "w") as f:
        f.write(ATEN_SRC)
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, src, "-o", exe], check=True)

    def run(triples):
        inp = "".join("%d %d %d\n" % t for t in triples)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return np.array([[int(v) for v in line.split()] for line in out.strip().splitlines()],
                        dtype=np.uint64)
    return run


def _bits(words, n):
    return oracle.bits_of(words, n)


def _rand_words(rng, nbits):
    w = rng.integers(0, 2**32, size=(nbits + 31) // 32, dtype=np.uint64).astype(np.uint32)
    if nbits % 32:
        w[-1] &= np.uint32((1 << (nbits % 32)) - 1)
    return w


def _pack(bits):
    bits = np.asarray(bits, dtype=np.uint8)
    pad = (-bits.shape[0]) % 32
    b = np.concatenate([bits, np.zeros(pad, dtype=np.uint8)])
    return np.packbits(b, bitorder="little").view("<u4").copy()


# --------------------------------------------------------------------------
# Philox and the sampling labels
# --------------------------------------------------------------------------

def test_philox_matches_aten(aten_philox):
    rng = np.random.default_rng(11)
    triples = [(0, 0, 0), (2**64 - 1, 2**64 - 1, 2**64 - 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    for _ in range(3000):
        triples.append(tuple(int(x) for x in rng.integers(0, 2**63, size=3, dtype=np.uint64) * 2
                             + rng.integers(0, 2, size=3)))
    ref = aten_philox(triples)
    for (seed, sub, off), r in zip(triples, ref):
        # ATen: key = seed, counter = (offset_lo, offset_hi, subseq_lo, subseq_hi)
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = oracle.philox4x32_10(ctr, key)
        assert list(got) == [int(x) for x in r], (seed, sub, off)


def test_sampling_labels_match_aten(aten_philox):
    K = 2
    idx = list(range(0, 300)) + [2**32 - 1, 2**31 + 12345, 2**32 - 2]
    ref = aten_philox([(K, 0, i) for i in idx])
    keys = oracle.sampling_keys(300, K)
    for t, i in enumerate(idx):
        want = (int(ref[t][0]) << 32) | int(ref[t][1])
        assert oracle.sampling_key(i, K) == want
        if i < 300:
            assert int(keys[i]) == want
    # a 64-bit sampling key uses both key words
    K2 = 0x123456789ABCDEF1
    ref2 = aten_philox([(K2, 0, 7)])
    assert oracle.sampling_key(7, K2) == (int(ref2[0][0]) << 32) | int(ref2[0][1])


def test_key_bits_hook_keeps_top_bits():
    full = oracle.sampling_keys(1000, 5)
    for b in (1, 4, 17, 63):
        masked = oracle.sampling_keys(1000, 5, oracle.KEY_BITS(b))
        want = full & np.uint64(((1 << b) - 1) << (64 - b))
        assert np.array_equal(masked, want)


# --------------------------------------------------------------------------
# Sampled order
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,K", [(1, 3), (2, 3), (1000, 2), (65536, 2), (100003, 99)])
def test_perm_is_stable_argsort(n, K):
    keys = oracle.sampling_keys(n, K)
    p = oracle.perm(n, K)
    assert np.array_equal(p, np.argsort(keys, kind="stable").astype(np.uint32))
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint32))  # bijection


@pytest.mark.parametrize("n,b", [(4096, 4), (4096, 1), (50000, 8)])
def test_perm_forced_ties_lower_index_first(n, b):
    flags = oracle.KEY_BITS(b)
    keys = oracle.sampling_keys(n, 2, flags)
    assert len(np.unique(keys)) <= 2**b
    p = oracle.perm(n, 2, flags)
    assert np.array_equal(p, np.argsort(keys, kind="stable").astype(np.uint32))
    ks = keys[p]
    assert np.all(ks[1:] >= ks[:-1])
    tie = ks[1:] == ks[:-1]
    assert tie.sum() > 0
    assert np.all(p[1:][tie] > p[:-1][tie])


def test_perm_range_matches_full_perm():
    rng = np.random.default_rng(5)
    for n, flags in [(200000, 0), (70000, oracle.KEY_BITS(6)), (5000, 0)]:
        keys = oracle.sampling_keys(n, 7, flags)
        p = oracle.perm_from_keys(keys)
        cases = [(0, n), (0, 1), (n - 1, 1), (n // 2, n // 3)]
        for _ in range(10):
            lo = int(rng.integers(0, n))
            cases.append((lo, int(rng.integers(0, n - lo + 1))))
        for lo, cnt in cases:
            assert np.array_equal(oracle.perm_range(keys, lo, cnt), p[lo:lo + cnt]), (n, lo, cnt)


def test_identity_flag():
    assert np.array_equal(oracle.perm(77, 2, oracle.IDENTITY_PERM), np.arange(77, dtype=np.uint32))


# --------------------------------------------------------------------------
# Toeplitz product
# --------------------------------------------------------------------------

def _explicit_T(seed_bits, s, k):
    i = np.arange(k)[:, None]
    c = np.arange(s)[None, :]
    return seed_bits[i - c + s - 1]  # T[i][c] = seed[i - c + s - 1]


@pytest.mark.parametrize("s,k", [(1, 1), (5, 3), (32, 32), (33, 1), (100, 77), (257, 256), (300, 123)])
def test_toeplitz_matches_explicit_matrix(s, k):
    rng = np.random.default_rng(s * 1000 + k)
    seed = _rand_words(rng, s + k - 1)
    sb = _bits(seed, s + k - 1)
    T = _explicit_T(sb, s, k)
    # T is diagonal-constant
    if s > 1 and k > 1:
        assert np.array_equal(T[1:, 1:], T[:-1, :-1])
    for _ in range(3):
        A = rng.integers(0, 2, size=s).astype(np.uint8)
        K = oracle.toeplitz(seed, s, A, 0, k)
        want = (T.astype(np.int64) @ A.astype(np.int64)) % 2
        assert np.array_equal(K, want.astype(np.uint8))


@pytest.mark.parametrize("s,k", [(1024, 512), (4096, 1000), (2**15, 2**13)])
def test_toeplitz_is_polynomial_middle_product(s, k):
    rng = np.random.default_rng(s + k)
    seed = _rand_words(rng, s + k - 1)
    sb = _bits(seed, s + k - 1).astype(np.int64)
    A = rng.integers(0, 2, size=s).astype(np.uint8)
    rows = np.arange(k) if k <= 1024 else np.sort(rng.choice(k, 600, replace=False))
    conv = np.convolve(sb, A.astype(np.int64)) % 2  # coefficients of sigma(x) * a(x)
    for i in rows:
        assert oracle.toeplitz_bit(seed, s, A, int(i)) == conv[i + s - 1]


def test_toeplitz_special_cases():
    rng = np.random.default_rng(3)
    s, k = 200, 90
    seed = _rand_words(rng, s + k - 1)
    sb = _bits(seed, s + k - 1)
    # A = e_c picks a seed window: K = seed[s-1-c : s-1-c+k]
    for c in (0, 1, 57, s - 1):
        A = np.zeros(s, dtype=np.uint8)
        A[c] = 1
        assert np.array_equal(oracle.toeplitz(seed, s, A, 0, k), sb[s - 1 - c:s - 1 - c + k])
    A = rng.integers(0, 2, size=s).astype(np.uint8)
    # seed = e_t: K[i] = A[i + s - 1 - t] where that index exists, else 0
    for t in (0, 5, s - 1, s + k - 2):
        e = np.zeros(s + k - 1, dtype=np.uint8)
        e[t] = 1
        K = oracle.toeplitz(_pack(e), s, A, 0, k)
        want = np.array([A[i + s - 1 - t] if 0 <= i + s - 1 - t < s else 0 for i in range(k)],
                        dtype=np.uint8)
        assert np.array_equal(K, want)
    # A = 0 gives 0; all-ones seed gives parity(A) in every row
    assert not oracle.toeplitz(seed, s, np.zeros(s, dtype=np.uint8), 0, k).any()
    ones = _pack(np.ones(s + k - 1, dtype=np.uint8))
    assert np.all(oracle.toeplitz(ones, s, A, 0, k) == (A.sum() & 1))
    # k = 1: one row, the dot product of reversed seed[0..s) and A
    K1 = oracle.toeplitz(seed, s, A, 0, 1)
    assert K1[0] == (sb[:s][::-1].astype(int) @ A.astype(int)) % 2


def test_toeplitz_bilinear():
    rng = np.random.default_rng(4)
    s, k = 333, 111
    sa, sb_ = _rand_words(rng, s + k - 1), _rand_words(rng, s + k - 1)
    A = rng.integers(0, 2, size=s).astype(np.uint8)
    B = rng.integers(0, 2, size=s).astype(np.uint8)
    h = lambda seed, x: oracle.toeplitz(seed, s, x, 0, k)
    assert np.array_equal(h(sa, A ^ B), h(sa, A) ^ h(sa, B))
    assert np.array_equal(h(sa ^ sb_, A), h(sa, A) ^ h(sb_, A))


def test_toeplitz_row_window_and_offset():
    rng = np.random.default_rng(8)
    s, k = 100, 40
    seed = _rand_words(rng, 3 * (s + k - 1))
    A = rng.integers(0, 2, size=s).astype(np.uint8)
    full = oracle.toeplitz(seed, s, A, 0, k)
    assert np.array_equal(oracle.toeplitz(seed, s, A, 13, 20), full[13:33])
    off = s + k - 1
    sb = _bits(seed, 3 * off)
    shifted = _pack(sb[off:])
    assert np.array_equal(oracle.toeplitz(seed, s, A, 0, k, off=off),
                          oracle.toeplitz(shifted, s, A, 0, k))


# --------------------------------------------------------------------------
# The whole method against a numpy composition of library routines
# --------------------------------------------------------------------------

def _numpy_method(n, m, s, k, in_words, seed_words, K, flags):
    in_bits = _bits(in_words, n)
    if flags & oracle.IDENTITY_PERM:
        perm = np.arange(n)
    else:
        perm = np.argsort(oracle.sampling_keys(n, K, flags), kind="stable")
    blocks = in_bits[perm[:m * s]].reshape(m, s).astype(np.int64)
    L = s + k - 1
    sb = _bits(seed_words, L * (m if flags & oracle.SEED_PER_SUBBLOCK else 1)).astype(np.int64)
    out = []
    for j in range(m):
        sj = sb[j * L:(j + 1) * L] if flags & oracle.SEED_PER_SUBBLOCK else sb
        out.append(np.convolve(sj, blocks[j])[s - 1:s - 1 + k] % 2)
    return _pack(np.concatenate(out))


CASES = [
    # n, m, s, k, flags
    (256, 4, 64, 32, 0),
    (1000, 3, 300, 77, 0),           # s, k not multiples of 32; n > m*s
    (4096, 1, 4096, 1, 0),           # m = 1, k = 1
    (3000, 7, 400, 400, 0),          # k = s
    (2048, 8, 256, 100, oracle.SEED_PER_SUBBLOCK),
    (1500, 1, 1500, 700, oracle.IDENTITY_PERM),  # direct whole-block
    (4096, 16, 256, 64, oracle.KEY_BITS(4)),     # heavy ties
    (65, 1, 33, 31, 0),
]


@pytest.mark.parametrize("n,m,s,k,flags", CASES)
def test_extract_matches_numpy_composition(n, m, s, k, flags):
    rng = np.random.default_rng(n + m + s + k)
    in_words = _rand_words(rng, n)
    L = (s + k - 1) * (m if flags & oracle.SEED_PER_SUBBLOCK else 1)
    seed = _rand_words(rng, L)
    got = oracle.extract(n, m, s, k, in_words, seed, 2, flags, nthreads=3)
    want = _numpy_method(n, m, s, k, in_words, seed, 2, flags)
    assert np.array_equal(got, want)
    # tail bits of the last word are zero
    if (m * k) % 32:
        assert int(got[-1]) >> ((m * k) % 32) == 0


def test_extract_window_matches_extract():
    rng = np.random.default_rng(21)
    n, m, s, k = 5000, 9, 500, 130
    in_words = _rand_words(rng, n)
    seed = _rand_words(rng, m * (s + k - 1))
    for flags in (0, oracle.SEED_PER_SUBBLOCK):
        full = _bits(oracle.extract(n, m, s, k, in_words, seed, 4, flags), m * k).reshape(m, k)
        p = oracle.perm(n, 4, flags)
        j0, nj, i0, ni = 2, 5, 17, 100
        win = oracle.extract_window(in_words, p[j0 * s:(j0 + nj) * s], s, k, seed, flags,
                                    j0, nj, i0, ni, nthreads=2)
        assert np.array_equal(win, full[j0:j0 + nj, i0:i0 + ni])


def test_extract_rejects_bad_shapes():
    w = np.zeros(10, dtype=np.uint32)
    for n, m, s, k in [(100, 2, 60, 10), (100, 1, 10, 11), (100, 0, 10, 1), (100, 1, 10, 0)]:
        with pytest.raises(ValueError):
            oracle.extract(n, m, s, k, w, w, 1)


def test_check_order_accepts_only_the_stable_argsort():
    n = 30000
    keys = oracle.sampling_keys(n, 9, oracle.KEY_BITS(10))
    p = oracle.perm_from_keys(keys)
    assert oracle.check_order(keys, p, nthreads=4) == -1
    q = p.copy()
    q[[100, 101]] = q[[101, 100]]           # swap two neighbours
    assert oracle.check_order(keys, q) in (99, 100, 101)
    q = p.copy()
    q[5000] = q[4000]                       # a duplicate, so not a bijection
    assert oracle.check_order(keys, q) >= 0
    q = p.copy()
    q[7] = n                                # out of range
    assert oracle.check_order(keys, q) >= 0
