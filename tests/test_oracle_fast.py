"""Pins for the word-packed oracle (oracle/oracle_fast.c).

It restates the sub-block assembly and the Toeplitz sum (Sec. III.B steps 1
and 3; Sec. I, K = T . A') on 64-bit words.  Each check here compares it with
something other than itself:

* the bit-loop oracle (oracle.c, already pinned to ATen's Philox, numpy's
  argsort and numpy's convolve) on every whole-method case of the oracle's
  own pins, and on windows of rows and sub-blocks;
* an explicitly built T times A over GF(2), and numpy's convolve;
* closed forms: a unit-vector sub-block reads one seed window, an all-ones
  seed gives the parity of the sub-block in every row;
* rank selection against numpy's stable argsort.

Planted mistakes in a copy of oracle_fast.c (a window off by one bit, the
sub-block not reversed, a dropped last word, a wrong seed offset per
sub-block, the word-aligned case reading the wrong word, a funnel shift by
the wrong amount, a rank off by one) must each be caught.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAST_SRC = open(os.path.join(ROOT, "oracle", "oracle_fast.c")).read()


def _words(rng, nbits):
    w = rng.integers(0, 2**32, size=(nbits + 31) // 32, dtype=np.uint64).astype(np.uint32)
    if nbits % 32:
        w[-1] &= np.uint32((1 << (nbits % 32)) - 1)
    return w


CASES = [
    # n, m, s, k, flags (the whole-method cases of the bit loop's pins, and more)
    (256, 4, 64, 32, 0),
    (1000, 3, 300, 77, 0),            # s, k not multiples of 32 or 64; n > m*s
    (4096, 1, 4096, 1, 0),            # m = 1, k = 1
    (3000, 7, 400, 400, 0),           # k = s
    (2048, 8, 256, 100, oracle.SEED_PER_SUBBLOCK),
    (1500, 1, 1500, 700, oracle.IDENTITY_PERM),
    (4096, 16, 256, 64, oracle.KEY_BITS(4)),
    (65, 1, 33, 31, 0),
    (5000, 3, 1664, 129, oracle.SEED_PER_SUBBLOCK),   # seeds start at odd bit offsets
    (2 ** 14, 2, 8192, 2048, 0),      # s a multiple of 64: window words word-aligned every 64 rows
    (1, 1, 1, 1, 0),
]


@pytest.mark.parametrize("n,m,s,k,flags", CASES)
def test_fast_extract_matches_bit_loop(n, m, s, k, flags):
    rng = np.random.default_rng(n * 7 + m + s + k)
    in_w = _words(rng, n)
    seed = _words(rng, (s + k - 1) * (m if flags & oracle.SEED_PER_SUBBLOCK else 1))
    want = oracle.extract(n, m, s, k, in_w, seed, 5, flags, nthreads=3)
    got = oracle.fast_extract(n, m, s, k, in_w, seed, 5, flags, nthreads=4)
    assert np.array_equal(got, want)


def test_fast_extract_matches_bit_loop_iid():
    n, m, k = 6000, 5, 150
    keys = oracle.sampling_keys(n, 8)
    _, _, largest = oracle.iid_order(keys, m, n, with_order=False)
    s = largest + 3
    rng = np.random.default_rng(4)
    in_w = _words(rng, n)
    seed = _words(rng, s + k - 1)
    want = oracle.extract(n, m, s, k, in_w, seed, 8, oracle.SAMPLING_IID)
    assert np.array_equal(oracle.fast_extract(n, m, s, k, in_w, seed, 8, oracle.SAMPLING_IID), want)


def test_fast_window_matches_bit_loop_window():
    rng = np.random.default_rng(21)
    n, m, s, k = 9000, 9, 900, 331
    in_w = _words(rng, n)
    seed = _words(rng, m * (s + k - 1))
    for flags in (0, oracle.SEED_PER_SUBBLOCK):
        p = oracle.perm(n, 4, flags)
        js = np.array([7, 2, 3, 8])                      # any sub-blocks, any order
        pos = np.concatenate([p[j * s:(j + 1) * s] for j in js])
        for i0, ni in ((0, k), (17, 100), (k - 1, 1), (64, 65)):
            got = oracle.fast_window(in_w, pos, s, k, seed, flags, js, i0, ni, nthreads=3,
                                     seed_len_bits=(m if flags else 1) * (s + k - 1))
            for t, j in enumerate(js):
                want = oracle.extract_window(in_w, p[j * s:(j + 1) * s], s, k, seed, flags, j, 1, i0, ni)
                assert np.array_equal(got[t], want[0]), (flags, j, i0, ni)


@pytest.mark.parametrize("s,k", [(1, 1), (63, 2), (64, 64), (65, 1), (130, 77), (200, 200)])
def test_fast_window_matches_explicit_matrix(s, k):
    rng = np.random.default_rng(s * 1000 + k)
    seed = _words(rng, s + k - 1)
    sb = oracle.bits_of(seed, s + k - 1).astype(np.int64)
    T = sb[np.arange(k)[:, None] - np.arange(s)[None, :] + s - 1]   # T[i][c] = seed[i - c + s - 1]
    in_w = _words(rng, s)
    A = oracle.bits_of(in_w, s).astype(np.int64)
    got = oracle.fast_window(in_w, np.arange(s), s, k, seed, 0, [0], 0, k, seed_len_bits=s + k - 1)[0]
    assert np.array_equal(got, (T @ A) % 2)
    assert np.array_equal(got, (np.convolve(sb, A) % 2)[s - 1:s - 1 + k])


def test_fast_window_closed_forms():
    s, k = 300, 120
    rng = np.random.default_rng(3)
    seed = _words(rng, s + k - 1)
    sb = oracle.bits_of(seed, s + k - 1)
    for c in (0, 1, 63, 64, s - 1):  # A = e_c reads the seed window starting at s - 1 - c
        in_w = np.zeros((s + 31) // 32, dtype=np.uint32)
        in_w[c >> 5] = np.uint32(1 << (c & 31))
        got = oracle.fast_window(in_w, np.arange(s), s, k, seed, 0, [0], 0, k, seed_len_bits=s + k - 1)[0]
        assert np.array_equal(got, sb[s - 1 - c:s - 1 - c + k]), c
    ones = np.full((s + k - 1 + 31) // 32, 0xFFFFFFFF, dtype=np.uint32)  # all-ones seed: parity of A
    in_w = _words(rng, s)
    par = int(oracle.bits_of(in_w, s).sum()) & 1
    got = oracle.fast_window(in_w, np.arange(s), s, k, ones, 0, [0], 0, k, seed_len_bits=s + k - 1)[0]
    assert np.all(got == par)


def test_perm_ranges_matches_stable_argsort():
    for n, K, flags in ((70000, 2, 0), (50000, 9, oracle.KEY_BITS(6))):
        keys = oracle.sampling_keys(n, K, flags)
        full = np.argsort(keys, kind="stable").astype(np.uint32)
        ranges = [(0, 1), (0, 1000), (12345, 6000), (n - 7, 7), (30000, 0), (100, 40000)]
        got = oracle.perm_ranges(keys, ranges)
        want = np.concatenate([full[lo:lo + c] for lo, c in ranges])
        assert np.array_equal(got, want)


# --------------------------------------------------------------------------
# planted mistakes
# --------------------------------------------------------------------------
MUTANTS = {
    "window off by one bit": ("const uint64_t t0 = off + i, q", "const uint64_t t0 = off + i + 1, q"),
    "sub-block not reversed": ("const uint64_t cr = s - 1 - c;", "const uint64_t cr = c;"),
    "last word dropped": ("for (uint64_t w = 0; w < nwords; ++w)\n            acc ^= ((S",
                          "for (uint64_t w = 0; w + 1 < nwords; ++w)\n            acc ^= ((S"),
    "per-sub-block seed offset": ("f->seed_len = s + k - 1;", "f->seed_len = s + k;"),
    "aligned window reads the next word": ("acc ^= S[q + w] & R[w];", "acc ^= S[q + w + 1] & R[w];"),
    "funnel shift by the wrong amount": ("(S[q + w + 1] << (64u - b))", "(S[q + w + 1] << (63u - b))"),
    "rank off by one": ("out[o++] = c[base[lo_b] + (rank - start[lo_b])].idx;",
                        "out[o++] = c[base[lo_b] + (rank + 1 - start[lo_b])].idx;"),
}


def _compile_fast(fast_src):
    d = tempfile.mkdtemp()
    for name, text in (("oracle_fast.c", fast_src),
                       ("oracle.c", open(os.path.join(ROOT, "oracle", "oracle.c")).read()),
                       ("oracle.h", open(os.path.join(ROOT, "oracle", "oracle.h")).read())):
        with open(os.path.join(d, name), "w") as f:
            f.write(text)
    so = os.path.join(d, "liboracle_fast_mutant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", so,
                    os.path.join(d, "oracle.c"), os.path.join(d, "oracle_fast.c"), "-lm"], check=True)
    return oracle.load_library(so)


def _fast_pins():
    failed = []
    for (n, m, s, k, flags) in CASES:
        rng = np.random.default_rng(n * 7 + m + s + k)
        in_w = _words(rng, n)
        seed = _words(rng, (s + k - 1) * (m if flags & oracle.SEED_PER_SUBBLOCK else 1))
        if not np.array_equal(oracle.fast_extract(n, m, s, k, in_w, seed, 5, flags, nthreads=2),
                              oracle.extract(n, m, s, k, in_w, seed, 5, flags, nthreads=2)):
            failed.append("whole method %r" % ((n, m, s, k, flags),))
    keys = oracle.sampling_keys(20000, 3)
    full = np.argsort(keys, kind="stable").astype(np.uint32)
    if not np.array_equal(oracle.perm_ranges(keys, [(100, 500), (9000, 77)]),
                          np.concatenate([full[100:600], full[9000:9077]])):
        failed.append("ranks")
    return failed


def test_unchanged_fast_oracle_passes_every_pin(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _compile_fast(FAST_SRC))
    assert _fast_pins() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_in_fast_oracle_is_caught(monkeypatch, name):
    old, new = MUTANTS[name]
    assert FAST_SRC.count(old) == 1, "mutation site not found: %s" % name
    monkeypatch.setattr(oracle, "_lib", _compile_fast(FAST_SRC.replace(old, new)))
    assert _fast_pins(), "no pin caught: %s" % name
