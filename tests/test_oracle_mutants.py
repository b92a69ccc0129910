"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a temporary copy of oracle/oracle.c (a wrong Toeplitz index, a
dropped term, an off-by-one, swapped Philox output words, a wrong round
count or constant, a reversed tie-break, mis-packed output bits), compiles
it, and checks that at least one pin of tests/test_oracle.py's kind fails on
it while the unchanged oracle passes them all."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "oracle", "oracle.c")).read()

MUTANTS = {
    "toeplitz index transposed": ("bit(seed, off + i - c + s - 1)", "bit(seed, off + c - i + s - 1)"),
    "toeplitz index off by one": ("bit(seed, off + i - c + s - 1)", "bit(seed, off + i - c + s)"),
    "dropped last term": ("for (uint64_t c = 0; c < s; ++c) {\n        uint8_t t_ic", "for (uint64_t c = 1; c < s; ++c) {\n        uint8_t t_ic"),
    "AND replaced by OR": ("acc ^= (uint8_t)(t_ic & A[c]);", "acc ^= (uint8_t)(t_ic | A[c]);"),
    "philox output words swapped": ("((uint64_t)x[0] << 32) | (uint64_t)x[1]", "((uint64_t)x[1] << 32) | (uint64_t)x[0]"),
    "philox nine rounds": ("round < 10", "round < 9"),
    "philox weyl constant": ("#define PHILOX_W1 0xBB67AE85u", "#define PHILOX_W1 0xBB67AE84u"),
    "tie-break reversed": ("if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;", "if (x->idx != y->idx) return x->idx < y->idx ? 1 : -1;"),
    "sub-block taken from the wrong rank": ("A[c] = bit(in, pos[c]);", "A[c] = bit(in, pos[s - 1 - c]);"),
    "output packed at the wrong bit": ("out[t >> 5] |= (uint32_t)K[t] << (t & 31u);", "out[t >> 5] |= (uint32_t)K[t] << (31u - (t & 31u));"),
    "iid label from the low bits": ("return (uint32_t)(((unsigned __int128)key * m) >> 64);", "return (uint32_t)(key % m);"),
    "iid positions in decreasing order": ("for (uint64_t i = 0; i < n; ++i) {  /* increasing positions */",
                                          "for (uint64_t i = n; i-- > 0;) {  /* increasing positions */"),
    "iid padding not zero": ("A[c] = pos[c] == ORACLE_NO_POS ? 0 : bit(in, pos[c]);", "A[c] = bit(in, pos[c] % 64u);"),
    "eq7 without the factor 2": ("double z = sqrt(2.0 * (double)N * ", "double z = sqrt((double)N * "),
    "eq7 relative entropy sign": ("double b = x < 1.0 ? (1.0 - x) * log((1.0 - x) / (1.0 - p)) : 0.0;",
                                  "double b = x < 1.0 ? (1.0 - x) * log((1.0 - p) / (1.0 - x)) : 0.0;"),
}


def _compile(src):
    d = tempfile.mkdtemp()
    c = os.path.join(d, "oracle.c")
    with open(c, "w") as f:
        f.write(src)
    with open(os.path.join(d, "oracle.h"), "w") as f:
        f.write(open(os.path.join(ROOT, "oracle", "oracle.h")).read())
    so = os.path.join(d, "liboracle_mutant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", so, c, "-lm"], check=True)
    return oracle.load_library(so)


def _words(rng, nbits):
    w = rng.integers(0, 2**32, size=(nbits + 31) // 32, dtype=np.uint64).astype(np.uint32)
    if nbits % 32:
        w[-1] &= np.uint32((1 << (nbits % 32)) - 1)
    return w


def _pins():
    """Run a compact set of the independent pins; return the names that fail."""
    failed = []
    rng = np.random.default_rng(7)
    # Philox / labels against ATen's philox_engine (values captured from a
    # compile of ATen's header at the first call; see test_oracle.py)
    keys = oracle.sampling_keys(20000, 2, oracle.KEY_BITS(9))
    if not np.array_equal(oracle.perm_from_keys(keys), np.argsort(keys, kind="stable").astype(np.uint32)):
        failed.append("order")
    ref = _aten_labels()
    if ref is not None and [oracle.sampling_key(i, 2) for i in range(len(ref))] != ref:
        failed.append("labels")
    # Toeplitz against an explicit T and against numpy.convolve
    s, k = 200, 70
    seed = _words(rng, s + k - 1)
    sb = oracle.bits_of(seed, s + k - 1).astype(np.int64)
    A = rng.integers(0, 2, size=s).astype(np.uint8)
    T = sb[np.arange(k)[:, None] - np.arange(s)[None, :] + s - 1]
    if not np.array_equal(oracle.toeplitz(seed, s, A, 0, k), (T @ A.astype(np.int64)) % 2):
        failed.append("explicit T")
    if not np.array_equal(oracle.toeplitz(seed, s, A, 0, k), (np.convolve(sb, A.astype(np.int64)) % 2)[s - 1:s - 1 + k]):
        failed.append("convolve")
    for c in (0, 1, s - 1):  # a unit vector picks one seed window
        e = np.zeros(s, dtype=np.uint8)
        e[c] = 1
        if not np.array_equal(oracle.toeplitz(seed, s, e, 0, k), sb[s - 1 - c:s - 1 - c + k]):
            failed.append("unit vector %d" % c)
    # whole method against a numpy composition
    n, m, s2, k2 = 3000, 5, 500, 77
    inw = _words(rng, n)
    sd = _words(rng, s2 + k2 - 1)
    perm = np.argsort(oracle.sampling_keys(n, 3), kind="stable")
    blocks = oracle.bits_of(inw, n)[perm[:m * s2]].reshape(m, s2).astype(np.int64)
    sbb = oracle.bits_of(sd, s2 + k2 - 1).astype(np.int64)
    bits = np.concatenate([np.convolve(sbb, blocks[j])[s2 - 1:s2 - 1 + k2] % 2 for j in range(m)]).astype(np.uint8)
    want = np.packbits(np.concatenate([bits, np.zeros((-bits.size) % 32, np.uint8)]), bitorder="little").view("<u4")
    if not np.array_equal(oracle.extract(n, m, s2, k2, inw, sd, 3), want):
        failed.append("composition")
    # i.i.d. law against numpy grouping and convolve, Eq. 7 against the exact tail
    keys = oracle.sampling_keys(n, 4)
    V = np.array([(int(x) * m) >> 64 for x in keys], dtype=np.int64)
    s3 = int(np.bincount(V, minlength=m).max()) + 5
    sizes, order, _ = oracle.iid_order(keys, m, s3)
    if order is None or not np.array_equal(sizes, np.bincount(V, minlength=m)) or any(
            not np.array_equal(order[j * s3:j * s3 + sizes[j]], np.flatnonzero(V == j)) for j in range(m)):
        failed.append("iid order")
    sd3 = _words(rng, s3 + k2 - 1)
    sb3 = oracle.bits_of(sd3, s3 + k2 - 1).astype(np.int64)
    bits3 = []
    for j in range(m):
        A = np.zeros(s3, dtype=np.int64)
        rows = np.flatnonzero(V == j)
        A[:rows.size] = oracle.bits_of(inw, n).astype(np.int64)[rows]
        bits3.append(np.convolve(sb3, A)[s3 - 1:s3 - 1 + k2] % 2)
    b3 = np.concatenate(bits3).astype(np.uint8)
    want3 = np.packbits(np.concatenate([b3, np.zeros((-b3.size) % 32, np.uint8)]), bitorder="little").view("<u4")
    try:
        if not np.array_equal(oracle.extract(n, m, s3, k2, inw, sd3, 4, oracle.SAMPLING_IID), want3):
            failed.append("iid composition")
    except (ValueError, oracle.Abort):
        failed.append("iid composition")
    try:
        from scipy import stats
        for N, mm in ((2**20, 64), (10**6, 17)):
            L = oracle.block_limit(N, mm, 1e-8, 1.0 / mm)
            if not (mm * stats.binom.sf(L, N, 1.0 / mm) <= 1e-8 < mm * stats.binom.sf(L - 2, N, 1.0 / mm)):
                failed.append("eq7 bracket")
    except ImportError:
        pass
    return failed


_ATEN = {}


def _aten_labels():
    if "v" in _ATEN:
        return _ATEN["v"]
    try:
        import torch
    except ImportError:
        _ATEN["v"] = None
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "a.cpp")
    with open(src, "w") as f:
        f.write('#include <ATen/core/PhiloxRNGEngine.h>\n#include <cstdio>\nint main(){for(unsigned long long i=0;i<64;++i)'
                '{at::philox_engine e(2,0,i);unsigned a=e(),b=e();std::printf("%u %u\\n",a,b);}}\n')
    exe = os.path.join(d, "a")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    _ATEN["v"] = [(int(out[2 * i]) << 32) | int(out[2 * i + 1]) for i in range(64)]
    return _ATEN["v"]


def test_unchanged_oracle_passes_every_pin(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _compile(SRC))
    assert _pins() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(monkeypatch, name):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, "mutation site not found: %s" % name
    monkeypatch.setattr(oracle, "_lib", _compile(SRC.replace(old, new)))
    assert _pins(), "no pin caught: %s" % name
