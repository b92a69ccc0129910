"""Pins of the oracle's i.i.d. sampling law (Sec. III.B step 1 as the paper
states it) and of the Eq. 7 block size limit, each against something other
than the oracle: Python integers, numpy's grouping routines, numpy.convolve,
and SciPy's exact binomial tail."""
import numpy as np
import pytest

import oracle

stats = pytest.importorskip("scipy.stats")


def _words(rng, nbits):
    w = rng.integers(0, 2**32, size=(nbits + 31) // 32, dtype=np.uint64).astype(np.uint32)
    if nbits % 32:
        w[-1] &= np.uint32((1 << (nbits % 32)) - 1)
    return w


def test_label_is_the_high_word_of_key_times_m():
    rng = np.random.default_rng(1)
    keys = [0, 1, 2**63, 2**64 - 1] + [int(x) for x in rng.integers(0, 2**63, size=300, dtype=np.uint64) * 2 + 1]
    for m in (1, 2, 3, 7, 17, 1000, 4096, 65535, 2**31 + 11):
        for key in keys:
            assert oracle.iid_label(key, m) == (key * m) >> 64
        assert oracle.iid_label(2**64 - 1, m) == m - 1


def test_labels_are_uniform():
    keys = oracle.sampling_keys(200_000, 9)
    m = 13
    V = np.array([oracle.iid_label(int(x), m) for x in keys[:20000]])
    counts = np.bincount(V, minlength=m)
    mean = 20000 / m
    assert np.all(np.abs(counts - mean) < 6 * np.sqrt(mean))


@pytest.mark.parametrize("n,m,key", [(1000, 7, 5), (4096, 64, 2), (777, 1, 3), (50, 100, 4), (30000, 17, 8)])
def test_order_groups_positions_in_increasing_order(n, m, key):
    keys = oracle.sampling_keys(n, key)
    V = np.array([(int(x) * m) >> 64 for x in keys], dtype=np.int64)
    want_sizes = np.bincount(V, minlength=m)
    s = int(want_sizes.max()) + 3
    sizes, order, largest = oracle.iid_order(keys, m, s)
    assert np.array_equal(sizes, want_sizes) and largest == want_sizes.max() and sizes.sum() == n
    order = order.reshape(m, s)
    for j in range(m):
        rows = np.flatnonzero(V == j)
        assert np.array_equal(order[j, :rows.size], rows)
        assert np.all(order[j, rows.size:] == oracle.NO_POS)


def test_abort_when_a_sub_block_exceeds_the_limit():
    n, m = 5000, 9
    keys = oracle.sampling_keys(n, 6)
    sizes, order, largest = oracle.iid_order(keys, m, 10**6)
    assert order is not None
    _, order2, largest2 = oracle.iid_order(keys, m, largest - 1)
    assert order2 is None and largest2 == largest
    rng = np.random.default_rng(0)
    inw = _words(rng, n)
    sd = _words(rng, largest - 1 + 8 - 1)
    with pytest.raises(oracle.Abort):
        oracle.extract(n, m, largest - 1, 8, inw, sd, 6, oracle.SAMPLING_IID)
    oracle.extract(n, m, largest, 8, inw, sd[:], 6, oracle.SAMPLING_IID)  # at the limit it runs


@pytest.mark.parametrize("n,m,k,slack,flags", [
    (3000, 5, 77, 0, 0), (4000, 8, 300, 37, 0), (999, 3, 1, 5, 0), (2500, 4, 100, 10, oracle.SEED_PER_SUBBLOCK),
    (6000, 16, 64, 3, oracle.KEY_BITS(12)),
])
def test_iid_method_matches_a_numpy_composition(n, m, k, slack, flags):
    rng = np.random.default_rng(n)
    key = 11
    keys = oracle.sampling_keys(n, key, flags)
    V = np.array([(int(x) * m) >> 64 for x in keys], dtype=np.int64)
    s = int(np.bincount(V, minlength=m).max()) + slack
    L = s + k - 1
    inw = _words(rng, n)
    sd = _words(rng, L * (m if flags & oracle.SEED_PER_SUBBLOCK else 1))
    bits = oracle.bits_of(inw, n).astype(np.int64)
    sbits = oracle.bits_of(sd, L * (m if flags & oracle.SEED_PER_SUBBLOCK else 1)).astype(np.int64)
    out = []
    for j in range(m):
        A = np.zeros(s, dtype=np.int64)
        rows = np.flatnonzero(V == j)
        A[:rows.size] = bits[rows]
        sj = sbits[j * L:(j + 1) * L] if flags & oracle.SEED_PER_SUBBLOCK else sbits
        out.append(np.convolve(sj, A)[s - 1:s - 1 + k] % 2)
    want_bits = np.concatenate(out).astype(np.uint8)
    want = np.packbits(np.concatenate([want_bits, np.zeros((-want_bits.size) % 32, np.uint8)]),
                       bitorder="little").view("<u4")
    got = oracle.extract(n, m, s, k, inw, sd, key, flags | oracle.SAMPLING_IID)
    assert np.array_equal(got, want)


def test_padding_reads_as_zero():
    inw = np.full(4, 0xFFFFFFFF, dtype=np.uint32)
    pos = np.array([0, 5, oracle.NO_POS, 7, oracle.NO_POS], dtype=np.uint32)
    assert list(oracle.subblock_padded(inw, pos)) == [1, 1, 0, 1, 0]


@pytest.mark.parametrize("N,L,p", [(1000, 30, 0.02), (10**6, 1100, 1e-3), (10**5, 6000, 0.05),
                                   (2**20, 17000, 1 / 64), (10**9, 58_900_000, 1 / 17)])
def test_tail_bound_brackets_the_exact_binomial_tail(N, L, p):
    """Zubkov-Serov: P(X > L) <= bound(L) <= P(X > L - 1) for L >= N p + 1."""
    b = oracle.size_tail_bound(N, L, p)
    assert stats.binom.sf(L, N, p) <= b * (1 + 1e-9)
    assert b <= stats.binom.sf(L - 1, N, p) * (1 + 1e-9)


@pytest.mark.parametrize("N,m,eps", [(2**20, 64, 1e-8), (10**6, 17, 1e-8), (10**9, 17, 1e-8),
                                     (2**30, 1024, 1e-8), (2**32, 4096, 1e-6), (5000, 5, 1e-3)])
def test_block_limit_is_the_first_limit_eq7_accepts(N, m, eps):
    """Eq. 7 with p_sift = 1/m.  The limit L makes the union bound hold for
    the exact tail (m P(X > L) <= eps), and the next smaller limit is already
    too small by the lower half of the bound (m P(X > L - 2) > eps)."""
    p = 1.0 / m
    L = oracle.block_limit(N, m, eps, p)
    assert N * p < L < N
    assert m * stats.binom.sf(L, N, p) <= eps
    assert m * stats.binom.sf(L - 2, N, p) > eps
    assert oracle.block_limit(N, m, eps / 100, p) > L  # a smaller failure chance needs a larger limit
