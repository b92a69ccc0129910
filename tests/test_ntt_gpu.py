"""The exact NTT middle product (the FFT direction of Sec. I / Sec. V, done in
integers modulo a prime): bit-exact against the CPU oracle and against the
direct GF(2) kernel, over transform lengths 2^12 .. 2^22 and every split of
a sub-block into 2^l pieces."""
import numpy as np
import pytest

import oracle
from paper_2308_02856_gb300 import build as pkg_build
from paper_2308_02856_gb300 import extract as X
from paper_2308_02856_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg_build.build()
    X.load()


def _dev(words):
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def _run(n, m, s, k, flags, in_w, seed, key=2):
    with X.Extractor(n, m, s, k, seed, key, flags) as ex:
        desc = ex.describe()
        out = _host(ex.run(_dev(in_w)))
    return out, desc


ORACLE_CASES = [
    # n, m, s, k  (s + k - 1 sets the transform length)
    (8192, 2, 4000, 1000),          # N = 8192
    (4096 * 3, 3, 4096, 1),         # k = 1, N = 4096
    (2049 * 2, 2, 2049, 1),         # s + k - 1 = 2049: the smallest NTT shape
    (6000, 1, 3000, 3000),          # k = s
    (200_000, 37, 5000, 3001),      # ragged
    (1 << 18, 8, 1 << 15, 1 << 13),  # the small plain sub-block case, N = 2^16
    (70_001, 5, 14_000, 7_000),     # N = 32768, n > m*s
]


@pytest.mark.parametrize("n,m,s,k", ORACLE_CASES)
def test_ntt_matches_oracle(n, m, s, k):
    in_w = synth.bernoulli_bits(n, 0.7, 11)
    seed = synth.uniform_bits(s + k - 1, 12)
    got, desc = _run(n, m, s, k, X.EXTRACT_METHOD_NTT, in_w, seed)
    assert desc.startswith("ntt")
    want = oracle.extract(n, m, s, k, in_w, seed, 2)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,m,s,k,p", [
    (1 << 22, 4, 1 << 20, 1 << 19, 0.6),     # the QRNG sub-block shape (P = 2, N = 2^20)
    (1 << 21, 2, 1 << 20, 104858, 0.9),      # the QKD sub-block shape (P = 8, N = 2^18; k mod 32 = 26)
    (3 * ((1 << 21) + 1), 3, (1 << 21) + 1, 1 << 21, 0.5),  # s + k - 1 = 2^22: the largest NTT shape
    (1 << 20, 16, 1 << 16, 1 << 15, 0.55),
    (5_000_000, 9, 333_333, 77_777, 0.8),
])
def test_ntt_matches_direct_kernel(n, m, s, k, p):
    in_w = synth.bernoulli_bits(n, p, 21)
    seed = synth.uniform_bits(s + k - 1, 22)
    a, da = _run(n, m, s, k, X.EXTRACT_METHOD_NTT, in_w, seed)
    b, db = _run(n, m, s, k, X.EXTRACT_METHOD_DIRECT, in_w, seed)
    assert da.startswith("ntt") and not db.startswith("ntt")
    assert np.array_equal(a, b)
    # and sampled rows of two sub-blocks against the oracle
    got = oracle.bits_of(a, m * k)
    perm = oracle.perm(n, 2)
    rng = np.random.default_rng(3)
    for j in (0, m - 1):
        A = oracle.subblock(in_w, perm[j * s:(j + 1) * s])
        for i in np.concatenate([[0, 1, k - 1], rng.choice(k, 20, replace=False)]):
            assert got[j * k + i] == oracle.toeplitz_bit(seed, s, A, int(i)), (j, i)


@pytest.mark.parametrize("n,m,s,k", [
    (8192, 2, 4000, 1000),            # last piece ragged (4000 = 2016 + 1984 at P = 2)
    (1 << 18, 8, 1 << 15, 1 << 13),   # pieces of whole words at every P
    (70_001, 5, 14_000, 7_000),
    (3 * 40_001, 3, 40_001, 333),     # small k: up to 16 pieces; s odd
])
def test_ntt_every_split_matches_oracle(n, m, s, k):
    """Each sub-block split into 2^l pieces (one middle product per piece,
    summed before the inverse transform) gives the oracle's bits."""
    in_w = synth.bernoulli_bits(n, 0.65, 31)
    seed = synth.uniform_bits(s + k - 1, 32)
    want = oracle.extract(n, m, s, k, in_w, seed, 2)
    ran = []
    for l in range(5):
        try:
            got, desc = _run(n, m, s, k, X.EXTRACT_METHOD_NTT | X.EXTRACT_NTT_SPLIT(l), in_w, seed)
        except X.ExtractError as e:
            assert e.code == X.EXTRACT_EINVAL  # no transform length for this split
            continue
        assert " P=%d " % (1 << l) in desc, desc
        assert np.array_equal(got, want), "split 2^%d" % l
        ran.append(l)
    assert len(ran) >= 3, ran


@pytest.mark.parametrize("n,m,s,k", [
    (1 << 18, 4, 1 << 15, 1 << 13),   # N = 2^16, P = 1
    (1 << 20, 8, 1 << 17, 1 << 15),   # P = 2
    (300_000, 3, 70_001, 9_999),      # P = 2, ragged last piece and seed windows
])
def test_ntt_independent_seeds_match_oracle(n, m, s, k):
    """One seed per sub-block (the paper's independent f_RE,j): each
    sub-block's seed windows are transformed in the run and multiplied into
    its own pieces."""
    in_w = synth.bernoulli_bits(n, 0.6, 41)
    seed = synth.uniform_bits((s + k - 1) * m, 42)
    got, desc = _run(n, m, s, k, X.EXTRACT_SEED_PER_SUBBLOCK | X.EXTRACT_METHOD_NTT, in_w, seed)
    assert desc.startswith("ntt") and "one seed per sub-block" in desc, desc
    want = oracle.extract(n, m, s, k, in_w, seed, 2, oracle.SEED_PER_SUBBLOCK)
    assert np.array_equal(got, want)


def test_ntt_independent_seeds_every_split():
    n, m, s, k = 1 << 20, 8, 1 << 17, 1 << 15
    in_w = synth.bernoulli_bits(n, 0.7, 43)
    seed = synth.uniform_bits((s + k - 1) * m, 44)
    want = oracle.extract(n, m, s, k, in_w, seed, 2, oracle.SEED_PER_SUBBLOCK)
    for l in range(5):
        got, desc = _run(n, m, s, k, X.EXTRACT_SEED_PER_SUBBLOCK | X.EXTRACT_METHOD_NTT | X.EXTRACT_NTT_SPLIT(l),
                         in_w, seed)
        assert " P=%d " % (1 << l) in desc, desc
        assert np.array_equal(got, want), "split 2^%d" % l


def test_ntt_independent_seeds_large_equal_direct():
    n, m, s, k = 5_000_000, 9, 333_333, 77_777
    in_w = synth.bernoulli_bits(n, 0.8, 45)
    seed = synth.uniform_bits((s + k - 1) * m, 46)
    a, da = _run(n, m, s, k, X.EXTRACT_SEED_PER_SUBBLOCK | X.EXTRACT_METHOD_NTT, in_w, seed)
    b, db = _run(n, m, s, k, X.EXTRACT_SEED_PER_SUBBLOCK | X.EXTRACT_METHOD_DIRECT, in_w, seed)
    assert da.startswith("ntt") and not db.startswith("ntt")
    assert np.array_equal(a, b)
    got = oracle.bits_of(a, m * k)
    perm = oracle.perm(n, 2)
    L = s + k - 1
    rng = np.random.default_rng(5)
    for j in (0, m - 1):
        A = oracle.subblock(in_w, perm[j * s:(j + 1) * s])
        for i in np.concatenate([[0, k - 1], rng.choice(k, 12, replace=False)]):
            assert got[j * k + i] == oracle.toeplitz_bit(seed, s, A, int(i), off=j * L), (j, i)


def test_ntt_flag_rejections():
    seed = np.zeros(10000, dtype=np.uint32)
    for n, m, s, k, fl in [
        (4096, 2, 1024, 512, 0),                                  # s + k - 1 <= 2^11
        (1 << 24, 1, 1 << 23, 1 << 22, 0),                       # s + k - 1 > 2^22
        (2 ** 14, 2, 4096, 100, X.EXTRACT_SEED_PER_SUBBLOCK),     # one seed per sub-block needs N >= 2^16
        (2 ** 14, 2, 4096, 100, X.EXTRACT_METHOD_DIRECT),         # both methods
        (4096 * 2, 2, 2049, 1000, X.EXTRACT_NTT_SPLIT(4)),        # 16 pieces would leave one empty
        (4096 * 2, 2, 2049, 1000, 6 << 16),                       # split field out of range
    ]:
        with pytest.raises(X.ExtractError) as e:
            X.extract_create(n, m, s, k, seed, 1, fl | X.EXTRACT_METHOD_NTT)
        assert e.value.code == X.EXTRACT_EINVAL


def test_auto_method_picks_ntt_for_large_sub_blocks_and_direct_for_small():
    seed = synth.uniform_bits((1 << 20) + (1 << 19), 1)
    with X.Extractor(1 << 22, 4, 1 << 20, 1 << 19, seed, 2) as ex:
        assert ex.describe().startswith("ntt")
    with X.Extractor(4096, 4, 1024, 512, seed, 2) as ex:
        assert not ex.describe().startswith("ntt")
