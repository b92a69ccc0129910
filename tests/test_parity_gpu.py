"""GPU parity: every step of the CUDA path, called through the C ABI, against
the CPU oracle on the same seeded inputs.  All results are bits, so the bar is
bit-exact equality."""
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


def _dev(words: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)).cuda()


def _host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def _seed_len(m, s, k, flags):
    return (s + k - 1) * (m if flags & X.EXTRACT_SEED_PER_SUBBLOCK else 1)


# --------------------------------------------------------------------------
# step 1: the sampled order
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,key,flags", [
    (1, 2, 0), (2, 2, 0), (33, 5, 0), (1000, 2, 0), (1024, 3, 0), (1025, 3, 0),
    (65536, 2, 0), (100003, 99, 0), (1 << 20, 2, 0), (3_000_001, 0x0123456789ABCDEF, 0),
    (4096, 2, X.EXTRACT_KEY_BITS(4)),     # 16 distinct labels, one bucket: heavy ties
    (50000, 7, X.EXTRACT_KEY_BITS(8)),
    (1 << 15, 3, X.EXTRACT_KEY_BITS(2)),  # buckets larger than shared memory
])
def test_sampled_order_matches_oracle(n, key, flags):
    seed = np.zeros(4, dtype=np.uint32)
    with X.Extractor(n, 1, 1, 1, seed, key, flags) as ex:
        got = ex.read_perm()
    want = oracle.perm(n, key, flags)
    assert np.array_equal(got, want)


# --------------------------------------------------------------------------
# step 1 (gather): sub-blocks as stored for the hashing kernel
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,s,flags", [
    (4096, 4, 1000, 0), (70000, 3, 20000, 0), (1 << 18, 8, 1 << 15, 0), (5000, 1, 5000, X.EXTRACT_IDENTITY_PERM),
    (100, 3, 33, 0),
])
def test_gather_matches_oracle(n, m, s, flags):
    in_w = synth.bernoulli_bits(n, 0.7, 1)
    seed = synth.uniform_bits(s, 3)
    p = oracle.perm(n, 2, flags)
    with X.Extractor(n, m, s, 1, seed, 2, flags) as ex:
        ex.gather(_dev(in_w))
        torch.cuda.synchronize()
        for j in range(m):
            A = oracle.subblock(in_w, p[j * s:(j + 1) * s])
            want = oracle.bits_of(np.packbits(np.concatenate([A[::-1], np.zeros((-s) % 32, np.uint8)]),
                                              bitorder="little").view("<u4"), s)
            got = oracle.bits_of(ex.read_subblock(j), s)
            assert np.array_equal(got, want), j


# --------------------------------------------------------------------------
# steps 1-3: whole runs
# --------------------------------------------------------------------------

CASES = [
    # n, m, s, k, p, flags
    (256, 4, 64, 32, 0.7, 0),
    (1000, 3, 300, 77, 0.6, 0),                 # s, k not multiples of 32; n > m*s
    (4096, 1, 4096, 1, 0.5, 0),                 # m = 1, k = 1
    (3000, 7, 400, 400, 0.7, 0),                # k = s
    (2048, 8, 256, 100, 0.7, X.EXTRACT_SEED_PER_SUBBLOCK),
    (1500, 1, 1500, 700, 0.7, X.EXTRACT_IDENTITY_PERM),
    (4096, 16, 256, 64, 0.9, X.EXTRACT_KEY_BITS(4)),
    (65, 1, 33, 31, 0.7, 0),
    (1 << 18, 8, 1 << 15, 1 << 13, 0.7, 0),     # the small plain sub-block case in full
    (185_123, 37, 5000, 3000, 0.55, 0),         # ragged rows, words, sub-block tiles
    (200_000, 40, 5000, 1111, 0.8, X.EXTRACT_SEED_PER_SUBBLOCK),
    (131072, 64, 2048, 1500, 0.9, 0),           # several sub-block tiles of 32
]


def _run_case(n, m, s, k, p, flags, plain=False, method=0):
    in_w = synth.bernoulli_bits(n, p, 1)
    seed = synth.uniform_bits(_seed_len(m, s, k, flags), 3)
    with X.Extractor(n, m, s, k, seed, 2, flags | method) as ex:
        out = ex.run_plain(_dev(in_w)) if plain else ex.run(_dev(in_w))
        got = _host(out)
        if method == X.EXTRACT_METHOD_TENSOR:
            assert ex.describe().startswith("tensor")
            ex.status()
        if method == X.EXTRACT_METHOD_DIRECT:
            assert ex.describe().startswith("lop3")
    want = oracle.extract(n, m, s, k, in_w, seed, 2, flags)
    return got, want


METHODS = {"auto": 0, "direct": X.EXTRACT_METHOD_DIRECT, "tensor": X.EXTRACT_METHOD_TENSOR}


@pytest.mark.parametrize("method", sorted(METHODS))
@pytest.mark.parametrize("n,m,s,k,p,flags", CASES)
def test_run_matches_oracle(n, m, s, k, p, flags, method):
    """Every case under the library's own choice of method and under the
    direct LOP3 kernel and the tensor-core product forced (the latter needs
    a shared seed)."""
    if method == "tensor" and flags & X.EXTRACT_SEED_PER_SUBBLOCK:
        pytest.skip("the tensor-core product needs a shared seed")
    got, want = _run_case(n, m, s, k, p, flags, method=METHODS[method])
    assert got.shape == want.shape
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "first differing word %s of %d" % (bad[:5], got.size)


@pytest.mark.parametrize("n,m,s,k,p,flags", [CASES[1], CASES[4], CASES[8], CASES[9]])
def test_plain_path_matches_oracle(n, m, s, k, p, flags):
    got, want = _run_case(n, m, s, k, p, flags, plain=True)
    assert np.array_equal(got, want)


def test_output_is_fully_overwritten_and_runs_repeat():
    n, m, s, k = 20000, 5, 3000, 999
    in_w = synth.bernoulli_bits(n, 0.6, 4)
    seed = synth.uniform_bits(s + k - 1, 5)
    want = oracle.extract(n, m, s, k, in_w, seed, 9)
    with X.Extractor(n, m, s, k, seed, 9) as ex:
        out = torch.full(((m * k + 31) // 32,), -1, dtype=torch.int32, device="cuda")
        d = _dev(in_w)
        for _ in range(3):
            ex.run(d, out)
            assert np.array_equal(_host(out), want)


def test_direct_whole_block_against_oracle_rows():
    """m = 1, identity order: the traditional whole-block hash (Sec. IV.C),
    checked on sampled rows at n = 2^18, k = 2^16."""
    n, k = 1 << 18, 1 << 16
    in_w = synth.bernoulli_bits(n, 0.7, 1)
    seed = synth.uniform_bits(n + k - 1, 3)
    with X.Extractor(n, 1, n, k, seed, 0, X.EXTRACT_IDENTITY_PERM) as ex:
        got = oracle.bits_of(_host(ex.run(_dev(in_w))), k)
    A = oracle.bits_of(in_w, n)
    rng = np.random.default_rng(0)
    rows = np.concatenate([np.arange(64), np.arange(k - 64, k), rng.choice(k, 200, replace=False)])
    for i in rows:
        assert got[i] == oracle.toeplitz_bit(seed, n, A, int(i)), i


def test_two_contexts_interleaved_on_streams():
    n, m, s, k = 50000, 6, 8000, 700
    a_in = synth.bernoulli_bits(n, 0.7, 11)
    b_in = synth.bernoulli_bits(n, 0.6, 12)
    seed = synth.uniform_bits(s + k - 1, 13)
    want_a = oracle.extract(n, m, s, k, a_in, seed, 21)
    want_b = oracle.extract(n, m, s, k, b_in, seed, 22)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with X.Extractor(n, m, s, k, seed, 21) as ea, X.Extractor(n, m, s, k, seed, 22) as eb:
        da, db = _dev(a_in), _dev(b_in)
        torch.cuda.synchronize()
        oa, ob = ea.new_output(), eb.new_output()
        for _ in range(3):
            ea.run(da, oa, stream=s1)
            eb.run(db, ob, stream=s2)
        torch.cuda.synchronize()
        assert np.array_equal(_host(oa), want_a)
        assert np.array_equal(_host(ob), want_b)
