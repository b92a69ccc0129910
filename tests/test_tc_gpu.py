"""The direct GF(2) product on the tensor cores (EXTRACT_METHOD_TENSOR):
tcgen05.mma with 0/1 e4m3 operands and f32 accumulators, parities read back
per K chunk.  Bit-exact against the CPU oracle on ragged shapes (row tiles,
sub-block tiles and K blocks all partial), for every chunk length, against
the closed form of an all-ones seed and input (every output bit is the parity
of s, every chunk's sums are as large as they get), and against the direct
LOP3 kernel at a larger shape."""
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


def _run(n, m, s, k, flags, in_w, seed, key=2):
    with X.Extractor(n, m, s, k, seed, key, flags | X.EXTRACT_METHOD_TENSOR) as ex:
        assert ex.describe().startswith("tensor"), ex.describe()
        out = ex.run(_dev(in_w)).cpu().numpy().view(np.uint32)
        ex.status()  # no kernel gave up on a wait
    return out


@pytest.mark.parametrize("n,m,s,k", [
    (1 << 16, 8, 4096, 1500),        # one sub-block tile, 12 row tiles (the last partial)
    (200_000, 37, 5000, 3001),       # ragged rows, K blocks and sub-blocks
    (1 << 18, 8, 1 << 15, 1 << 13),  # the small plain sub-block case
    (300 * 512, 300, 512, 300),      # two sub-block tiles (256 + 44)
    (100, 1, 100, 1),                # one partial K block, one row
    (70_001, 5, 14_000, 7_000),      # n > m*s
])
def test_tensor_core_hash_matches_oracle(n, m, s, k):
    in_w = synth.bernoulli_bits(n, 0.7, 61)
    seed = synth.uniform_bits(s + k - 1, 62)
    assert np.array_equal(_run(n, m, s, k, 0, in_w, seed), oracle.extract(n, m, s, k, in_w, seed, 2))


def test_tensor_core_whole_block_identity_order():
    n = s = 1 << 16
    k = 1 << 15
    in_w = synth.bernoulli_bits(n, 0.6, 63)
    seed = synth.uniform_bits(s + k - 1, 64)
    got = _run(n, 1, s, k, X.EXTRACT_IDENTITY_PERM, in_w, seed)
    assert np.array_equal(got, oracle.extract(n, 1, s, k, in_w, seed, 0, oracle.IDENTITY_PERM))


@pytest.mark.parametrize("l", [0, 2, 5, 7])
def test_every_chunk_length_gives_the_same_bits(l):
    n, m, s, k = 300_000, 9, 30_000, 4_000
    in_w = synth.bernoulli_bits(n, 0.65, 65)
    seed = synth.uniform_bits(s + k - 1, 66)
    got = _run(n, m, s, k, X.EXTRACT_TC_CHUNK(l), in_w, seed)
    assert np.array_equal(got, oracle.extract(n, m, s, k, in_w, seed, 2))


@pytest.mark.parametrize("s", [(1 << 16) + 1, 1 << 16, 4096 * 3 + 5])
def test_all_ones_gives_the_parity_of_s(s):
    """All-ones seed and input: D[i][j] = s and every chunk sums to its full
    length (4096 by default), so K_j[i] = s mod 2 for every row."""
    m, k = 300, 1000
    n = m * s
    in_w = np.full((n + 31) // 32, 0xFFFFFFFF, dtype=np.uint32)
    if n % 32:
        in_w[-1] = np.uint32((1 << (n % 32)) - 1)
    seed = np.full((s + k - 1 + 31) // 32, 0xFFFFFFFF, dtype=np.uint32)
    got = oracle.bits_of(_run(n, m, s, k, 0, in_w, seed), m * k)
    assert np.all(got == (s & 1))


def test_tensor_core_hash_equals_direct_kernel_large():
    n, m, s, k = 1 << 24, 64, 1 << 18, 6553
    in_w = synth.bernoulli_bits(n, 0.8, 67)
    seed = synth.uniform_bits(s + k - 1, 68)
    a = _run(n, m, s, k, 0, in_w, seed)
    with X.Extractor(n, m, s, k, seed, 2, X.EXTRACT_METHOD_DIRECT) as ex:
        b = ex.run(_dev(in_w)).cpu().numpy().view(np.uint32)
    assert np.array_equal(a, b)
    # and two whole sub-blocks against the word-packed oracle
    keys = oracle.sampling_keys(n, 2)
    js = [0, m - 1]
    pos = oracle.perm_ranges(keys, [(j * s, s) for j in js])
    K = oracle.fast_window(in_w, pos, s, k, seed, 0, js, 0, k, seed_len_bits=s + k - 1)
    got = oracle.bits_of(a, m * k)
    for t, j in enumerate(js):
        assert np.array_equal(got[j * k:(j + 1) * k], K[t])


def test_tensor_method_rejects_per_subblock_seeds_and_two_methods():
    seed = np.zeros(100000, dtype=np.uint32)
    for fl in (X.EXTRACT_SEED_PER_SUBBLOCK, X.EXTRACT_METHOD_DIRECT, X.EXTRACT_METHOD_NTT):
        with pytest.raises(X.ExtractError) as e:
            X.extract_create(1 << 16, 4, 1 << 14, 100, seed, 1, fl | X.EXTRACT_METHOD_TENSOR)
        assert e.value.code == X.EXTRACT_EINVAL


def test_a_wait_that_runs_out_is_reported_and_the_device_stays_usable():
    """The error path of the bounded waits, without a GPU fault: with the
    test hook every CTA waits on a barrier nothing arrives on; after about a
    second the kernel sets the context's error word, frees its tensor memory
    and returns.  extract_status reports EXTRACT_ETIMEDOUT once, and a run
    right after it on the same device is bit-exact."""
    n, m, s, k = 1 << 16, 8, 4096, 1500
    in_w = synth.bernoulli_bits(n, 0.7, 69)
    seed = synth.uniform_bits(s + k - 1, 70)
    with X.Extractor(n, m, s, k, seed, 2, X.EXTRACT_METHOD_TENSOR | X.EXTRACT_TC_TEST_STALL) as ex:
        ex.run(_dev(in_w))
        with pytest.raises(X.ExtractError) as e:
            ex.status()
        assert e.value.code == X.EXTRACT_ETIMEDOUT
        ex.status()  # reported once, then cleared
    assert np.array_equal(_run(n, m, s, k, 0, in_w, seed), oracle.extract(n, m, s, k, in_w, seed, 2))
