"""The bucketed two-stage gather (EXTRACT_GATHER_BUCKETS, the default for
inputs of 2^22 bits and more): every stored bit of every sub-block against
the oracle's sub-blocks, on shapes that span several 2^16-bit input chunks
with ragged tails, ties in the labels, unselected positions, both sampling
laws, and through the hash against the oracle's output."""
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


def _dev(words, offset_words=0):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    t = torch.zeros(w.size + offset_words, dtype=torch.int32, device="cuda")
    t[offset_words:] = torch.from_numpy(w.view(np.int32)).cuda()
    return t[offset_words:]


def _stored(ex, j, s):
    return oracle.bits_of(ex.read_subblock(j), s)[::-1]  # stored reversed: bit c = slot s-1-c


def _check_sorted(n, m, s, key, flags=0, offset_words=0, blocks=None):
    in_w = synth.bernoulli_bits(n, 0.5, 11)
    keys = oracle.sampling_keys(n, key, flags)
    seed = synth.uniform_bits(s, 1)
    with X.Extractor(n, m, s, 1, seed, key, flags | X.EXTRACT_GATHER_BUCKETS | X.EXTRACT_METHOD_DIRECT) as ex:
        assert "gather=buckets" in ex.describe()
        chunk = "2^18-bit chunks" if flags & X.EXTRACT_GATHER_WIDE_CHUNKS else "2^16-bit chunks"
        assert chunk in ex.describe()
        ex.gather(_dev(in_w, offset_words))
        for j in (range(m) if blocks is None else blocks):
            want = oracle.subblock(in_w, oracle.perm_range(keys, j * s, s))
            assert np.array_equal(_stored(ex, j, s), want), "sub-block %d" % j


@pytest.mark.parametrize("n,m,s,key,flags", [
    (3 * 65536 + 12345, 7, 27999, 3, 0),          # four chunks, ragged tail, m*s < n
    (1 << 20, 64, 1 << 14, 2, 0),                 # m*s = n: every position sampled
    (1 << 18, 1, 1 << 18, 5, 0),                  # one sub-block over every chunk
    (100_000, 1000, 100, 7, 0),                   # many tiny sub-blocks, mostly empty runs
    (200_000, 9, 20_000, 4, X.EXTRACT_KEY_BITS(12)),  # many equal labels
    (65_536, 3, 21_845, 9, 0),                    # exactly one chunk
    (65_537, 2, 32_768, 6, 0),                    # one bit in the last chunk
    (777, 5, 150, 8, 0),                          # less than one word group
])
def test_sorted_order_subblocks_match_the_oracle(n, m, s, key, flags):
    _check_sorted(n, m, s, key, flags)


W = X.EXTRACT_GATHER_WIDE_CHUNKS


@pytest.mark.parametrize("n,m,s,key,flags", [
    (3 * 262144 + 12345, 7, 100_001, 3, W),       # four 2^18-bit chunks, ragged tail, m*s < n
    (1 << 20, 64, 1 << 14, 2, W),                 # m*s = n
    (200_000, 9, 20_000, 4, W | X.EXTRACT_KEY_BITS(12)),
    (262_144, 3, 87_381, 9, W),                   # exactly one chunk
    (777, 5, 150, 8, W),
])
def test_wide_chunks_subblocks_match_the_oracle(n, m, s, key, flags):
    """2^18-bit input chunks with 32-bit table entries (the form the library
    takes for inputs of more than 25600 chunks of 2^16 bits)."""
    _check_sorted(n, m, s, key, flags)


def test_wide_chunks_input_not_16_byte_aligned():
    _check_sorted(3 * 262144 + 100, 6, 100_000, 13, W, offset_words=1)


def test_many_small_subblocks():
    """m = 20000 sub-blocks of 50 bits: most runs are empty or one word."""
    _check_sorted(1 << 20, 20000, 50, 12, 0, blocks=[0, 1, 777, 8191, 16383, 19999])


def test_input_not_16_byte_aligned():
    _check_sorted(3 * 65536 + 100, 6, 30_000, 13, 0, offset_words=1)


@pytest.mark.parametrize("n,m,key,flags", [
    (100_000, 7, 3, 0), (1 << 18, 64, 2, 0), (200_000, 33, 4, X.EXTRACT_KEY_BITS(14)), (70_000, 1, 5, 0),
    (600_000, 5, 6, X.EXTRACT_GATHER_WIDE_CHUNKS),
])
def test_iid_law_subblocks_match_the_oracle(n, m, key, flags):
    in_w = synth.bernoulli_bits(n, 0.5, 12)
    keys = oracle.sampling_keys(n, key, flags)
    _, _, largest = oracle.iid_order(keys, m, n, with_order=False)
    s = largest + 33
    sizes, order, _ = oracle.iid_order(keys, m, s)
    seed = synth.uniform_bits(s, 1)
    with X.Extractor(n, m, s, 1, seed, key, flags | X.EXTRACT_SAMPLING_IID | X.EXTRACT_GATHER_BUCKETS |
                     X.EXTRACT_METHOD_DIRECT) as ex:
        assert "gather=buckets" in ex.describe()
        ex.gather(_dev(in_w))
        for j in range(m):
            want = oracle.subblock_padded(in_w, order[j * s:(j + 1) * s])
            assert np.array_equal(_stored(ex, j, s), want), "sub-block %d" % j


@pytest.mark.parametrize("n,m,s,k,method,flags", [
    (300_000, 9, 30_000, 4_000, X.EXTRACT_METHOD_DIRECT, 0),
    (300_000, 9, 30_000, 4_000, X.EXTRACT_METHOD_NTT, 0),
    (1 << 18, 4, 1 << 16, 1 << 15, X.EXTRACT_METHOD_NTT, X.EXTRACT_SEED_PER_SUBBLOCK),
])
def test_hash_through_the_buckets_matches_the_oracle(n, m, s, k, method, flags):
    in_w = synth.bernoulli_bits(n, 0.6, 13)
    seed = synth.uniform_bits((s + k - 1) * (m if flags & X.EXTRACT_SEED_PER_SUBBLOCK else 1), 4)
    with X.Extractor(n, m, s, k, seed, 2, flags | method | X.EXTRACT_GATHER_BUCKETS) as ex:
        got = ex.run(_dev(in_w)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.extract(n, m, s, k, in_w, seed, 2, flags))


def test_iid_hash_through_the_buckets_matches_the_oracle():
    n, m, k = 250_000, 6, 2_000
    _, _, largest = oracle.iid_order(oracle.sampling_keys(n, 7), m, n, with_order=False)
    s = largest + 3
    in_w = synth.bernoulli_bits(n, 0.6, 14)
    seed = synth.uniform_bits(s + k - 1, 5)
    flags = X.EXTRACT_SAMPLING_IID | X.EXTRACT_GATHER_BUCKETS
    with X.Extractor(n, m, s, k, seed, 7, flags) as ex:
        got = ex.run(_dev(in_w)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.extract(n, m, s, k, in_w, seed, 7, oracle.SAMPLING_IID))


def test_default_choice_and_plain_give_the_same_subblocks():
    n, m, s = 1 << 22, 64, 1 << 16
    in_w = synth.bernoulli_bits(n, 0.5, 15)
    seed = synth.uniform_bits(s, 1)
    d_in = _dev(in_w)
    with X.Extractor(n, m, s, 1, seed, 3, X.EXTRACT_METHOD_DIRECT) as a, \
            X.Extractor(n, m, s, 1, seed, 3, X.EXTRACT_METHOD_DIRECT | X.EXTRACT_GATHER_PLAIN) as b:
        assert "gather=buckets" in a.describe() and "gather=plain" in b.describe()
        a.gather(d_in)
        b.gather(d_in)
        for j in (0, 1, 31, 63):
            assert np.array_equal(a.read_subblock(j), b.read_subblock(j)), "sub-block %d" % j
    keys = oracle.sampling_keys(n, 3)
    for j in (0, 63):
        with X.Extractor(n, m, s, 1, seed, 3, X.EXTRACT_METHOD_DIRECT) as a:
            a.gather(d_in)
            assert np.array_equal(_stored(a, j, s), oracle.subblock(in_w, oracle.perm_range(keys, j * s, s)))


def test_too_wide_region_falls_back_or_is_refused():
    """One sub-block of 2^22 bits needs 512 KiB in one CTA: the default keeps
    the plain gather, the explicit flag is refused."""
    n = s = 1 << 22
    seed = synth.uniform_bits(s, 1)
    with X.Extractor(n, 1, s, 1, seed, 3, X.EXTRACT_METHOD_DIRECT) as ex:
        assert "gather=plain" in ex.describe()
    with pytest.raises(X.ExtractError) as e:
        X.Extractor(n, 1, s, 1, seed, 3, X.EXTRACT_METHOD_DIRECT | X.EXTRACT_GATHER_BUCKETS)
    assert e.value.code == X.EXTRACT_EINVAL


@pytest.mark.parametrize("n,m,s,flags", [
    (1000, 2, 100, X.EXTRACT_GATHER_BUCKETS | X.EXTRACT_GATHER_PLAIN),
    (1000, 2, 100, X.EXTRACT_GATHER_WIDE_CHUNKS | X.EXTRACT_GATHER_PLAIN),
    (1000, 2, 100, X.EXTRACT_GATHER_BUCKETS | X.EXTRACT_IDENTITY_PERM),
])
def test_rejected_combinations(n, m, s, flags):
    seed = synth.uniform_bits(s, 1)
    with pytest.raises(X.ExtractError) as e:
        X.Extractor(n, m, s, 1, seed, 3, flags | X.EXTRACT_METHOD_DIRECT)
    assert e.value.code == X.EXTRACT_EINVAL


@pytest.mark.parametrize("n,m,s,k,flags", [
    (300_000, 9, 30_000, 4_000, X.EXTRACT_GATHER_BUCKETS | X.EXTRACT_METHOD_DIRECT),
    (5 << 20, 5, 1 << 20, 1000, 0),  # default choice at 5 Mbit: the tables
    (5 << 20, 5, 1 << 20, 1000, X.EXTRACT_GATHER_WIDE_CHUNKS),
])
def test_host_buffers_through_the_buckets_match_the_oracle(n, m, s, k, flags):
    """extract_run_host overlaps its copies with stage 1 and the hash."""
    in_w = synth.bernoulli_bits(n, 0.6, 16)
    seed = synth.uniform_bits(s + k - 1, 6)
    want = oracle.extract(n, m, s, k, in_w, seed, 2)
    with X.Extractor(n, m, s, k, seed, 2, flags) as ex:
        assert "gather=buckets" in ex.describe()
        for _ in range(2):  # the second call reuses the copy stream and events
            got = ex.run_host(np.ascontiguousarray(in_w, dtype=np.uint32))
            assert np.array_equal(got, want)


def test_host_buffers_ntt_in_several_launch_groups():
    """Two launch groups (128 + 16 sub-blocks of the QRNG sub-block shape);
    k mod 32 = 25, so neighbouring groups share an output word and each
    group's words go to the host while later groups run.  Sampled rows of
    every sub-block against the oracle, the first and last rows of each
    included."""
    n, m, s, k = 144 << 20, 144, 1 << 20, (1 << 19) - 7
    in_w = synth.bernoulli_bits(n, 0.6, 16)
    seed = synth.uniform_bits(s + k - 1, 6)
    with X.Extractor(n, m, s, k, seed, 2, X.EXTRACT_METHOD_NTT) as ex:
        plan = ex.describe()
        assert "gather=buckets" in plan
        assert int(plan.split(" sub-blocks per launch group")[0].split(",")[-1]) < m
        got = oracle.bits_of(ex.run_host(np.ascontiguousarray(in_w, dtype=np.uint32)), m * k)
        dev = oracle.bits_of(ex.run(_dev(in_w)).cpu().numpy().view(np.uint32), m * k)
    assert np.array_equal(got, dev)
    keys = oracle.sampling_keys(n, 2)
    rng = np.random.default_rng(3)
    for j in range(m):
        A = oracle.subblock(in_w, oracle.perm_range(keys, j * s, s))
        rows = np.unique(np.concatenate([np.arange(4), np.arange(k - 4, k), rng.choice(k, 8, replace=False)]))
        want = np.array([oracle.toeplitz_bit(seed, s, A, int(i)) for i in rows], dtype=np.uint8)
        assert np.array_equal(got[j * k + rows], want), "sub-block %d" % j


def test_iid_host_buffers_through_the_buckets_match_the_oracle():
    n, m, k = 250_000, 6, 2_000
    _, _, largest = oracle.iid_order(oracle.sampling_keys(n, 7), m, n, with_order=False)
    s = largest + 3
    in_w = synth.bernoulli_bits(n, 0.6, 17)
    seed = synth.uniform_bits(s + k - 1, 5)
    with X.Extractor(n, m, s, k, seed, 7, X.EXTRACT_SAMPLING_IID | X.EXTRACT_GATHER_BUCKETS) as ex:
        got = ex.run_host(np.ascontiguousarray(in_w, dtype=np.uint32))
    assert np.array_equal(got, oracle.extract(n, m, s, k, in_w, seed, 7, oracle.SAMPLING_IID))


@pytest.mark.parametrize("n,m,s,k,flags,count", [
    (300_000, 9, 30_000, 4_000, X.EXTRACT_GATHER_BUCKETS | X.EXTRACT_METHOD_DIRECT, 5),
    (5 << 20, 5, 1 << 20, 1000, 0, 4),                    # NTT, bucket tables
    (1 << 18, 8, 1 << 15, 1 << 13, X.EXTRACT_GATHER_PLAIN, 3),
    (1 << 18, 8, 1 << 15, 1 << 13, X.EXTRACT_METHOD_TENSOR, 1),
])
def test_host_many_blocks_match_the_oracle(n, m, s, k, flags, count):
    """extract_run_host_many on a stream of different blocks (pinned host
    buffers; the copies of neighbouring blocks overlap the work, the staging
    buffers alternate): every block's output equals the oracle's, and a
    second call on the same context (reusing streams, events and staging)
    gives the same."""
    seed = synth.uniform_bits(s + k - 1, 6)
    ins = [synth.bernoulli_bits(n, 0.5 + 0.05 * b, 40 + b) for b in range(count)]
    wants = [oracle.fast_extract(n, m, s, k, w, seed, 2) for w in ins]
    pins = [torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint32).view(np.int32)).pin_memory() for w in ins]
    with X.Extractor(n, m, s, k, seed, 2, flags) as ex:
        for _ in range(2):
            outs = [torch.empty(ex.out_words, dtype=torch.int32).pin_memory() for _ in range(count)]
            ex.run_host_many(pins, outs)
            for b in range(count):
                assert np.array_equal(outs[b].numpy().view(np.uint32), wants[b]), "block %d" % b
        with pytest.raises(X.ExtractError) as e:
            X.extract_run_host_many(ex.h, None, [pins[0]], [0])  # a null output buffer
        assert e.value.code == X.EXTRACT_EINVAL


def test_host_many_blocks_iid_law_and_independent_seeds():
    """extract_run_host_many with the paper's i.i.d. law (padded sub-blocks)
    and with one seed per sub-block: three blocks each, every output equal
    to the oracle's."""
    n, m, k = 250_000, 6, 2_000
    _, _, largest = oracle.iid_order(oracle.sampling_keys(n, 7), m, n, with_order=False)
    s = largest + 3
    seed = synth.uniform_bits(s + k - 1, 5)
    ins = [synth.bernoulli_bits(n, 0.6 + 0.1 * b, 60 + b) for b in range(3)]
    pins = [torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint32).view(np.int32)).pin_memory() for w in ins]
    with X.Extractor(n, m, s, k, seed, 7, X.EXTRACT_SAMPLING_IID) as ex:
        outs = ex.run_host_many(pins)
    for b in range(3):
        assert np.array_equal(outs[b], oracle.extract(n, m, s, k, ins[b], seed, 7, oracle.SAMPLING_IID)), b
    n, m, s, k = 1 << 20, 8, 1 << 17, 1 << 15
    seed = synth.uniform_bits((s + k - 1) * m, 42)
    ins = [synth.bernoulli_bits(n, 0.55 + 0.1 * b, 70 + b) for b in range(3)]
    pins = [torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint32).view(np.int32)).pin_memory() for w in ins]
    with X.Extractor(n, m, s, k, seed, 2, X.EXTRACT_SEED_PER_SUBBLOCK | X.EXTRACT_METHOD_NTT) as ex:
        outs = ex.run_host_many(pins)
    for b in range(3):
        assert np.array_equal(outs[b], oracle.fast_extract(n, m, s, k, ins[b], seed, 2, oracle.SEED_PER_SUBBLOCK)), b
