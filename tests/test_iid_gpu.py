"""The paper's i.i.d. sampling law on the GPU (EXTRACT_SAMPLING_IID): the
binomial sub-block sizes, the padded order, the abort, and the hashed bits,
all bit-exact against the CPU oracle, with both hashing methods."""
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


def _largest(n, m, key, flags=0):
    _, _, largest = oracle.iid_order(oracle.sampling_keys(n, key, flags), m, n, with_order=False)
    return largest


@pytest.mark.parametrize("n,m,key,flags", [
    (100_000, 7, 3, 0), (1 << 18, 64, 2, 0), (65537, 1, 5, 0), (3000, 100, 9, 0),
    (200_000, 33, 4, X.EXTRACT_KEY_BITS(14)), (1 << 17, 4096, 6, 0), (70_000, 20_000, 8, 0),
])
def test_sizes_and_order_match_the_oracle(n, m, key, flags):
    keys = oracle.sampling_keys(n, key, flags)
    largest = _largest(n, m, key, flags)
    s, k = largest + 5, 1
    sizes, order, _ = oracle.iid_order(keys, m, s)
    seed = synth.uniform_bits(s + k - 1, 1)
    with X.Extractor(n, m, s, k, seed, key, flags | X.EXTRACT_SAMPLING_IID | X.EXTRACT_METHOD_DIRECT) as ex:
        assert np.array_equal(ex.sizes(), sizes)
        assert np.array_equal(ex.read_perm(), order)


@pytest.mark.parametrize("n,m,k,slack,method,flags", [
    (100_000, 7, 3000, 0, X.EXTRACT_METHOD_DIRECT, 0),
    (100_000, 7, 3000, 17, X.EXTRACT_METHOD_NTT, 0),
    (1 << 18, 8, 1 << 13, 40, X.EXTRACT_METHOD_NTT, 0),
    (1 << 18, 8, 1 << 13, 40, X.EXTRACT_METHOD_DIRECT, 0),
    (50_000, 5, 777, 3, X.EXTRACT_METHOD_DIRECT, X.EXTRACT_SEED_PER_SUBBLOCK),
    (80_000, 16, 1000, 9, 0, X.EXTRACT_KEY_BITS(13)),
    (9_999, 3, 1, 0, X.EXTRACT_METHOD_DIRECT, 0),
])
def test_hash_matches_the_oracle(n, m, k, slack, method, flags):
    key = 21
    s = _largest(n, m, key, flags) + slack
    L = (s + k - 1) * (m if flags & X.EXTRACT_SEED_PER_SUBBLOCK else 1)
    in_w = synth.bernoulli_bits(n, 0.7, 31)
    seed = synth.uniform_bits(L, 32)
    want = oracle.extract(n, m, s, k, in_w, seed, key, flags | oracle.SAMPLING_IID)
    with X.Extractor(n, m, s, k, seed, key, flags | method | X.EXTRACT_SAMPLING_IID) as ex:
        if method == X.EXTRACT_METHOD_NTT:
            assert ex.describe().startswith("ntt")
        got = _host(ex.run(_dev(in_w)))
        again = _host(ex.run(_dev(in_w)))
    assert np.array_equal(got, want)
    assert np.array_equal(again, want)


def test_abort_when_a_sub_block_exceeds_the_limit():
    n, m, key = 100_000, 9, 12
    largest = _largest(n, m, key)
    seed = synth.uniform_bits(largest + 50, 1)
    with pytest.raises(X.ExtractError) as e:
        X.extract_create(n, m, largest - 1, 10, seed, key, X.EXTRACT_SAMPLING_IID)
    assert e.value.code == X.EXTRACT_EABORT and "abort" in str(e.value)
    with X.Extractor(n, m, largest, 10, seed, key, X.EXTRACT_SAMPLING_IID) as ex:  # at the limit it runs
        assert int(ex.sizes().max()) == largest


def test_rejections():
    seed = np.zeros(4096, dtype=np.uint32)
    for n, m, s, k, fl in [
        (1 << 32, 4, 1 << 30, 8, 0),                          # n must be < 2^32
        (4096, 1 << 17, 64, 8, 0),                            # m <= 2^16
        (4096, 4, 2000, 8, X.EXTRACT_IDENTITY_PERM),          # no identity order
    ]:
        with pytest.raises(X.ExtractError) as e:
            X.extract_create(n, m, s, k, seed, 1, fl | X.EXTRACT_SAMPLING_IID)
        assert e.value.code == X.EXTRACT_EINVAL
    job = {"n": 4096, "m": 2, "s": 2100, "k": 8, "key": 1,
           "flags": X.EXTRACT_SAMPLING_IID | X.EXTRACT_IDENTITY_PERM, "seed": synth.uniform_bits(2107, 1)}
    with pytest.raises(X.ExtractError) as e:
        X.Batch([job])
    assert e.value.code == X.EXTRACT_EINVAL


def _iid_jobs():
    """i.i.d.-law jobs (both methods) mixed with sorted-order jobs."""
    jobs = []
    for i, (n, m, k, slack, fl) in enumerate([
            (100_000, 7, 3000, 3, X.EXTRACT_SAMPLING_IID),
            (1 << 18, 8, 1 << 13, 40, X.EXTRACT_SAMPLING_IID),
            (50_000, 5, 777, 0, X.EXTRACT_SAMPLING_IID | X.EXTRACT_SEED_PER_SUBBLOCK),
            (1 << 16, 4, 1 << 12, 0, 0),
            (70_000, 20_000, 2, 1, X.EXTRACT_SAMPLING_IID),
            (1 << 20, 2, 1 << 18, 100, X.EXTRACT_SAMPLING_IID)]):
        key = 40 + i
        if fl & X.EXTRACT_SAMPLING_IID:
            s = _largest(n, m, key) + slack
        else:
            s = n // m
        L = (s + k - 1) * (m if fl & X.EXTRACT_SEED_PER_SUBBLOCK else 1)
        jobs.append({"n": n, "m": m, "s": s, "k": k, "key": key, "flags": fl,
                     "seed": synth.uniform_bits(L, 50 + i), "in": synth.bernoulli_bits(n, 0.6, 60 + i)})
    return jobs


def _out(j, fill=-1):
    return torch.full(((j["m"] * j["k"] + 31) // 32,), fill, dtype=torch.int32, device="cuda")


def test_batch_with_iid_jobs_matches_single_contexts_and_the_oracle():
    jobs = _iid_jobs()
    d_in = [_dev(j["in"]) for j in jobs]
    with X.Batch(jobs) as b:
        outs = [_out(j) for j in jobs]
        b.run(d_in, outs)
        seq = [_out(j, 7) for j in jobs]
        b.run_sequential(d_in, seq)
        torch.cuda.synchronize()
    for i, (j, d) in enumerate(zip(jobs, d_in)):
        with X.Extractor(j["n"], j["m"], j["s"], j["k"], j["seed"], j["key"], j["flags"]) as ex:
            want = _host(ex.run(d))
        assert np.array_equal(_host(outs[i]), want), "job %d" % i
        assert np.array_equal(_host(seq[i]), want), "sequential job %d" % i
    for i in (0, 2, 4):
        j = jobs[i]
        fl = oracle.SAMPLING_IID | (oracle.SEED_PER_SUBBLOCK if j["flags"] & X.EXTRACT_SEED_PER_SUBBLOCK else 0)
        want = oracle.extract(j["n"], j["m"], j["s"], j["k"], j["in"], j["seed"], j["key"], fl)
        assert np.array_equal(_host(outs[i]), want), "job %d vs oracle" % i


def test_batch_aborts_naming_the_job():
    jobs = _iid_jobs()[:2]
    jobs[1] = dict(jobs[1])
    jobs[1]["s"] -= 41  # one below its largest sub-block
    jobs[1]["seed"] = synth.uniform_bits(jobs[1]["s"] + jobs[1]["k"] - 1, 5)
    with pytest.raises(X.ExtractError) as e:
        X.Batch(jobs)
    assert e.value.code == X.EXTRACT_EABORT and "job 1" in str(e.value)


def test_server_serves_iid_jobs_and_fails_an_aborting_one():
    jobs = _iid_jobs()
    bad = dict(jobs[0])
    bad["s"] = _largest(bad["n"], bad["m"], bad["key"]) - 1
    bad["seed"] = synth.uniform_bits(bad["s"] + bad["k"] - 1, 9)
    d_in = [_dev(j["in"]) for j in jobs]
    outs = [_out(j) for j in jobs]
    with X.Server(8 << 30, max_slots=8, wave_us=500) as srv:
        tickets = [srv.submit(j, d, o) for j, d, o in zip(jobs, d_in, outs)]
        bt = srv.submit(bad, _dev(bad["in"]), _out(bad))
        for t in tickets:
            srv.wait(t)
        with pytest.raises(X.ExtractError) as e:
            srv.wait(bt)
        assert e.value.code == X.EXTRACT_EABORT
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 1
    for i, (j, d) in enumerate(zip(jobs, d_in)):
        with X.Extractor(j["n"], j["m"], j["s"], j["k"], j["seed"], j["key"], j["flags"]) as ex:
            assert np.array_equal(_host(outs[i]), _host(ex.run(d))), "job %d" % i


def test_qrng_shaped_block_with_the_eq7_limit():
    """n = 2^24, m = 64, s = Eq. 7's limit at eps = 1e-8: the NTT and direct
    methods agree everywhere and sampled rows match the oracle."""
    n, m, k, key = 1 << 24, 64, 1 << 15, 2
    s = X.extract_block_limit(n, m, 1e-8, 1.0 / m)
    assert s == oracle.block_limit(n, m, 1e-8, 1.0 / m)
    in_w = synth.bernoulli_bits(n, 0.6, 1)
    seed = synth.uniform_bits(s + k - 1, 3)
    d_in = _dev(in_w)
    with X.Extractor(n, m, s, k, seed, key, X.EXTRACT_SAMPLING_IID | X.EXTRACT_METHOD_NTT) as a, \
            X.Extractor(n, m, s, k, seed, key, X.EXTRACT_SAMPLING_IID | X.EXTRACT_METHOD_DIRECT) as b:
        ga, gb = _host(a.run(d_in)), _host(b.run(d_in))
        sizes = a.sizes()
    assert np.array_equal(ga, gb)
    keys = oracle.sampling_keys(n, key)
    want_sizes, order, _ = oracle.iid_order(keys, m, s)
    assert np.array_equal(sizes, want_sizes) and int(sizes.sum()) == n
    got = oracle.bits_of(ga, m * k)
    rng = np.random.default_rng(4)
    for j in (0, 17, m - 1):
        A = oracle.subblock_padded(in_w, order[j * s:(j + 1) * s])
        for i in np.concatenate([[0, 1, k - 1], rng.choice(k, 24, replace=False)]):
            assert got[j * k + i] == oracle.toeplitz_bit(seed, s, A, int(i)), (j, i)
