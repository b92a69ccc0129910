"""Forms of the path that only large inputs reach, checked on whole
sub-blocks against the oracle:

* the window-major gather (inputs of more than two 2^29-bit windows without
  bucket tables), forced with EXTRACT_GATHER_PLAIN;
* the plain gather in two 2^29-bit input windows (inputs of 2^29 .. 2^30
  bits), forced the same way, under both hashing methods;
* a served job of the serving workload's largest shape (n = 2^30,
  s = 2^20), in a mix with small jobs;
* direct whole-block Toeplitz hashing of n = 2^24 bits to k = 2^23 (m = 1,
  identity order: the "traditional" method of Sec. IV.C at the comparison
  size of the QRNG-shaped block), every bit of 2^17 whole rows.
"""
import time

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


def _check_rows(got_bits, in_w, pos, blocks, s, k, seed):
    K = oracle.fast_window(in_w, pos, s, k, seed, 0, blocks, 0, k, seed_len_bits=s + k - 1)
    for t, j in enumerate(blocks):
        bad = np.flatnonzero(got_bits[j * k:(j + 1) * k] != K[t])
        assert bad.size == 0, "sub-block %d: %d of %d rows differ, first %s" % (j, bad.size, k, bad[:5])


def _large_case(n, m, s, k, flags, gather_frag, stored_blocks, row_blocks, key):
    in_w = synth.bernoulli_bits(n, 0.7, 5)
    seed = synth.uniform_bits(s + k - 1, 6)
    with X.Extractor(n, m, s, k, seed, key, flags | X.EXTRACT_GATHER_PLAIN) as ex:
        plan = ex.describe()
        assert gather_frag in plan, plan
        out = ex.run(_dev(in_w))
        got = oracle.bits_of(_host(out), m * k)
        stored = {j: oracle.bits_of(ex.read_subblock(j), s)[::-1] for j in stored_blocks}
    keys = oracle.sampling_keys(n, key)
    blocks = sorted(set(stored_blocks) | set(row_blocks))
    pos = oracle.perm_ranges(keys, [(j * s, s) for j in blocks])
    del keys
    at = {j: t for t, j in enumerate(blocks)}
    for j in stored_blocks:
        A = oracle.subblock(in_w, pos[at[j] * s:(at[j] + 1) * s])
        assert np.array_equal(stored[j], A), "gathered sub-block %d" % j
    _check_rows(got, in_w, pos, blocks, s, k, seed)


def test_window_major_gather():
    """n = 2^31 + 777 (five 2^29-bit windows, the last ragged), s = 2^20 + 3,
    m*s far below n: the order re-laid window by window."""
    _large_case((1 << 31) + 777, 40, (1 << 20) + 3, 4097, 0, "gather=windows (5 input windows)",
                [0, 1, 19, 39], list(range(40)), 11)


@pytest.mark.parametrize("method", [X.EXTRACT_METHOD_DIRECT, X.EXTRACT_METHOD_NTT])
def test_two_window_plain_gather(method):
    """n = 2^30 - 12345: two passes of the plain gather over 2^29-bit input
    windows, the second ORing its bits into the words the first stored."""
    m = 1000
    _large_case((1 << 30) - 12345, m, 1 << 20, 3000, method, "gather=plain", [0, 500, m - 1],
                [0, 1, 2, 250, 499, 500, 501, 750, 997, 998, m - 1], 12)


def test_served_job_of_the_largest_serving_shape():
    """One job of n = 2^30, m = 1024, s = 2^20, k = 0.3 s among small jobs
    arriving while it runs: every row of 24 whole sub-blocks of the large job
    against the word-packed oracle, the small jobs' whole outputs against the
    bit-loop oracle."""
    n, m, s, k = 1 << 30, 1024, 1 << 20, 314572
    big = {"n": n, "m": m, "s": s, "k": k, "key": 77, "seed": synth.uniform_bits(s + k - 1, 78)}
    big_in = synth.bernoulli_bits(n, 0.7, 79)
    shapes = synth.job_shapes(6, 91, 2 ** 14, 2 ** 18, s_set=(1 << 12, 1 << 14))
    small, small_in = [], []
    for j in shapes:
        j = dict(j)
        j["seed"] = synth.uniform_bits(j["s"] + j["k"] - 1, j["seed_seed"])
        small.append(j)
        small_in.append(synth.bernoulli_bits(j["n"], j["p"], j["in_seed"]))
    jobs = [big] + small
    ins = [_dev(big_in)] + [_dev(w) for w in small_in]
    outs = [torch.full(((j["m"] * j["k"] + 31) // 32,), -1, dtype=torch.int32, device="cuda") for j in jobs]
    with X.Server(40 << 30, max_slots=8, wave_us=500) as srv:
        tickets = [srv.submit(jobs[0], ins[0], outs[0])]
        time.sleep(0.005)
        for j, d, o in zip(jobs[1:], ins[1:], outs[1:]):
            tickets.append(srv.submit(j, d, o))
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for j, w, o in zip(small, small_in, outs[1:]):
        want = oracle.extract(j["n"], j["m"], j["s"], j["k"], w, j["seed"], j["key"])
        assert np.array_equal(_host(o), want)
    got = oracle.bits_of(_host(outs[0]), m * k)
    blocks = [0, 1, 2, 15, 16, 17, 31, 32, 100, 255, 256, 511, 512, 513, 700, 767, 768, 900, 1000, 1007, 1008,
              1020, 1022, 1023]
    keys = oracle.sampling_keys(n, 77)
    pos = oracle.perm_ranges(keys, [(j * s, s) for j in blocks])
    del keys
    _check_rows(got, big_in, pos, blocks, s, k, big["seed"])


def test_direct_whole_block_n2e24_k2e23():
    """m = 1, identity order: K = T . A for the whole 2^24-bit block, T of
    2^23 x 2^24 (past the NTT method's range, so the direct kernel); every
    bit of the first and last 2^15 rows and of 64 runs of 1024 rows drawn
    at random, and the plain per-block path gives the same bits."""
    n = s = 1 << 24
    k = 1 << 23
    in_w = synth.bernoulli_bits(n, 0.6, 1)
    seed = synth.uniform_bits(n + k - 1, 3)
    with X.Extractor(n, 1, s, k, seed, 0, X.EXTRACT_IDENTITY_PERM) as ex:
        assert not ex.describe().startswith("ntt")
        d = _dev(in_w)
        tiled = _host(ex.run(d))
        plain = _host(ex.run_plain(d))
    assert np.array_equal(tiled, plain)
    got = oracle.bits_of(tiled, k)
    rng = np.random.default_rng(8)
    starts = [0, k - (1 << 15)] + sorted(int(x) * 1024 for x in rng.choice(k // 1024 - 32, 64, replace=False) + 32)
    for r0 in starts:  # runs of whole rows: 2^15 at each end, 64 runs of 1024 drawn at random
        cnt = (1 << 15) if r0 in (0, k - (1 << 15)) else 1024
        K = oracle.fast_window(in_w, np.arange(s, dtype=np.uint32), s, k, seed, 0, [0], r0, cnt,
                               seed_len_bits=s + k - 1)[0]
        bad = np.flatnonzero(got[r0:r0 + cnt] != K)
        assert bad.size == 0, "rows from %d: %d of %d differ, first %s" % (r0, bad.size, cnt, r0 + bad[:5])
