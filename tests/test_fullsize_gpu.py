"""Full-size blocks in the launch configuration bench.py times.

* The sampled order is checked completely: the oracle computes all n labels
  and checks that the GPU order increases strictly in (label, position)
  order with every entry < n, which makes it a bijection and the unique
  stable argsort.
* The gather is checked on whole sub-blocks (every bit, as stored for the
  hash) and the hash on sampled outputs: the oracle selects sub-blocks by
  rank from its own labels and computes sampled rows one bit at a time.
"""
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


def _full_size_case(n, m, s, k, p, rows_per_block, blocks):
    in_w = synth.bernoulli_bits(n, p, 1)
    seed = synth.uniform_bits(s + k - 1, 3)
    with X.Extractor(n, m, s, k, seed, 2) as ex:
        d_in = torch.from_numpy(in_w.view(np.int32)).cuda()
        out = ex.run(d_in)
        got = oracle.bits_of(out.cpu().numpy().view(np.uint32), m * k)
        stored = {j: oracle.bits_of(ex.read_subblock(j), s)[::-1] for j in blocks}  # stored reversed
        del d_in, out
        perm = ex.read_perm()
    keys = oracle.sampling_keys(n, 2)
    assert oracle.check_order(keys, perm) == -1
    del perm
    rng = np.random.default_rng(1)
    for j in blocks:
        pos = oracle.perm_range(keys, j * s, s)
        A = oracle.subblock(in_w, pos)
        assert np.array_equal(stored[j], A), "gathered sub-block %d" % j
        rows = np.unique(np.concatenate([np.arange(16), np.arange(k - 16, k),
                                         rng.choice(k, rows_per_block, replace=False)]))
        want = np.array([oracle.toeplitz_bit(seed, s, A, int(i)) for i in rows], dtype=np.uint8)
        assert np.array_equal(got[j * k + rows], want), "sub-block %d" % j


def test_qrng_shaped_block_n2e30():
    """n = 2^30 Bernoulli(0.6), m = 1024 sub-blocks of s = 2^20, k = 2^19."""
    _full_size_case(1 << 30, 1024, 1 << 20, 1 << 19, 0.6, 48, [0, 1, 511, 1023])


def test_qkd_shaped_block_n2e32():
    """n = 2^32 Bernoulli(0.9), m = 4096 sub-blocks of s = 2^20, k = 104858
    (k mod 32 = 26: every sub-block's output starts at an unaligned bit)."""
    _full_size_case(1 << 32, 4096, 1 << 20, 104858, 0.9, 32, [0, 1, 2047, 4095])
