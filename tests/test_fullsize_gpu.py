"""Full-size blocks in the launch configuration bench.py times.

* The sampled order is checked completely: the oracle computes all n labels
  and checks that the GPU order increases strictly in (label, position)
  order with every entry < n, which makes it a bijection and the unique
  stable argsort.
* Whole sub-blocks, every bit: the gathered sub-block as stored for the hash,
  and every output row of its hash, against the word-packed oracle.  The
  sub-blocks are chosen across many NTT launch groups (the first and last
  sub-block of each chosen group, and a few in between), from groups run on
  both of the hash's two lanes.
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


def _group_blocks(G, m, groups, extra):
    """The first, last and two inner sub-blocks of each launch group in
    ``groups`` (groups of G sub-blocks alternate between two lanes; negative
    indices count from the last group), plus ``extra``."""
    ng = (m + G - 1) // G
    groups = sorted({g % ng for g in groups})
    assert {g % 2 for g in groups} == {0, 1}
    offsets = sorted({0, G // 3, (2 * G) // 3, G - 1})
    blocks = [min(m - 1, G * g + r) for g in groups for r in offsets] + [j for j in extra if j < m]
    return sorted(set(blocks))


def _full_size_case(n, m, s, k, p, groups, extra, plan_has, nblocks):
    in_w = synth.bernoulli_bits(n, p, 1)
    seed = synth.uniform_bits(s + k - 1, 3)
    with X.Extractor(n, m, s, k, seed, 2) as ex:
        plan = ex.describe()
        for frag in plan_has:
            assert frag in plan, plan
        G = int(plan.split(" sub-blocks per launch group")[0].split(",")[-1])
        blocks = _group_blocks(G, m, groups, extra)
        assert len(blocks) >= nblocks, blocks
        d_in = torch.from_numpy(in_w.view(np.int32)).cuda()
        out = ex.run(d_in)
        got = oracle.bits_of(out.cpu().numpy().view(np.uint32), m * k)
        stored = {j: oracle.bits_of(ex.read_subblock(j), s)[::-1] for j in blocks}  # stored reversed
        del d_in, out
        perm = ex.read_perm()
    keys = oracle.sampling_keys(n, 2)
    assert oracle.check_order(keys, perm) == -1
    del perm
    pos = oracle.perm_ranges(keys, [(j * s, s) for j in blocks])
    del keys
    for t, j in enumerate(blocks):
        A = oracle.subblock(in_w, pos[t * s:(t + 1) * s])
        assert np.array_equal(stored[j], A), "gathered sub-block %d" % j
    K = oracle.fast_window(in_w, pos, s, k, seed, 0, blocks, 0, k, seed_len_bits=s + k - 1)
    for t, j in enumerate(blocks):
        bad = np.flatnonzero(got[j * k:(j + 1) * k] != K[t])
        assert bad.size == 0, "sub-block %d: %d of %d rows differ, first %s" % (j, bad.size, k, bad[:5])


def test_qrng_shaped_block_n2e30():
    """n = 2^30 Bernoulli(0.6), m = 1024 sub-blocks of s = 2^20, k = 2^19:
    P = 2 pieces, N = 2^20, launch groups on two lanes; every row of at
    least 32 whole sub-blocks from every launch group."""
    _full_size_case(1 << 30, 1024, 1 << 20, 1 << 19, 0.6, (0, 1, 2, 3, 4, 5, 30, 31, 32, 33, -4, -3, -2, -1),
                    (7, 8, 1016, 1017), ("ntt: N=1048576", "P=2 ", "gather=buckets (2^16-bit"), 32)


def test_qkd_shaped_block_n2e32():
    """n = 2^32 Bernoulli(0.9), m = 4096 sub-blocks of s = 2^20, k = 104858
    (k mod 32 = 26: every sub-block's output starts at an unaligned bit):
    P = 7 pieces, N = 2^18, launch groups on two lanes (the last one
    partial), bucket tables over 2^18-bit chunks; every row of at least 16
    whole sub-blocks."""
    _full_size_case(1 << 32, 4096, 1 << 20, 104858, 0.9, (0, 1, 100, 101, -2, -1), (7, 1603, 2000, 3000, 3228),
                    ("ntt: N=262144", "P=7 ", "gather=buckets (2^18-bit"), 16)


@pytest.mark.parametrize("n,m,s,k", [
    (1 << 32, 4096, 1 << 20, 104858),   # P = 7, N = 2^18: tensor-core pass A, bulk-copied rows in pass B
    (1 << 30, 1024, 1 << 20, 1 << 19),  # P = 2, N = 2^20
])
def test_repeated_runs_are_bit_identical(n, m, s, k):
    """Races show up as outputs that change from run to run on the same input
    (a rare one slips past sampled parity checks): twelve hashes of one
    gathered block and three whole runs must all give the same words."""
    import hashlib
    in_w = synth.bernoulli_bits_device(n, 0.8, 5)
    seed = synth.uniform_bits(s + k - 1, 6)
    with X.Extractor(n, m, s, k, seed, 2) as ex:
        out = ex.new_output()
        digests = set()
        for _ in range(3):
            ex.run(in_w, out)
            digests.add(hashlib.sha256(out.cpu().numpy().tobytes()).hexdigest())
        for _ in range(12):
            ex.hash(out)
            digests.add(hashlib.sha256(out.cpu().numpy().tobytes()).hexdigest())
        ex.status()
    assert len(digests) == 1, "%d different outputs from 15 runs on one input" % len(digests)
