"""The NTT's column pass A on the tensor cores (transform lengths 2^16, 2^17
and 2^18, i.e. 32, 64 and 128 rows per column): the column DFTs of the
piece bits are an exact integer product with three 11-bit f16 slices of the
DFT matrix (f32 sums below 2^18).  Bit-exact against the oracle for every
number of nonzero rows per piece (K steps of 16 rows from 1 to R1 / 16),
ragged pieces and seed windows, one seed per sub-block and forced splits
(the word-packed oracle); the plan says which pass A it runs."""
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


def _run(n, m, s, k, flags, in_w, seed):
    with X.Extractor(n, m, s, k, seed, 2, flags | X.EXTRACT_METHOD_NTT) as ex:
        desc = ex.describe()
        d_in = torch.from_numpy(np.ascontiguousarray(in_w).view(np.int32)).cuda()
        out = ex.run(d_in).cpu().numpy().view(np.uint32)
        ex.status()  # no tensor-core wait gave up
    return out, desc


def _N(desc):
    return int(desc.split("N=")[1].split(" ")[0])


# (n, m, s, k, l): N = 2^16, 2^17, 2^18 with pieces of 1 .. R1/16 K steps of
# 16 rows (a piece of len bits has data in rows below len / 2048); l forces
# 2^l pieces per sub-block, None leaves the choice to the library
CASES = [
    (1 << 18, 8, 1 << 15, 1 << 13, None),       # N = 2^16, 32768 bits: 1 K step
    (300_000, 7, 40_001, 20_000, None),         # N = 2^16, 40001 bits: 2 K steps (ragged)
    (3 * 70_001, 3, 70_001, 9_999, 0),          # N = 2^17, 70001 bits: 3 K steps
    (4 * 120_000, 4, 120_000, 5_000, 0),        # N = 2^17, 120000 bits: 4 K steps (all)
    (2 * (1 << 17), 2, 1 << 17, 104_858, None),  # N = 2^18, 4 K steps
    (3 * 150_001, 3, 150_001, 104_858, None),   # N = 2^18, 5 K steps
    (2 * 250_000, 2, 250_000, 12_000, 0),       # N = 2^18, 8 K steps (all)
    (1 << 21, 2, 1 << 20, 104_858, 3),          # the QKD sub-block shape in 8 pieces: N = 2^18
    (1 << 21, 2, 1 << 20, 104_858, None),       # ... in the library's 7 pieces of 149824 bits
    # more pieces than 9 per 128-column block: CTAs take several pieces, so the
    # accumulator buffers are reused (each row group's phase parities)
    (1 << 20, 32, 1 << 15, 1 << 13, None),      # N = 2^16, 32 pieces
    (20 * 70_001, 20, 70_001, 9_999, 0),        # N = 2^17, 20 pieces
    (48 * 150_001, 48, 150_001, 10_000, 0),     # N = 2^18, 48 pieces
]


@pytest.mark.parametrize("n,m,s,k,split", CASES)
def test_tensor_core_pass_a_matches_oracle(n, m, s, k, split):
    in_w = synth.bernoulli_bits(n, 0.7, 81)
    seed = synth.uniform_bits(s + k - 1, 82)
    got, desc = _run(n, m, s, k, 0 if split is None else X.EXTRACT_NTT_SPLIT(split), in_w, seed)
    assert _N(desc) in (1 << 16, 1 << 17, 1 << 18), desc
    assert "column pass A on the tensor cores" in desc, desc
    want = oracle.fast_extract(n, m, s, k, in_w, seed, 2)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, "%d of %d words differ, first %s" % (bad.size, want.size, bad[:5])


def test_tensor_core_pass_a_independent_seeds():
    """Seed windows through the tensor-core pass A as well (one seed per
    sub-block, windows transformed in the run)."""
    n, m, s, k = 1 << 20, 8, 1 << 17, 1 << 15
    in_w = synth.bernoulli_bits(n, 0.6, 83)
    seed = synth.uniform_bits((s + k - 1) * m, 84)
    got, desc = _run(n, m, s, k, X.EXTRACT_SEED_PER_SUBBLOCK, in_w, seed)
    assert "column pass A on the tensor cores" in desc and "one seed per sub-block" in desc, desc
    assert np.array_equal(got, oracle.fast_extract(n, m, s, k, in_w, seed, 2, oracle.SEED_PER_SUBBLOCK))


def test_butterfly_pass_a_outside_the_tensor_core_lengths():
    """N = 2^20 keeps the butterfly column kernels."""
    n, m, s, k = 1 << 21, 2, 1 << 20, 1 << 19
    in_w = synth.bernoulli_bits(n, 0.6, 85)
    seed = synth.uniform_bits(s + k - 1, 86)
    got, desc = _run(n, m, s, k, 0, in_w, seed)
    assert _N(desc) == 1 << 20 and "column pass A by butterflies" in desc, desc
    with X.Extractor(n, m, s, k, seed, 2, X.EXTRACT_METHOD_DIRECT) as ex:
        d_in = torch.from_numpy(in_w.view(np.int32)).cuda()
        want = ex.run(d_in).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)
