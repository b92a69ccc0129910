"""extract_run_static: the run for callers that may not allocate device
memory (their memory is budgeted and handed out by someone else, or they
cannot afford the device-wide synchronisation cudaMalloc/cudaFree can cause).

It must give the same bits as the ordinary entry point, extract_run, on two
calls in a row that share the library's one static scratch array, including
with a padded order of the paper's i.i.d. law and with an input long enough
for the gather's two input windows, and a further call must leave the
device's free memory unchanged.  This file is collected last on purpose, so
that a failure here stops a -x run only after every other test has run."""
import numpy as np
import pytest

from paper_2308_02856_gb300 import build as pkg_build
from paper_2308_02856_gb300 import extract as X
from paper_2308_02856_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(words):
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def _iid_limit(n, m, key):
    """A block size limit just above the largest i.i.d.-law sub-block."""
    with X.Extractor(n, m, n, 1, synth.uniform_bits(n, 1), key, X.EXTRACT_SAMPLING_IID) as ex:
        return int(ex.sizes().max()) + 5


@pytest.mark.parametrize("n,m,s,k,flags", [
    (1 << 18, 8, 1 << 15, 1 << 13, 0),             # sampled sub-blocks
    (200_000, 37, 5000, 3001, 0),                   # ragged rows, words and sub-block tiles
    (1 << 20, 1, 1 << 20, 1 << 16, X.EXTRACT_IDENTITY_PERM),  # direct whole-block, no order
    ((1 << 30) - 5, 64, 1 << 20, 1000, 0),          # the gather in two 2^29-bit input windows
    (300_000, 7, None, 2000, X.EXTRACT_SAMPLING_IID),  # the i.i.d. law's padded order (m*s > n)
])
def test_static_run_matches_extract_run_twice(n, m, s, k, flags):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg_build.build()
    if s is None:
        s = _iid_limit(n, m, 2)
        assert m * s > n
    seed = synth.uniform_bits(s + k - 1, 3)
    ins = [synth.bernoulli_bits(n, 0.7, 1), synth.bernoulli_bits(n, 0.55, 2)]
    with X.Extractor(n, m, s, k, seed, 2, flags) as ex:
        want = [_host(ex.run(_dev(w))) for w in ins]
        perm = None if flags & X.EXTRACT_IDENTITY_PERM else _dev(ex.read_perm())
    d_seed = _dev(seed)
    d_ins = [_dev(w) for w in ins]
    outs = [torch.full(((m * k + 31) // 32,), -1, dtype=torch.int32, device="cuda") for _ in ins]
    for d, out, ref in zip(d_ins, outs, want):  # two calls in a row on the shared static scratch
        X.extract_run_static(n, m, s, k, perm, d_seed, d, out)
        torch.cuda.synchronize()
        assert np.array_equal(_host(out), ref)
    # a further call allocates nothing: free device memory is unchanged
    # (any cudaMalloc would show in steps of at least 2 MiB)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    X.extract_run_static(n, m, s, k, perm, d_seed, d_ins[0], outs[1])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(_host(outs[1]), want[0])


def test_static_run_rejects_shapes_beyond_the_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = s = 1 << 28  # 2^23 words of sub-block data: over the 4 Mi-word array
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(X.ExtractError) as e:
        X.extract_run_static(n, 1, s, 64, None, d, d, d)
    assert e.value.code == X.EXTRACT_EINVAL
    assert "static limit" in str(e.value)
