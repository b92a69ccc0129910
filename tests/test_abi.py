"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every symbol include/extract.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2308_02856_gb300 import build as pkg_build
from paper_2308_02856_gb300 import extract as X

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(extract_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return X.load()


def test_binding_constants_match_the_header():
    """Every plain numeric #define EXTRACT_* in include/*.h has the same value
    in the Python binding (return codes, create and batch flags)."""
    seen = 0
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for name, val in re.findall(r"^#define\s+(EXTRACT_[A-Z0-9_]+)\s+\(?\s*(-?(?:0x[0-9a-fA-F]+|\d+))u?\s*\)?\s*$",
                                    text, flags=re.M):
            assert hasattr(X, name), name
            assert getattr(X, name) == int(val, 0), name
            seen += 1
    assert seen >= 20


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("extract_create", "extract_run", "extract_destroy", "extract_last_error"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    d = _declared()
    assert d, "no declarations parsed"
    for name in d:
        assert hasattr(lib, name), name
    assert sorted(X.EXPORTED) == sorted(n for n in d if n in X.EXPORTED)
    missing = [n for n in d if n not in X.EXPORTED]
    assert not missing, "binding lacks %s" % missing


def test_library_is_sm103a_only():
    log = open(os.path.join(ROOT, "paper_2308_02856_gb300", "_build", "ptxas.log")).read()
    assert "sm_103a" in log
    for bad in ("sm_100", "sm_90", "sm_80"):
        assert "'%s'" % bad not in log


@pytest.mark.parametrize("n,m,s,k", [
    (100, 2, 60, 10),     # m*s > n
    (100, 1, 10, 11),     # k > s
    (100, 0, 10, 1),      # m = 0
    (100, 1, 10, 0),      # k = 0
    (1 << 33, 1, 10, 1),  # n > 2^32
])
def test_create_rejects_bad_shapes_without_touching_the_gpu(lib, n, m, s, k):
    seed = np.zeros(64, dtype=np.uint32)
    with pytest.raises(X.ExtractError) as e:
        X.extract_create(n, m, s, k, seed, 1)
    assert e.value.code == X.EXTRACT_EINVAL
    assert X.extract_last_error()


def test_create_rejects_null_and_unknown_flags(lib):
    h = ctypes.c_void_p()
    assert lib.extract_create(ctypes.byref(h), 64, 1, 64, 8, None, 1, 0) == X.EXTRACT_EINVAL
    seed = np.zeros(8, dtype=np.uint32)
    assert lib.extract_create(ctypes.byref(h), 64, 1, 64, 8, seed.ctypes.data, 1, 0x200000) == X.EXTRACT_EINVAL
    assert lib.extract_create(None, 64, 1, 64, 8, seed.ctypes.data, 1, 0) == X.EXTRACT_EINVAL


def test_calls_on_a_null_context_fail_cleanly(lib):
    assert lib.extract_run(None, None, None, None) == X.EXTRACT_EINVAL
    assert lib.extract_hash(None, None, None) == X.EXTRACT_EINVAL
    assert lib.extract_destroy(None) == X.EXTRACT_OK
    buf = ctypes.create_string_buffer(16)
    assert lib.extract_describe(None, buf, 16) == X.EXTRACT_EINVAL


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(X, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(X, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        X.load()


def test_block_limit_matches_the_oracle_and_rejects_bad_arguments():
    """extract_block_limit is host code: it runs without a GPU.  The library's
    Eq. 7 and the oracle's give the same limit on a grid of parameters."""
    for N in (1000, 10**6, 2**24, 2**30, 10**9, 2**32 - 1):
        for m in (1, 2, 17, 64, 1024, 4096):
            for eps in (1e-3, 1e-8, 1e-12):
                p = 1.0 / m if m > 1 else 0.5
                assert X.extract_block_limit(N, m, eps, p) == oracle.block_limit(N, m, eps, p), (N, m, eps)
    for args in ((0, 4, 1e-8, 0.25), (100, 0, 1e-8, 0.25), (100, 4, 0.0, 0.25), (100, 4, 1e-8, 1.0),
                 (100, 4, 1e-8, 0.0)):
        with pytest.raises(X.ExtractError) as e:
            X.extract_block_limit(*args)
        assert e.value.code == X.EXTRACT_EINVAL
