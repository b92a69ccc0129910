"""Thin ctypes binding of libextract.so (include/extract.h), same names.

Argument marshalling only: every step of the path runs in the CUDA library.
Device buffers are passed as torch CUDA tensors of 32-bit words (int32 or
uint32 dtype; the bits are what count) or as raw integer device addresses.
There is no CPU fallback: if the library is not built, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libextract.so")

EXTRACT_OK = 0
EXTRACT_EINVAL = -1
EXTRACT_ENOMEM = -2
EXTRACT_ECUDA = -3
EXTRACT_ETIMEDOUT = -4
EXTRACT_EBUDGET = -5
EXTRACT_EBUSY = -6
EXTRACT_EINTERNAL = -7
EXTRACT_EABORT = -8

EXTRACT_SEED_PER_SUBBLOCK = 0x1
EXTRACT_IDENTITY_PERM = 0x2
EXTRACT_METHOD_DIRECT = 0x4
EXTRACT_METHOD_NTT = 0x8
EXTRACT_SAMPLING_IID = 0x10
EXTRACT_GATHER_PLAIN = 0x20
EXTRACT_GATHER_BUCKETS = 0x40
EXTRACT_GATHER_WIDE_CHUNKS = 0x80
EXTRACT_METHOD_TENSOR = 0x100000
EXTRACT_TC_TEST_STALL = 0x10000000
NO_POS = 0xFFFFFFFF  # padding slot of the i.i.d. law's order


def EXTRACT_KEY_BITS(b: int) -> int:
    return (int(b) & 0x3F) << 8


def EXTRACT_TC_CHUNK(l: int) -> int:
    """Tensor-core method: 2^l K blocks of 128 per parity read-back (l = 0 .. 14)."""
    return ((int(l) + 1) & 0xF) << 24


def EXTRACT_NTT_SPLIT(l: int) -> int:
    """NTT method: 2^l pieces per sub-block (l = 0 .. 4) instead of the automatic split."""
    return ((int(l) + 1) & 0x7) << 16


# Every symbol include/extract.h declares (checked by the CPU test suite).
EXPORTED = [
    "extract_create", "extract_run", "extract_run_host", "extract_run_host_many", "extract_gather", "extract_hash",
    "extract_run_plain",
    "extract_read_perm", "extract_read_subblock", "extract_describe", "extract_destroy",
    "extract_subblock_sizes", "extract_block_limit", "extract_gather_bytes", "extract_status",
    "extract_last_error", "extract_run_static",
    "extract_batch_create", "extract_batch_run", "extract_batch_run_sequential", "extract_batch_describe",
    "extract_batch_status",
    "extract_batch_destroy",
    "extract_server_create", "extract_server_submit", "extract_server_wait", "extract_server_stats",
    "extract_server_destroy",
]

EXTRACT_BATCH_NO_GRAPH = 0x1
EXTRACT_BATCH_NO_TUNE = 0x2
EXTRACT_BATCH_DIRECT_ONLY = 0x4
EXTRACT_BATCH_TENSOR = 0x8


class extract_job_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("m", ctypes.c_uint32), ("s", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("sampling_key", ctypes.c_uint64),
                ("seed_bits_host", ctypes.c_void_p)]


class extract_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in
                ("submitted", "admitted", "completed", "failed", "rejected", "queued", "active", "waves",
                 "bytes_in_use", "bytes_peak")] + \
               [(name, ctypes.c_double) for name in
                ("p50_ms", "p99_ms", "mean_ms", "max_ms", "input_bits_done", "span_s", "gbit_per_s")]

EXTRACT_STATIC_SCRATCH_WORDS = 4 * 1024 * 1024


class ExtractError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libextract error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    """Load libextract.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libextract.so is not built (%s); run __graft_entry__.build(). "
                           "There is no CPU fallback." % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    L.extract_create.argtypes = [ctypes.POINTER(vp), u64, u32, u32, u32, vp, u64, u32]
    L.extract_run.argtypes = [vp, vp, vp, vp]
    L.extract_run_host.argtypes = [vp, vp, vp, vp]
    L.extract_run_host_many.argtypes = [vp, vp, vp, vp, u32]
    L.extract_gather.argtypes = [vp, vp, vp]
    L.extract_hash.argtypes = [vp, vp, vp]
    L.extract_run_plain.argtypes = [vp, vp, vp, vp]
    L.extract_read_perm.argtypes = [vp, u64, u64, vp]
    L.extract_read_subblock.argtypes = [vp, u32, vp]
    L.extract_subblock_sizes.argtypes = [vp, vp]
    L.extract_block_limit.argtypes = [u64, u32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(u64)]
    L.extract_describe.argtypes = [vp, ctypes.c_char_p, u32]
    L.extract_gather_bytes.argtypes = [vp, ctypes.POINTER(u64)]
    L.extract_status.argtypes = [vp]
    L.extract_destroy.argtypes = [vp]
    L.extract_run_static.argtypes = [u64, u32, u32, u32, vp, vp, vp, vp, vp]
    L.extract_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(extract_job_desc), u32, u32]
    L.extract_batch_run.argtypes = [vp, vp, vp, vp]
    L.extract_batch_run_sequential.argtypes = [vp, vp, vp, vp]
    L.extract_batch_describe.argtypes = [vp, ctypes.c_char_p, u32]
    L.extract_batch_status.argtypes = [vp]
    L.extract_batch_destroy.argtypes = [vp]
    L.extract_server_create.argtypes = [ctypes.POINTER(vp), u64, u32, u32, u32]
    L.extract_server_submit.argtypes = [vp, ctypes.POINTER(extract_job_desc), vp, vp, ctypes.POINTER(u64)]
    L.extract_server_wait.argtypes = [vp, u64, u32, ctypes.POINTER(ctypes.c_double)]
    L.extract_server_stats.argtypes = [vp, ctypes.POINTER(extract_stats)]
    L.extract_server_destroy.argtypes = [vp]
    L.extract_last_error.argtypes = []
    L.extract_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "extract_last_error":
            getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc: int) -> int:
    if rc != EXTRACT_OK:
        raise ExtractError(rc, load().extract_last_error().decode(errors="replace"))
    return rc


def _dev_ptr(x) -> int:
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if x.element_size() != 4:
        raise ValueError("expected 32-bit words")
    return x.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def extract_create(n: int, m: int, s: int, k: int, seed_bits: np.ndarray, sampling_key: int,
                   flags: int = 0) -> ctypes.c_void_p:
    seed = np.ascontiguousarray(seed_bits, dtype=np.uint32)
    h = ctypes.c_void_p()
    _check(load().extract_create(ctypes.byref(h), n, m, s, k, seed.ctypes.data, sampling_key, flags))
    return h


def extract_run(h, stream, in_bits, out_bits) -> None:
    _check(load().extract_run(h, _stream(stream), _dev_ptr(in_bits), _dev_ptr(out_bits)))


def _host_ptr(x, writable=False) -> int:
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] or x.dtype.itemsize != 4:
            raise ValueError("expected a contiguous array of 32-bit words")
        return x.ctypes.data
    if x.is_cuda or not x.is_contiguous() or x.element_size() != 4:
        raise ValueError("expected a contiguous host tensor of 32-bit words")
    return x.data_ptr()


def extract_run_host(h, stream, in_bits_host, out_bits_host) -> None:
    _check(load().extract_run_host(h, _stream(stream), _host_ptr(in_bits_host), _host_ptr(out_bits_host)))


def extract_run_host_many(h, stream, ins_host, outs_host) -> None:
    if len(ins_host) != len(outs_host):
        raise ValueError("one output per input")
    n = len(ins_host)
    pin = (ctypes.c_void_p * max(1, n))(*[_host_ptr(x) for x in ins_host])
    pout = (ctypes.c_void_p * max(1, n))(*[_host_ptr(x) for x in outs_host])
    _check(load().extract_run_host_many(h, _stream(stream), pin, pout, n))


def extract_gather(h, stream, in_bits) -> None:
    _check(load().extract_gather(h, _stream(stream), _dev_ptr(in_bits)))


def extract_hash(h, stream, out_bits) -> None:
    _check(load().extract_hash(h, _stream(stream), _dev_ptr(out_bits)))


def extract_run_plain(h, stream, in_bits, out_bits) -> None:
    _check(load().extract_run_plain(h, _stream(stream), _dev_ptr(in_bits), _dev_ptr(out_bits)))


def extract_read_perm(h, start: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.uint32)
    _check(load().extract_read_perm(h, start, count, out.ctypes.data))
    return out[:count]


def extract_subblock_sizes(h, m: int) -> np.ndarray:
    out = np.empty(max(m, 1), dtype=np.uint64)
    _check(load().extract_subblock_sizes(h, out.ctypes.data))
    return out[:m]


def extract_block_limit(N: int, m: int, eps: float, p: float) -> int:
    """Eq. 7's block size limit (host computation in the library)."""
    out = ctypes.c_uint64(0)
    _check(load().extract_block_limit(N, m, float(eps), float(p), ctypes.byref(out)))
    return int(out.value)


def extract_read_subblock(h, j: int, s: int) -> np.ndarray:
    out = np.empty((s + 31) // 32, dtype=np.uint32)
    _check(load().extract_read_subblock(h, j, out.ctypes.data))
    return out


def extract_describe(h) -> str:
    buf = ctypes.create_string_buffer(512)
    _check(load().extract_describe(h, buf, 512))
    return buf.value.decode()


def extract_status(h) -> None:
    """Raises ExtractError(EXTRACT_ETIMEDOUT) when a kernel of the context gave
    up on a bounded wait since the last call."""
    _check(load().extract_status(h))


def extract_gather_bytes(h) -> int:
    v = ctypes.c_uint64(0)
    _check(load().extract_gather_bytes(h, ctypes.byref(v)))
    return int(v.value)


def extract_run_static(n, m, s, k, perm, seed, in_bits, out_bits, stream=None) -> None:
    """The run without any device allocation (scratch in the library's static
    device memory); ``perm`` None means the identity order."""
    _check(load().extract_run_static(n, m, s, k, None if perm is None else _dev_ptr(perm), _dev_ptr(seed),
                                     _dev_ptr(in_bits), _dev_ptr(out_bits), _stream(stream)))


def extract_destroy(h) -> None:
    if h:
        _check(load().extract_destroy(h))


def extract_last_error() -> str:
    return load().extract_last_error().decode(errors="replace")


class Batch:
    """Owns one extract_batch.  ``jobs``: list of dicts with n, m, s, k, seed
    (np.uint32 words), key and optional flags."""

    def __init__(self, jobs, flags=0):
        self._seeds = [np.ascontiguousarray(j["seed"], dtype=np.uint32) for j in jobs]
        arr = (extract_job_desc * len(jobs))()
        for i, j in enumerate(jobs):
            arr[i] = extract_job_desc(j["n"], j["m"], j["s"], j["k"], j.get("flags", 0), j["key"],
                                      self._seeds[i].ctypes.data)
        self.jobs = jobs
        self.h = ctypes.c_void_p()
        _check(load().extract_batch_create(ctypes.byref(self.h), arr, len(jobs), flags))

    def _ptrs(self, ins, outs):
        n = len(self.jobs)
        if len(ins) != n or len(outs) != n:
            raise ValueError("need one input and one output per job")
        pi = (ctypes.c_void_p * n)(*[_dev_ptr(x) for x in ins])
        po = (ctypes.c_void_p * n)(*[_dev_ptr(x) for x in outs])
        return pi, po

    def run(self, ins, outs, stream=None):
        pi, po = self._ptrs(ins, outs)
        _check(load().extract_batch_run(self.h, _stream(stream), pi, po))

    def run_sequential(self, ins, outs, stream=None):
        pi, po = self._ptrs(ins, outs)
        _check(load().extract_batch_run_sequential(self.h, _stream(stream), pi, po))

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(1024)
        _check(load().extract_batch_describe(self.h, buf, 1024))
        return buf.value.decode()

    def status(self) -> None:
        """Raises ExtractError(EXTRACT_ETIMEDOUT) when a tensor-core kernel of
        the batch gave up on a bounded wait since the last call."""
        _check(load().extract_batch_status(self.h))

    def close(self):
        if self.h:
            _check(load().extract_batch_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns one extract_server (continuous batching under a memory budget)."""

    def __init__(self, hbm_budget_bytes, max_slots=64, wave_us=0):
        self.h = ctypes.c_void_p()
        self._keep = {}
        _check(load().extract_server_create(ctypes.byref(self.h), int(hbm_budget_bytes), max_slots, wave_us, 0))

    def submit(self, job, in_bits, out_bits) -> int:
        """``job``: dict with n, m, s, k, seed, key (and optional flags)."""
        seed = np.ascontiguousarray(job["seed"], dtype=np.uint32)
        d = extract_job_desc(job["n"], job["m"], job["s"], job["k"], job.get("flags", 0), job["key"],
                             seed.ctypes.data)
        t = ctypes.c_uint64()
        _check(load().extract_server_submit(self.h, ctypes.byref(d), _dev_ptr(in_bits), _dev_ptr(out_bits),
                                            ctypes.byref(t)))
        self._keep[t.value] = (in_bits, out_bits)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 600000) -> float:
        lat = ctypes.c_double()
        rc = load().extract_server_wait(self.h, ticket, timeout_ms, ctypes.byref(lat))
        if rc == EXTRACT_OK:
            self._keep.pop(ticket, None)
        _check(rc)
        return lat.value

    def stats(self) -> dict:
        st = extract_stats()
        _check(load().extract_server_stats(self.h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in st._fields_}

    def close(self):
        if self.h:
            _check(load().extract_server_destroy(self.h))
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Extractor:
    """Owns one extract_ctx: ``with Extractor(n, m, s, k, seed, key) as ex: ex.run(in_t, out_t)``."""

    def __init__(self, n, m, s, k, seed_bits, sampling_key, flags=0):
        self.n, self.m, self.s, self.k, self.flags = n, m, s, k, flags
        self.h = extract_create(n, m, s, k, seed_bits, sampling_key, flags)

    @property
    def out_words(self) -> int:
        return (self.m * self.k + 31) // 32

    def new_output(self):
        import torch
        return torch.empty(self.out_words, dtype=torch.int32, device="cuda")

    def run(self, in_bits, out_bits=None, stream=None):
        if out_bits is None:
            out_bits = self.new_output()
        extract_run(self.h, stream, in_bits, out_bits)
        return out_bits

    def run_host(self, in_bits_host, out_bits_host=None, stream=None):
        if out_bits_host is None:
            out_bits_host = np.empty(self.out_words, dtype=np.uint32)
        extract_run_host(self.h, stream, in_bits_host, out_bits_host)
        return out_bits_host

    def run_host_many(self, ins_host, outs_host=None, stream=None):
        if outs_host is None:
            outs_host = [np.empty(self.out_words, dtype=np.uint32) for _ in ins_host]
        extract_run_host_many(self.h, stream, ins_host, outs_host)
        return outs_host

    def run_plain(self, in_bits, out_bits=None, stream=None):
        if out_bits is None:
            out_bits = self.new_output()
        extract_run_plain(self.h, stream, in_bits, out_bits)
        return out_bits

    def gather(self, in_bits, stream=None):
        extract_gather(self.h, stream, in_bits)

    def hash(self, out_bits=None, stream=None):
        if out_bits is None:
            out_bits = self.new_output()
        extract_hash(self.h, stream, out_bits)
        return out_bits

    def read_perm(self, start=0, count=None):
        length = self.m * self.s if self.flags & EXTRACT_SAMPLING_IID else self.n
        return extract_read_perm(self.h, start, length - start if count is None else count)

    def sizes(self) -> np.ndarray:
        return extract_subblock_sizes(self.h, self.m)

    def read_subblock(self, j):
        return extract_read_subblock(self.h, j, self.s)

    def describe(self) -> str:
        return extract_describe(self.h)

    def status(self) -> None:
        extract_status(self.h)

    def gather_bytes(self) -> int:
        """Device-memory bytes one gather of this context reads and writes by design."""
        return extract_gather_bytes(self.h)

    def close(self):
        if self.h:
            extract_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
