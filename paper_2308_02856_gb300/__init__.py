"""GB300 (sm_103a) sampled sub-block Toeplitz hashing (arXiv 2308.02856).

The hashing path runs in hand-written CUDA kernels behind the C ABI of
``libextract.so`` (``include/extract.h``); ``extract`` is its ctypes binding
and ``synth`` draws seeded synthetic inputs.
"""
from . import synth  # noqa: F401
from .extract import (  # noqa: F401
    EXTRACT_IDENTITY_PERM,
    EXTRACT_KEY_BITS,
    EXTRACT_METHOD_DIRECT,
    EXTRACT_METHOD_NTT,
    EXTRACT_SEED_PER_SUBBLOCK,
    ExtractError,
    Extractor,
    extract_create,
    extract_describe,
    extract_destroy,
    extract_gather,
    extract_hash,
    extract_last_error,
    extract_read_perm,
    extract_read_subblock,
    extract_run,
    extract_run_host,
    extract_run_plain,
    extract_run_static,
)
