"""GB300-native fractal image coder: the modified no-search (MNS) quadtree
encoder of arxiv 1501.02894, its comparison modes and an iterated decoder,
as hand-written sm_103a CUDA kernels behind the C ABI in include/fic.h.

This package is the Python binding of that library (``fic.py``) and its
build script (``build.py``); the kernels live in ``csrc/``.
"""
from .fic import (  # noqa: F401
    INFO_WORDS,
    RECORD_DTYPE,
    Server,
    Tuning,
    DecodePlan,
    EncodePlan,
    FicError,
    Params,
    Stream,
    fic_decode,
    fic_decode_batch,
    fic_encode,
    fic_encode_batch,
    fic_encode_noalloc,
    lib,
    offset_histogram,
    params,
    parse,
    parse_batch,
    records_to_host,
    rescale,
    serialize,
    serialize_batch,
    stream_sizes,
    validate,
)
