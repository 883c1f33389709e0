"""TEST INFRASTRUCTURE: Python access to the C oracle in ``fic_oracle.c``.

The oracle is the plain CPU restatement of the paper's encoder and of the
iterated decoder; only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
library.  ``build()`` compiles it with the host C compiler (no SIMD flags, no
architecture-specific options) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES = {"nosearch": 0, "mns": 1, "local": 2, "exhaustive": 3}

LEAF_DTYPE = np.dtype([
    ("x", "<u2"), ("y", "<u2"), ("level", "u1"), ("phase", "u1"), ("k", "u1"),
    ("q", "u1"), ("d", "i1", (3,)), ("iso", "u1"), ("dx", "<u2"), ("dy", "<u2"),
])
assert LEAF_DTYPE.itemsize == 16


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32), ("bmax", ctypes.c_int32), ("bmin", ctypes.c_int32),
        ("thr_rms", ctypes.c_double * 4), ("s_bits", ctypes.c_int32), ("o_bits", ctypes.c_int32),
        ("phase2", ctypes.c_int32), ("local_radius", ctypes.c_int32), ("local_step", ctypes.c_int32),
        ("dom_step", ctypes.c_int32), ("isometries", ctypes.c_int32), ("phase2_domain", ctypes.c_int32),
    ]


def make_params(mode="mns", bmax=32, bmin=4, thr=8.0, s_bits=5, o_bits=7, phase2=True,
                local_radius=16, local_step=4, dom_step=4, isometries=8, phase2_domain=0) -> OrcParams:
    p = OrcParams()
    p.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    p.bmax, p.bmin = int(bmax), int(bmin)
    thr = list(thr) if isinstance(thr, (list, tuple)) else [float(thr)] * 4
    thr = (thr + [thr[-1]] * 4)[:4]
    for i in range(4):
        p.thr_rms[i] = float(thr[i])
    p.s_bits, p.o_bits = int(s_bits), int(o_bits)
    p.phase2 = 1 if phase2 else 0
    p.phase2_domain = int(phase2_domain)
    p.local_radius, p.local_step = int(local_radius), int(local_step)
    p.dom_step, p.isometries = int(dom_step), int(isometries)
    return p


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (plain -O2, no SIMD flags)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        u8p = P(ctypes.c_uint8)
        L.orc_encode.argtypes = [u8p, ctypes.c_int, ctypes.c_int, P(OrcParams), ctypes.c_void_p,
                                 ctypes.c_int, P(ctypes.c_uint32), P(ctypes.c_int), P(ctypes.c_int64)]
        L.orc_encode.restype = ctypes.c_int
        L.orc_decode.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 P(OrcParams), ctypes.c_int, u8p]
        L.orc_decode.restype = ctypes.c_int
        L.orc_bits.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               P(OrcParams), ctypes.c_int]
        L.orc_bits.restype = ctypes.c_int64
        vp = ctypes.c_void_p
        L.orc_serialize.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(OrcParams), ctypes.c_int, vp,
                                    ctypes.c_int64, vp, P(ctypes.c_int64)]
        L.orc_serialize.restype = ctypes.c_int
        L.orc_parse.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P(OrcParams), ctypes.c_int, vp,
                                ctypes.c_int, vp, vp, P(ctypes.c_int)]
        L.orc_parse.restype = ctypes.c_int
        L.orc_rescale.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(OrcParams), ctypes.c_int, vp,
                                  P(OrcParams), P(ctypes.c_int), P(ctypes.c_int)]
        L.orc_rescale.restype = ctypes.c_int
        L.orc_fit_pair.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32),
                                   P(ctypes.c_int32), P(ctypes.c_int64)]
        L.orc_fit_pair.restype = None
        i32p = P(ctypes.c_int32)
        L.orc_search_ranges.argtypes = [u8p, ctypes.c_int, ctypes.c_int, P(OrcParams), ctypes.c_int,
                                        i32p, i32p, i32p, i32p, i32p, i32p, i32p, i32p,
                                        P(ctypes.c_int64)]
        L.orc_search_ranges.restype = ctypes.c_int
        L.orc_count_ranges.argtypes = [ctypes.c_int] * 3
        L.orc_count_ranges.restype = ctypes.c_int64
        L.orc_count_domains.argtypes = [ctypes.c_int] * 4
        L.orc_count_domains.restype = ctypes.c_int64
        L.orc_contrast.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_contrast.restype = ctypes.c_int64
        L.orc_luminance.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_luminance.restype = ctypes.c_int64
        L.orc_phase2_contrast.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_phase2_contrast.restype = ctypes.c_int64
        L.orc_centred.argtypes = [ctypes.c_int] * 3
        L.orc_centred.restype = ctypes.c_int
        L.orc_threshold.argtypes = [ctypes.c_double, ctypes.c_int64]
        L.orc_threshold.restype = ctypes.c_int64
        L.orc_iso_source.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     P(ctypes.c_int), P(ctypes.c_int)]
        L.orc_iso_source.restype = None
        L.orc_count_candidates.argtypes = [u8p, ctypes.c_int, ctypes.c_int, P(OrcParams),
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_count_candidates.restype = ctypes.c_int
        L.orc_check.argtypes = [ctypes.c_int, ctypes.c_int, P(OrcParams)]
        L.orc_check.restype = ctypes.c_int
        _lib = L
    return _lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def nlevels(p: OrcParams) -> int:
    L, b = 1, p.bmax
    while b > p.bmin:
        b //= 2
        L += 1
    return L


class OracleError(RuntimeError):
    pass


def encode(img: np.ndarray, p: OrcParams):
    """Encode a uint8 (H, W) image.  Returns (leaves, split, fits)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    cap = max(1, (W // p.bmin) * (H // p.bmin))
    leaves = np.zeros(cap, dtype=LEAF_DTYPE)
    ntop = max(1, (W // p.bmax) * (H // p.bmax))
    split = np.zeros(ntop, dtype=np.uint32)
    nl = ctypes.c_int(0)
    fits = ctypes.c_int64(0)
    rc = lib().orc_encode(_u8(img), W, H, ctypes.byref(p), leaves.ctypes.data, cap,
                          split.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                          ctypes.byref(nl), ctypes.byref(fits))
    if rc != 0:
        raise OracleError(f"orc_encode failed: {rc}")
    return leaves[: nl.value].copy(), split, int(fits.value)


def decode(leaves: np.ndarray, W: int, H: int, p: OrcParams, iters: int) -> np.ndarray:
    leaves = np.ascontiguousarray(leaves, dtype=LEAF_DTYPE)
    out = np.zeros((H, W), dtype=np.uint8)
    rc = lib().orc_decode(leaves.ctypes.data, len(leaves), W, H, ctypes.byref(p), iters, _u8(out))
    if rc != 0:
        raise OracleError(f"orc_decode failed: {rc}")
    return out


def bits(leaves: np.ndarray, W: int, H: int, p: OrcParams, technique2: bool = True) -> int:
    leaves = np.ascontiguousarray(leaves, dtype=LEAF_DTYPE)
    return int(lib().orc_bits(leaves.ctypes.data, len(leaves), W, H, ctypes.byref(p),
                              1 if technique2 else 0))


def serialize(leaves: np.ndarray, W: int, H: int, p: OrcParams, technique2: bool = True):
    """The bitstream of Sections 3.3-3.4: (uint32 words, tile bit index of
    ntop + 1 entries, number of bits)."""
    leaves = np.ascontiguousarray(leaves, dtype=LEAF_DTYPE)
    ntop = (W // p.bmax) * (H // p.bmax)
    words = np.zeros(len(leaves) * 3 + 8, dtype=np.uint32)
    tile_bits = np.zeros(ntop + 1, dtype=np.uint64)
    nbits = ctypes.c_int64()
    rc = lib().orc_serialize(leaves.ctypes.data, len(leaves), W, H, ctypes.byref(p), 1 if technique2 else 0,
                             words.ctypes.data, words.size, tile_bits.ctypes.data, ctypes.byref(nbits))
    if rc:
        raise RuntimeError(f"orc_serialize failed ({rc})")
    return words[: (nbits.value + 31) // 32].copy(), tile_bits, int(nbits.value)


def parse(words: np.ndarray, nbits: int, W: int, H: int, p: OrcParams, technique2: bool = True):
    """Read a bitstream back: (leaves, split masks, tile bit index)."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    if words.size == 0:
        words = np.zeros(1, dtype=np.uint32)
    ntop = (W // p.bmax) * (H // p.bmax)
    cap = (W // p.bmin) * (H // p.bmin)
    out = np.zeros(cap, dtype=LEAF_DTYPE)
    split = np.zeros(ntop, dtype=np.uint32)
    tile_bits = np.zeros(ntop + 1, dtype=np.uint64)
    n = ctypes.c_int()
    rc = lib().orc_parse(words.ctypes.data, int(nbits), W, H, ctypes.byref(p), 1 if technique2 else 0,
                         out.ctypes.data, cap, split.ctypes.data, tile_bits.ctypes.data, ctypes.byref(n))
    if rc:
        raise ValueError(f"orc_parse: malformed stream ({rc})")
    return out[: n.value].copy(), split, tile_bits


def rescale(leaves: np.ndarray, W: int, H: int, p: OrcParams, shift: int):
    """The stream at 2**shift times the resolution (shift = +1 or -1):
    (leaves, params, W, H).  ValueError when it does not exist."""
    leaves = np.ascontiguousarray(leaves, dtype=LEAF_DTYPE)
    out = np.zeros_like(leaves)
    po = OrcParams()
    W2, H2 = ctypes.c_int(), ctypes.c_int()
    rc = lib().orc_rescale(leaves.ctypes.data, len(leaves), W, H, ctypes.byref(p), int(shift), out.ctypes.data,
                           ctypes.byref(po), ctypes.byref(W2), ctypes.byref(H2))
    if rc:
        raise ValueError(f"orc_rescale: no stream at this scale ({rc})")
    return out, po, W2.value, H2.value


def fit_pair(img, x, y, B, dx, dy, iso=0, s_bits=5, o_bits=7):
    """Moments (Sr, Srr, Sd, Sdd, Sdr), best (k, q) and E of one pair."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    mom = (ctypes.c_int64 * 5)()
    k, q, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    lib().orc_fit_pair(_u8(img), W, x, y, B, dx, dy, iso, s_bits, o_bits, mom,
                       ctypes.byref(k), ctypes.byref(q), ctypes.byref(e))
    return tuple(int(v) for v in mom), int(k.value), int(q.value), int(e.value)


def search_ranges(img, p: OrcParams, xs, ys, bs):
    """Phase-1 search of the listed ranges only: returns dict of arrays."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    n = len(xs)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    bs = np.ascontiguousarray(bs, dtype=np.int32)
    out = {name: np.zeros(n, dtype=np.int32) for name in ("k", "q", "dx", "dy", "iso")}
    e = np.zeros(n, dtype=np.int64)
    i32 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
    lib().orc_search_ranges(_u8(img), W, H, ctypes.byref(p), n, i32(xs), i32(ys), i32(bs),
                            i32(out["k"]), i32(out["q"]), i32(out["dx"]), i32(out["dy"]),
                            i32(out["iso"]), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    out["e"] = e
    return out


def contrast(k: int, s_bits: int = 5) -> int:
    return int(lib().orc_contrast(k, s_bits))


def luminance(q: int, o_bits: int = 7) -> int:
    return int(lib().orc_luminance(q, o_bits))


def phase2_contrast(level: int, bit: int) -> int:
    return int(lib().orc_phase2_contrast(level, bit))


def phase2_mbits(level: int) -> int:
    """Bits of a phase-2 mean difference at `level`, sign included (Section 3.3)."""
    return int(lib().orc_phase2_mbits(level))


def centred(x: int, B: int, W: int) -> int:
    return int(lib().orc_centred(x, B, W))


def threshold(thr_rms: float, n: int) -> int:
    return int(lib().orc_threshold(thr_rms, n))


def iso_source(iso: int, B: int, u: int, v: int):
    su, sv = ctypes.c_int(), ctypes.c_int()
    lib().orc_iso_source(iso, B, u, v, ctypes.byref(su), ctypes.byref(sv))
    return su.value, sv.value


def count_ranges(W, H, n):
    return int(lib().orc_count_ranges(W, H, n))


def count_domains(W, H, n, step=1):
    return int(lib().orc_count_domains(W, H, n, step))


def count_candidates(img, p: OrcParams, x: int, y: int, B: int) -> int:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    return int(lib().orc_count_candidates(_u8(img), W, H, ctypes.byref(p), x, y, B))


def check(W, H, p: OrcParams) -> int:
    return int(lib().orc_check(W, H, ctypes.byref(p)))


def offset_histogram(leaves: np.ndarray, W: int, H: int):
    """Counts of x_d - x_r (bin + W, 2W bins) and y_d - y_r (bin + H, 2H
    bins) over the leaves: the distributions Section 2 (Figs. 2, 3) shows
    for an exhaustive search."""
    ox = leaves["dx"].astype(np.int64) - leaves["x"].astype(np.int64) + W
    oy = leaves["dy"].astype(np.int64) - leaves["y"].astype(np.int64) + H
    return (np.bincount(ox, minlength=2 * W).astype(np.int64), np.bincount(oy, minlength=2 * H).astype(np.int64))


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    """Peak signal-to-noise ratio with peak 255 (Section 4)."""
    d = a.astype(np.float64) - b.astype(np.float64)
    mse = float(np.mean(d * d))
    if mse == 0.0:
        return float("inf")
    return 10.0 * np.log10(255.0 ** 2 / mse)
