"""Thin Python binding of libfic.so (ctypes): argument marshalling only.

Every step of the coder runs in the library's CUDA kernels; PyTorch is used
here only to allocate device memory and to name the CUDA stream.  If the
library is missing, importing this module tries to build it with nvcc and
raises if that is impossible -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

MODES = {"nosearch": 0, "mns": 1, "local": 2, "exhaustive": 3}

RECORD_DTYPE = np.dtype([
    ("x", "<u2"), ("y", "<u2"), ("level", "u1"), ("phase", "u1"), ("k", "u1"),
    ("q", "u1"), ("d", "i1", (3,)), ("iso", "u1"), ("dx", "<u2"), ("dy", "<u2"),
])
assert RECORD_DTYPE.itemsize == 16

INFO_WORDS = 16
ERRORS = {
    0: "ok", -1: "unsupported image size", -2: "invalid parameter", -3: "buffer or workspace too small",
    -4: "record buffer too small", -5: "CUDA error", -6: "device wait timed out",
    -7: "request exceeds the memory budget", -8: "busy", -9: "cancelled",
}


class FicError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {ERRORS.get(code, 'error')} ({code})")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32), ("bmax", ctypes.c_int32), ("bmin", ctypes.c_int32),
        ("thr_rms", ctypes.c_double * 4), ("s_bits", ctypes.c_int32), ("o_bits", ctypes.c_int32),
        ("phase2", ctypes.c_int32), ("local_radius", ctypes.c_int32), ("local_step", ctypes.c_int32),
        ("dom_step", ctypes.c_int32), ("isometries", ctypes.c_int32), ("engine", ctypes.c_int32),
        ("phase2_domain", ctypes.c_int32),
    ]


class StreamC(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("params", Params),
        ("ntop", ctypes.c_int32), ("capacity", ctypes.c_int32),
        ("records", ctypes.c_void_p), ("tile_offsets", ctypes.c_void_p),
        ("split", ctypes.c_void_p), ("info", ctypes.c_void_p),
    ]


def params(mode="mns", bmax=32, bmin=4, thr=8.0, s_bits=5, o_bits=7, phase2=True,
           local_radius=16, local_step=4, dom_step=4, isometries=8, engine=0, phase2_domain=0) -> Params:
    p = Params()
    p.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    p.bmax, p.bmin = int(bmax), int(bmin)
    thr = list(thr) if isinstance(thr, (list, tuple)) else [float(thr)] * 4
    thr = (thr + [thr[-1]] * 4)[:4]
    for i in range(4):
        p.thr_rms[i] = float(thr[i])
    p.s_bits, p.o_bits = int(s_bits), int(o_bits)
    p.phase2 = 1 if phase2 else 0
    p.local_radius, p.local_step = int(local_radius), int(local_step)
    p.dom_step, p.isometries = int(dom_step), int(isometries)
    p.phase2_domain = int(phase2_domain)
    p.engine = int(engine)
    return p


class Tuning(ctypes.Structure):
    _fields_ = [("enc_warps", ctypes.c_int32), ("enc_ctas_per_sm", ctypes.c_int32), ("enc_dynamic", ctypes.c_int32),
                ("dec_ctas_per_sm", ctypes.c_int32), ("enc_fused_pack", ctypes.c_int32),
                ("dec_single_launch", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("host_staging_bytes", ctypes.c_int64)]


class JobC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("params", Params), ("iters", ctypes.c_int32), ("nrecords", ctypes.c_int32),
                ("image", ctypes.c_void_p), ("records", ctypes.c_void_p), ("out_image", ctypes.c_void_p),
                ("out_records", ctypes.c_void_p), ("out_split", ctypes.c_void_p)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("nrecords", ctypes.c_int32), ("fits", ctypes.c_int64),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("peak_device_bytes", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_batch", ctypes.c_double)]


_lib = None


def lib():
    """Load the in-tree libfic.so (building it with nvcc if it is missing)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            path = _build.build()
        L = ctypes.CDLL(path)
        vp, P = ctypes.c_void_p, ctypes.POINTER
        i32p = P(ctypes.c_int)
        L.fic_version.restype = ctypes.c_int
        L.fic_validate.argtypes = [ctypes.c_int, ctypes.c_int, P(Params)]
        L.fic_stream_sizes.argtypes = [ctypes.c_int, ctypes.c_int, P(Params), P(ctypes.c_int32), P(ctypes.c_int32)]
        L.fic_encode_workspace_bytes.argtypes = [ctypes.c_int, i32p, i32p, P(Params)]
        L.fic_encode_workspace_bytes.restype = ctypes.c_size_t
        L.fic_encode.argtypes = [vp, ctypes.c_int, ctypes.c_int, P(Params), P(StreamC), vp, ctypes.c_size_t, vp]
        L.fic_encode_batch.argtypes = [P(vp), i32p, i32p, ctypes.c_int, P(Params), P(StreamC), vp,
                                       ctypes.c_size_t, vp]
        L.fic_decode_workspace_bytes.argtypes = [ctypes.c_int, i32p, i32p]
        L.fic_decode_workspace_bytes.restype = ctypes.c_size_t
        L.fic_decode.argtypes = [P(StreamC), ctypes.c_int, vp, vp, ctypes.c_size_t, vp]
        L.fic_decode_batch.argtypes = [P(StreamC), ctypes.c_int, ctypes.c_int, P(vp), vp, ctypes.c_size_t, vp]
        L.fic_stream_info.argtypes = [P(StreamC), P(ctypes.c_int64), P(ctypes.c_int64), vp]
        L.fic_encode_plan_create.argtypes = [P(vp), i32p, i32p, ctypes.c_int, P(Params), P(StreamC), vp,
                                             ctypes.c_size_t, vp, P(vp)]
        L.fic_encode_plan_run.argtypes = [vp, vp]
        L.fic_decode_plan_create.argtypes = [P(StreamC), ctypes.c_int, P(vp), vp, ctypes.c_size_t, vp, P(vp)]
        L.fic_decode_plan_run.argtypes = [vp, ctypes.c_int, vp]
        L.fic_records_to_host.argtypes = [P(StreamC), ctypes.c_int, P(vp), P(vp), vp]
        L.fic_plan_destroy.argtypes = [vp]
        L.fic_plan_get_tuning.argtypes = [vp, P(Tuning)]
        L.fic_plan_run_timed.argtypes = [vp, ctypes.c_int, vp, P(ctypes.c_float), P(ctypes.c_char_p), ctypes.c_int,
                                         P(ctypes.c_int)]
        L.fic_plan_set_tuning.argtypes = [vp, P(Tuning)]
        L.fic_plan_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, P(Tuning), P(ctypes.c_float),
                                        P(ctypes.c_float), ctypes.c_int, P(ctypes.c_int)]
        L.fic_plan_destroy.restype = None
        L.fic_encode_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, P(Params), P(StreamC), vp]
        L.fic_server_create.argtypes = [P(ServerConfig), P(vp)]
        L.fic_submit.argtypes = [vp, P(JobC), P(ctypes.c_int64)]
        L.fic_poll.argtypes = [vp, ctypes.c_int64, P(JobResult)]
        L.fic_wait.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, P(JobResult)]
        L.fic_server_get_stats.argtypes = [vp, P(ServerStats)]
        L.fic_server_destroy.argtypes = [vp]
        L.fic_offset_histogram.argtypes = [P(StreamC), vp, vp, vp]
        L.fic_selftest_waits.argtypes = [vp, vp, vp]
        L.fic_validate_stream.argtypes = [ctypes.c_int, ctypes.c_int, P(Params)]
        L.fic_rescale_params.argtypes = [ctypes.c_int, ctypes.c_int, P(Params), ctypes.c_int, P(ctypes.c_int),
                                         P(ctypes.c_int), P(Params)]
        L.fic_stream_rescale.argtypes = [P(StreamC), ctypes.c_int, P(StreamC), vp]
        L.fic_bitstream_max_words.argtypes = [ctypes.c_int, ctypes.c_int, P(Params)]
        L.fic_bitstream_max_words.restype = ctypes.c_int64
        L.fic_bitstream_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, P(Params)]
        L.fic_bitstream_workspace_bytes.restype = ctypes.c_size_t
        L.fic_serialize.argtypes = [P(StreamC), ctypes.c_int, vp, ctypes.c_int64, vp, vp, ctypes.c_size_t, vp]
        L.fic_parse.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int, P(StreamC), vp, ctypes.c_size_t, vp]
        L.fic_bitstream_batch_workspace_bytes.argtypes = [P(StreamC), ctypes.c_int]
        L.fic_bitstream_batch_workspace_bytes.restype = ctypes.c_size_t
        L.fic_serialize_batch.argtypes = [P(StreamC), ctypes.c_int, ctypes.c_int, P(vp), P(ctypes.c_int64), P(vp), vp,
                                          ctypes.c_size_t, vp]
        L.fic_parse_batch.argtypes = [P(vp), P(ctypes.c_int64), P(vp), ctypes.c_int, P(StreamC), ctypes.c_int, vp,
                                      ctypes.c_size_t, vp]
        L.fic_strerror.argtypes = [ctypes.c_int]
        L.fic_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise FicError(rc, where)


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def stream_sizes(width: int, height: int, p: Params):
    """(top-level blocks, record capacity) of a stream."""
    ntop, cap = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().fic_stream_sizes(width, height, ctypes.byref(p), ctypes.byref(ntop), ctypes.byref(cap)),
           "fic_stream_sizes")
    return ntop.value, cap.value


class Stream:
    """A transform stream whose device buffers are owned by torch tensors.

    `records` / `info` may be given (uint8 views of capacity * 16 bytes,
    16-byte aligned, and int32 views of 16 words), e.g. slices of one arena
    so that a batch's streams come back to the host in one copy."""

    def __init__(self, width: int, height: int, p: Params, device="cuda", records=None, info=None):
        ntop, cap = stream_sizes(width, height, p)
        self.width, self.height, self.params = int(width), int(height), p
        self.ntop, self.capacity = ntop, cap
        if records is not None and (records.numel() < cap * 16 or records.data_ptr() % 16):
            raise ValueError("records view too small or not 16-byte aligned")
        if info is not None and info.numel() < INFO_WORDS:
            raise ValueError("info view too small")
        self.records = records if records is not None else torch.empty(cap * 16, dtype=torch.uint8, device=device)
        self.tile_offsets = torch.empty(self.ntop + 1, dtype=torch.int32, device=device)
        self.split = torch.empty(self.ntop, dtype=torch.int32, device=device)
        self.info = info if info is not None else torch.zeros(INFO_WORDS, dtype=torch.int32, device=device)
        self.c = StreamC()
        self.c.width, self.c.height, self.c.params = self.width, self.height, p
        self.c.ntop, self.c.capacity = self.ntop, self.capacity
        self.c.records = self.records.data_ptr()
        self.c.tile_offsets = self.tile_offsets.data_ptr()
        self.c.split = self.split.data_ptr()
        self.c.info = self.info.data_ptr()

    def info_host(self, stream=None):
        """(record count, fits); raises FicError on a device error."""
        n, f = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().fic_stream_info(ctypes.byref(self.c), ctypes.byref(n), ctypes.byref(f),
                                     _stream_handle(stream)), "fic_stream_info")
        return int(n.value), int(f.value)

    def to_host(self, stream=None):
        n, fits = self.info_host(stream)
        rec = self.records[: n * 16].cpu().numpy().view(RECORD_DTYPE).copy()
        return {
            "records": rec,
            "split": self.split.cpu().numpy().view(np.uint32).copy(),
            "tile_offsets": self.tile_offsets.cpu().numpy().view(np.uint32).copy(),
            "fits": fits,
        }


def encode_workspace(widths, heights, plist, device="cuda") -> torch.Tensor:
    n = len(widths)
    W = (ctypes.c_int * n)(*widths)
    H = (ctypes.c_int * n)(*heights)
    P = (Params * n)(*plist)
    b = lib().fic_encode_workspace_bytes(n, W, H, P)
    if b == 0:
        raise FicError(-2, "fic_encode_workspace_bytes")
    return torch.empty(int(b), dtype=torch.uint8, device=device)


def decode_workspace(widths, heights, device="cuda") -> torch.Tensor:
    n = len(widths)
    W = (ctypes.c_int * n)(*widths)
    H = (ctypes.c_int * n)(*heights)
    b = lib().fic_decode_workspace_bytes(n, W, H)
    if b == 0:
        raise FicError(-2, "fic_decode_workspace_bytes")
    return torch.empty(int(b), dtype=torch.uint8, device=device)


def _as_image(img: torch.Tensor) -> torch.Tensor:
    if not isinstance(img, torch.Tensor) or img.dtype != torch.uint8 or img.dim() != 2 or not img.is_cuda:
        raise TypeError("image must be a 2-D uint8 CUDA tensor")
    return img.contiguous()


def fic_encode(img: torch.Tensor, p: Params, out: Stream | None = None, workspace: torch.Tensor | None = None,
               stream=None) -> Stream:
    img = _as_image(img)
    H, W = img.shape
    out = out or Stream(W, H, p, img.device)
    ws = workspace if workspace is not None else encode_workspace([W], [H], [p], img.device)
    _check(lib().fic_encode(_ptr(img), W, H, ctypes.byref(p), ctypes.byref(out.c), _ptr(ws), ws.numel(),
                            _stream_handle(stream)), "fic_encode")
    out._keep = (img, ws)
    return out


def fic_encode_noalloc(img: torch.Tensor, p: Params, out: Stream | None = None, stream=None) -> Stream:
    """Encode one image without any workspace: for callers that cannot
    allocate device memory, the library keeps the encoder's scratch in a
    static device array (images up to 64 Mi pixels).  Calls whose work
    overlaps on the GPU must not be issued (they share that array)."""
    img = _as_image(img)
    H, W = img.shape
    out = out or Stream(W, H, p, img.device)
    _check(lib().fic_encode_noalloc(_ptr(img), W, H, ctypes.byref(p), ctypes.byref(out.c), _stream_handle(stream)),
           "fic_encode_noalloc")
    out._keep = (img,)
    return out


def fic_encode_batch(imgs, plist, outs=None, workspace=None, stream=None):
    imgs = [_as_image(t) for t in imgs]
    n = len(imgs)
    if n == 0:
        raise FicError(-2, "fic_encode_batch")
    if isinstance(plist, Params):
        plist = [plist] * n
    Ws = [int(t.shape[1]) for t in imgs]
    Hs = [int(t.shape[0]) for t in imgs]
    outs = outs or [Stream(Ws[i], Hs[i], plist[i], imgs[i].device) for i in range(n)]
    ws = workspace if workspace is not None else encode_workspace(Ws, Hs, plist, imgs[0].device)
    ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in imgs])
    Pa = (Params * n)(*plist)
    Sa = (StreamC * n)(*[o.c for o in outs])
    _check(lib().fic_encode_batch(ptrs, (ctypes.c_int * n)(*Ws), (ctypes.c_int * n)(*Hs), n, Pa, Sa,
                                  _ptr(ws), ws.numel(), _stream_handle(stream)), "fic_encode_batch")
    for i, o in enumerate(outs):
        o.c = Sa[i]
        o._keep = (imgs[i], ws)
    return outs


def fic_decode(st: Stream, iters: int, out: torch.Tensor | None = None, workspace=None, stream=None):
    out = out if out is not None else torch.empty((st.height, st.width), dtype=torch.uint8,
                                                  device=st.records.device)
    ws = workspace if workspace is not None else decode_workspace([st.width], [st.height], out.device)
    _check(lib().fic_decode(ctypes.byref(st.c), int(iters), _ptr(out), _ptr(ws), ws.numel(),
                            _stream_handle(stream)), "fic_decode")
    return out


def records_to_host(sts, h_records, h_info=None, stream=None):
    """Copy each Stream's records (as many as its info block counts) into the
    page-locked host tensor h_records[i] (uint8, room for its capacity), and
    its info block into h_info[i] when given, without waiting for the counts
    on the host (fic_records_to_host).  Asynchronous on `stream`."""
    n = len(sts)
    Sa = (StreamC * n)(*[s.c for s in sts])
    for s, h in zip(sts, h_records):
        if not h.is_pinned() or h.numel() < 16 * s.capacity:
            raise FicError(-2, "records_to_host: h_records must be pinned and hold the stream's capacity")
    hr = (ctypes.c_void_p * n)(*[h.data_ptr() for h in h_records])
    hi = (ctypes.c_void_p * n)(*[h.data_ptr() for h in h_info]) if h_info is not None else None
    _check(lib().fic_records_to_host(Sa, n, hr, hi, _stream_handle(stream)), "fic_records_to_host")


def fic_decode_batch(sts, iters: int, outs=None, workspace=None, stream=None):
    n = len(sts)
    if n == 0:
        raise FicError(-2, "fic_decode_batch")
    dev = sts[0].records.device
    outs = outs or [torch.empty((s.height, s.width), dtype=torch.uint8, device=dev) for s in sts]
    ws = workspace if workspace is not None else decode_workspace([s.width for s in sts],
                                                                  [s.height for s in sts], dev)
    Sa = (StreamC * n)(*[s.c for s in sts])
    ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(lib().fic_decode_batch(Sa, n, int(iters), ptrs, _ptr(ws), ws.numel(), _stream_handle(stream)),
           "fic_decode_batch")
    return outs


class _Tunable:
    """Launch mapping of a plan (fic_plan_get_tuning / set / autotune)."""

    @property
    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().fic_plan_get_tuning(self.handle, ctypes.byref(t)), "fic_plan_get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        _check(lib().fic_plan_get_tuning(self.handle, ctypes.byref(t)), "fic_plan_get_tuning")
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check(lib().fic_plan_set_tuning(self.handle, ctypes.byref(t)), "fic_plan_set_tuning")

    def _run_timed(self, iters, stream, cap=256):
        ms = (ctypes.c_float * cap)()
        labels = (ctypes.c_char_p * cap)()
        n = ctypes.c_int()
        _check(lib().fic_plan_run_timed(self.handle, int(iters), _stream_handle(stream), ms, labels, cap,
                                        ctypes.byref(n)), "fic_plan_run_timed")
        return [(labels[i].decode(), float(ms[i])) for i in range(n.value)]

    def _autotune(self, iters, reps, stream):
        best, ms, n = Tuning(), ctypes.c_float(), ctypes.c_int()
        cap = 64
        trace = (ctypes.c_float * (7 * cap))()
        _check(lib().fic_plan_autotune(self.handle, int(iters), int(reps), _stream_handle(stream), ctypes.byref(best),
                                       ctypes.byref(ms), trace, cap, ctypes.byref(n)), "fic_plan_autotune")
        rows = [tuple(trace[7 * i: 7 * i + 7]) for i in range(n.value)]
        keys = ("enc_warps", "enc_ctas_per_sm", "enc_dynamic", "dec_ctas_per_sm", "enc_fused_pack",
                "dec_single_launch")
        return {"best": best.as_dict(), "best_ms": ms.value,
                "trials": [dict({k: int(r[j]) for j, k in enumerate(keys)}, ms=float(r[6])) for r in rows]}


class EncodePlan(_Tunable):
    """Prepared batch encode: `run()` only enqueues kernels (graph-capturable)."""

    def __init__(self, imgs, plist, outs=None, workspace=None, stream=None):
        self.imgs = [_as_image(t) for t in imgs]
        n = len(self.imgs)
        if isinstance(plist, Params):
            plist = [plist] * n
        Ws = [int(t.shape[1]) for t in self.imgs]
        Hs = [int(t.shape[0]) for t in self.imgs]
        dev = self.imgs[0].device
        self.outs = outs or [Stream(Ws[i], Hs[i], plist[i], dev) for i in range(n)]
        self.ws = workspace if workspace is not None else encode_workspace(Ws, Hs, plist, dev)
        ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in self.imgs])
        Sa = (StreamC * n)(*[o.c for o in self.outs])
        self.handle = ctypes.c_void_p()
        _check(lib().fic_encode_plan_create(ptrs, (ctypes.c_int * n)(*Ws), (ctypes.c_int * n)(*Hs), n,
                                            (Params * n)(*plist), Sa, _ptr(self.ws), self.ws.numel(),
                                            _stream_handle(stream), ctypes.byref(self.handle)),
               "fic_encode_plan_create")
        for i, o in enumerate(self.outs):
            o.c = Sa[i]

    def run(self, stream=None):
        _check(lib().fic_encode_plan_run(self.handle, _stream_handle(stream)), "fic_encode_plan_run")

    def autotune(self, reps=5, stream=None):
        return self._autotune(0, reps, stream)

    def run_timed(self, stream=None):
        """Run once; [(kernel name, ms)] per launch (synchronous)."""
        return self._run_timed(0, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.fic_plan_destroy(h)
            self.handle = None


class DecodePlan(_Tunable):
    def __init__(self, sts, outs=None, workspace=None, stream=None):
        n = len(sts)
        dev = sts[0].records.device
        self.sts = sts
        self.outs = outs or [torch.empty((s.height, s.width), dtype=torch.uint8, device=dev) for s in sts]
        self.ws = workspace if workspace is not None else decode_workspace([s.width for s in sts],
                                                                           [s.height for s in sts], dev)
        Sa = (StreamC * n)(*[s.c for s in sts])
        ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        self.handle = ctypes.c_void_p()
        _check(lib().fic_decode_plan_create(Sa, n, ptrs, _ptr(self.ws), self.ws.numel(), _stream_handle(stream),
                                            ctypes.byref(self.handle)), "fic_decode_plan_create")

    def run(self, iters: int, stream=None):
        _check(lib().fic_decode_plan_run(self.handle, int(iters), _stream_handle(stream)), "fic_decode_plan_run")

    def autotune(self, iters: int, reps=5, stream=None):
        return self._autotune(iters, reps, stream)

    def run_timed(self, iters: int, stream=None):
        """Run once; [(kernel name, ms)] per launch (synchronous)."""
        return self._run_timed(iters, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.fic_plan_destroy(h)
            self.handle = None


def offset_histogram(st: Stream, stream=None):
    """Histograms (torch int32 on the stream's device) of x_d - x_r (2W bins,
    bin offset + W) and y_d - y_r (2H bins) over the stream's records."""
    hx = torch.zeros(2 * st.width, dtype=torch.int32, device=st.records.device)
    hy = torch.zeros(2 * st.height, dtype=torch.int32, device=st.records.device)
    _check(lib().fic_offset_histogram(ctypes.byref(st.c), _ptr(hx), _ptr(hy), _stream_handle(stream)),
           "fic_offset_histogram")
    return hx, hy


def serialize(st: Stream, technique2: bool = True, stream=None):
    """Bitstream of a stream (Sections 3.3-3.4): (uint32 word tensor of the
    maximal size, uint64 tile bit index).  The bit count is index[-1]."""
    L = lib()
    nw = int(L.fic_bitstream_max_words(st.width, st.height, ctypes.byref(st.params)))
    ws_n = int(L.fic_bitstream_workspace_bytes(st.width, st.height, ctypes.byref(st.params)))
    dev = st.records.device
    words = torch.empty(nw, dtype=torch.int32, device=dev)
    index = torch.empty(st.ntop + 1, dtype=torch.int64, device=dev)
    ws = torch.empty(ws_n, dtype=torch.uint8, device=dev)
    _check(L.fic_serialize(ctypes.byref(st.c), 1 if technique2 else 0, _ptr(words), nw, _ptr(index), _ptr(ws), ws_n,
                           _stream_handle(stream)), "fic_serialize")
    return words, index


def parse(words: torch.Tensor, index: torch.Tensor, width: int, height: int, p: Params, technique2: bool = True,
          stream=None) -> Stream:
    """Read a bitstream back into a new Stream on the words' device."""
    L = lib()
    st = Stream(width, height, p, words.device)
    ws_n = int(L.fic_bitstream_workspace_bytes(width, height, ctypes.byref(p)))
    ws = torch.empty(ws_n, dtype=torch.uint8, device=words.device)
    _check(L.fic_parse(_ptr(words), words.numel(), _ptr(index), 1 if technique2 else 0, ctypes.byref(st.c), _ptr(ws),
                       ws_n, _stream_handle(stream)), "fic_parse")
    return st


def serialize_batch(sts, technique2: bool = True, stream=None, outs=None, workspace=None):
    """Bitstreams of several streams in one batched call: [(words, index)]
    as serialize() gives them, stream by stream.  `outs` (a previous
    result) and `workspace` may be passed to reuse their buffers."""
    L = lib()
    n = len(sts)
    if n == 0:
        raise FicError(-2, "serialize_batch: no streams")
    dev = sts[0].records.device
    if outs is None:
        outs = []
        for st in sts:
            nw = int(L.fic_bitstream_max_words(st.width, st.height, ctypes.byref(st.params)))
            outs.append((torch.empty(nw, dtype=torch.int32, device=dev),
                         torch.empty(st.ntop + 1, dtype=torch.int64, device=dev)))
    wp = [w.data_ptr() for w, _ in outs]
    ip = [ix.data_ptr() for _, ix in outs]
    nws = [w.numel() for w, _ in outs]
    Sa = (StreamC * n)(*[st.c for st in sts])
    ws_n = int(L.fic_bitstream_batch_workspace_bytes(Sa, n))
    ws = workspace if workspace is not None else torch.empty(max(ws_n, 1), dtype=torch.uint8, device=dev)
    if ws.numel() < ws_n:
        raise FicError(-3, "serialize_batch: workspace too small")
    _check(L.fic_serialize_batch(Sa, n, 1 if technique2 else 0, (ctypes.c_void_p * n)(*wp), (ctypes.c_int64 * n)(*nws),
                                 (ctypes.c_void_p * n)(*ip), _ptr(ws), ws_n, _stream_handle(stream)),
           "fic_serialize_batch")
    return outs


def parse_batch(items, technique2: bool = True, stream=None, outs=None, workspace=None):
    """Read several bitstreams back in one batched call.  `items`: (words,
    index, width, height, params) per stream; returns Streams (new ones, or
    the given `outs`, whose geometry must match).  `workspace` may be
    passed to reuse it."""
    L = lib()
    n = len(items)
    if n == 0:
        raise FicError(-2, "parse_batch: no streams")
    dev = items[0][0].device
    if outs is None:
        outs = [Stream(W, H, p, dev) for (_, _, W, H, p) in items]
    Sa = (StreamC * n)(*[o.c for o in outs])
    ws_n = int(L.fic_bitstream_batch_workspace_bytes(Sa, n))
    ws = workspace if workspace is not None else torch.empty(max(ws_n, 1), dtype=torch.uint8, device=dev)
    if ws.numel() < ws_n:
        raise FicError(-3, "parse_batch: workspace too small")
    _check(L.fic_parse_batch((ctypes.c_void_p * n)(*[w.data_ptr() for (w, _, _, _, _) in items]),
                             (ctypes.c_int64 * n)(*[w.numel() for (w, _, _, _, _) in items]),
                             (ctypes.c_void_p * n)(*[ix.data_ptr() for (_, ix, _, _, _) in items]),
                             1 if technique2 else 0, Sa, n, _ptr(ws), ws_n, _stream_handle(stream)), "fic_parse_batch")
    for o, c in zip(outs, Sa):
        o.c = c  # the call filled the C structs
    return outs


def rescale(st: Stream, shift: int, stream=None) -> Stream:
    """The stream at 2**shift times the resolution (shift +1 or -1), as a new
    Stream on the same device (Section 1: resolution-independent decoding)."""
    W, H, q = ctypes.c_int(), ctypes.c_int(), Params()
    _check(lib().fic_rescale_params(st.width, st.height, ctypes.byref(st.params), int(shift), ctypes.byref(W),
                                    ctypes.byref(H), ctypes.byref(q)), "fic_rescale_params")
    out = Stream(W.value, H.value, q, st.records.device)
    _check(lib().fic_stream_rescale(ctypes.byref(st.c), int(shift), ctypes.byref(out.c), _stream_handle(stream)),
           "fic_stream_rescale")
    return out


def validate(width: int, height: int, p: Params) -> int:
    return int(lib().fic_validate(int(width), int(height), ctypes.byref(p)))


JOB_ENCODE, JOB_DECODE = 0, 1


class Server:
    """Continuous-batching request server of the library (fic_submit & co).

    Host buffers of a job (numpy arrays) are kept alive here until the job
    has been polled or waited for."""

    def __init__(self, hbm_budget_bytes=1 << 30, streams=4, max_batch=64, queue_capacity=100000,
                 host_staging_bytes=1 << 30, device=None):
        cfg = ServerConfig()
        cfg.device = torch.cuda.current_device() if device is None else int(device)
        cfg.streams, cfg.max_batch, cfg.queue_capacity = int(streams), int(max_batch), int(queue_capacity)
        cfg.hbm_budget_bytes, cfg.host_staging_bytes = int(hbm_budget_bytes), int(host_staging_bytes)
        self.handle = ctypes.c_void_p()
        _check(lib().fic_server_create(ctypes.byref(cfg), ctypes.byref(self.handle)), "fic_server_create")
        self._live = {}

    def submit_encode(self, image: np.ndarray, p: Params, out_records=None, out_split=None) -> int:
        """Queue an encode; out_records / out_split (optional, reused by the
        caller) must hold (W/bmin)*(H/bmin) records and (W/bmax)*(H/bmax) words."""
        image = np.ascontiguousarray(image, dtype=np.uint8)
        H, W = image.shape
        cap = (W // p.bmin) * (H // p.bmin)
        ntop = (W // p.bmax) * (H // p.bmax)
        out_rec = out_records if out_records is not None else np.zeros(max(cap, 1), dtype=RECORD_DTYPE)
        out_split = out_split if out_split is not None else np.zeros(max(ntop, 1), dtype=np.uint32)
        if out_rec.dtype != RECORD_DTYPE or out_rec.size < cap or not out_rec.flags.c_contiguous:
            raise ValueError("out_records too small or not a contiguous record array")
        if out_split.dtype != np.uint32 or out_split.size < ntop or not out_split.flags.c_contiguous:
            raise ValueError("out_split too small or not contiguous uint32")
        j = JobC()
        j.kind, j.width, j.height, j.params = JOB_ENCODE, W, H, p
        j.image = image.ctypes.data
        j.out_records = out_rec.ctypes.data
        j.out_split = out_split.ctypes.data
        t = ctypes.c_int64()
        _check(lib().fic_submit(self.handle, ctypes.byref(j), ctypes.byref(t)), "fic_submit")
        self._live[t.value] = ("encode", image, out_rec, out_split)
        return t.value

    def submit_decode(self, records: np.ndarray, W: int, H: int, p: Params, iters: int, out=None) -> int:
        records = np.ascontiguousarray(records, dtype=RECORD_DTYPE)
        out = out if out is not None else np.zeros((H, W), dtype=np.uint8)
        if out.dtype != np.uint8 or out.shape != (H, W) or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous (H, W) uint8 array")
        j = JobC()
        j.kind, j.width, j.height, j.params, j.iters = JOB_DECODE, W, H, p, int(iters)
        j.nrecords = len(records)
        j.records = records.ctypes.data
        j.out_image = out.ctypes.data
        t = ctypes.c_int64()
        _check(lib().fic_submit(self.handle, ctypes.byref(j), ctypes.byref(t)), "fic_submit")
        self._live[t.value] = ("decode", records, out)
        return t.value

    def _output(self, ticket, res):
        ent = self._live.pop(ticket)
        if ent[0] == "encode":
            # views of the output buffers (the caller's own, when it passed them)
            return {"records": ent[2][: res.nrecords], "split": ent[3], "fits": int(res.fits),
                    "latency_ms": res.latency_ms, "queue_ms": res.queue_ms}
        return {"image": ent[2], "latency_ms": res.latency_ms, "queue_ms": res.queue_ms}

    def poll(self, ticket):
        res = JobResult()
        rc = lib().fic_poll(self.handle, ticket, ctypes.byref(res))
        if rc == -8:
            return None
        _check(rc, "fic_poll")
        return self._output(ticket, res)

    def wait(self, ticket, timeout_ms=-1):
        res = JobResult()
        _check(lib().fic_wait(self.handle, ticket, int(timeout_ms), ctypes.byref(res)), "fic_wait")
        return self._output(ticket, res)

    def stats(self):
        st = ServerStats()
        _check(lib().fic_server_get_stats(self.handle, ctypes.byref(st)), "fic_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().fic_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
