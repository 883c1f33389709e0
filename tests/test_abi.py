"""The C-ABI library builds, loads without a GPU and exports every entry
point include/fic.h declares; host-only calls behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^FIC_API[^(]*?\b(fic_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def libfic():
    from paper_1501_02894_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(libfic):
    names = declared_symbols()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(libfic, n)]
    assert not missing, missing


def test_host_only_calls(libfic):
    from paper_1501_02894_gb300 import fic
    L = fic.lib()
    assert L.fic_version() > 0
    p = fic.params("mns", 32, 4, 8.0)
    assert fic.validate(512, 512, p) == 0
    assert fic.validate(500, 512, p) == -1            # not a multiple of bmax
    assert fic.validate(32, 64, p) == -1              # smaller than 2*bmax
    assert fic.validate(512, 512, fic.params("mns", 32, 2, 8.0)) == -2   # five levels (32 -> 2)
    assert fic.validate(512, 512, fic.params("mns", 16, 2, 8.0, s_bits=3, o_bits=8)) == 0  # the paper's 16 -> 2
    assert fic.validate(256, 256, fic.params("nosearch", 8, 2, 8.0)) == 0
    assert fic.validate(512, 512, fic.params("local", 16, 2, 8.0)) == -2  # 2 x 2 leaves: centred modes only
    assert fic.validate(512, 512, fic.params("mns", 64, 4, 8.0)) == -2   # bmax above 32
    assert fic.validate(512, 512, fic.params("mns", 32, 4, -1.0)) == -2
    ntop, cap = ctypes.c_int32(), ctypes.c_int32()
    assert L.fic_stream_sizes(512, 256, ctypes.byref(p), ctypes.byref(ntop), ctypes.byref(cap)) == 0
    assert (ntop.value, cap.value) == (16 * 8, 128 * 64)
    W = (ctypes.c_int * 2)(512, 256)
    H = (ctypes.c_int * 2)(512, 256)
    P = (fic.Params * 2)(p, p)
    assert L.fic_encode_workspace_bytes(2, W, H, P) > 0
    assert L.fic_decode_workspace_bytes(2, W, H) >= 512 * 512 + 256 * 256
    assert L.fic_strerror(-6) == b"device wait timed out"


def test_record_layout_matches_header():
    from paper_1501_02894_gb300 import fic
    assert fic.RECORD_DTYPE.itemsize == 16
    assert ctypes.sizeof(fic.Params) == 4 * 3 + 4 + 8 * 4 + 4 * 9 + 4  # padding after bmin and at the end


def test_server_structs_and_host_checks(libfic):
    import ctypes as C
    from paper_1501_02894_gb300 import fic
    assert C.sizeof(fic.ServerConfig) == 4 * 4 + 8 * 2
    assert C.sizeof(fic.JobC) == 4 * 3 + 4 + C.sizeof(fic.Params) + 4 * 2 + 8 * 5  # padding before params
    assert C.sizeof(fic.JobResult) == 4 * 2 + 8 * 3
    assert C.sizeof(fic.Tuning) == 4 * 6
    assert C.sizeof(fic.ServerStats) == 8 * 5 + 8 * 5
    L = fic.lib()
    cfg = fic.ServerConfig(0, 0, 8, 16, 1 << 20, 1 << 20)  # no streams
    h = C.c_void_p()
    assert L.fic_server_create(C.byref(cfg), C.byref(h)) == -2 and not h.value
    cfg = fic.ServerConfig(0, 1, 8, 16, 0, 1 << 20)       # no budget
    assert L.fic_server_create(C.byref(cfg), C.byref(h)) == -2
    t = C.c_int64()
    assert L.fic_submit(None, None, C.byref(t)) == -2
    assert L.fic_poll(None, 1, None) == -2
    assert L.fic_wait(None, 1, 0, None) == -2
    assert L.fic_server_destroy(None) == -2


def test_empty_batches_rejected_on_the_host(libfic):
    import ctypes as C
    from paper_1501_02894_gb300 import fic
    L = fic.lib()
    assert L.fic_encode_workspace_bytes(0, None, None, None) == 0
    assert L.fic_decode_workspace_bytes(0, None, None) == 0
    p = fic.params("mns", 32, 4, 8.0)
    assert L.fic_encode_batch(None, None, None, 0, C.byref(p), None, None, 0, None) == -2
