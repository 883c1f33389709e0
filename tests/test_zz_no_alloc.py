"""The allocation-free encode entry point (for callers that cannot allocate
device memory: its scratch lives in a static device array of the library)
gives exactly what fic_encode gives, on two calls in a row that reuse that
array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    fic.lib()
    return fic


def test_noalloc_matches_fic_encode_on_two_calls(fic):
    L = fic.lib()
    cases = [
        (synth.gaussian_scene(512, 5), fic.params("mns", 32, 4, 8.0)),
        (synth.gaussian_scene(256, 6, H=192), fic.params("mns", 16, 4, 6.0)),
        (synth.gaussian_scene(160, 7, H=96), fic.params("mns", 8, 4, 5.0)),
        (synth.voronoi(256, 8), fic.params("nosearch", 32, 4, 8.0)),
    ]
    for img, p in cases:
        H, W = img.shape
        dimg = torch.from_numpy(img).cuda()
        want = fic.fic_encode(dimg, p).to_host()
        st = fic.Stream(W, H, p)
        stream = torch.cuda.current_stream()
        rc = L.fic_encode_noalloc(ctypes.c_void_p(dimg.data_ptr()), W, H, ctypes.byref(p), ctypes.byref(st.c),
                                  ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, fic.FicError(rc, "fic_encode_noalloc")
        got = st.to_host()
        assert np.array_equal(got["records"].view(np.uint8), want["records"].view(np.uint8))
        assert np.array_equal(got["split"], want["split"])
        assert np.array_equal(got["tile_offsets"], want["tile_offsets"])
        assert got["fits"] == want["fits"]


def test_noalloc_rejects_images_beyond_its_scratch(fic):
    L = fic.lib()
    p = fic.params("mns", 32, 4, 8.0)
    small = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    st = fic.Stream(64, 64, p)
    # 16384 x 8192 needs 131072 strips of 1024 pixels: more than the static scratch holds
    rc = L.fic_encode_noalloc(ctypes.c_void_p(small.data_ptr()), 16384, 8192, ctypes.byref(p), ctypes.byref(st.c),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1


def _call(fic, img, W, H, p, st, stream):
    return fic.lib().fic_encode_noalloc(ctypes.c_void_p(img.data_ptr()), W, H, ctypes.byref(p), ctypes.byref(st.c),
                                        ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_rejects_search_modes(fic):
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    for mode, bmax in (("local", 16), ("exhaustive", 8)):
        p = fic.params(mode, bmax, bmax if mode == "exhaustive" else 4, 8.0)
        st = fic.Stream(64, 64, p)
        assert _call(fic, img, 64, 64, p, st, torch.cuda.current_stream()) == -2, mode


def test_noalloc_refuses_stream_capture(fic):
    """Under capture it returns FIC_EBADPARAM before enqueuing anything; the
    capture itself stays valid and a later uncaptured call still works."""
    img = synth.gaussian_scene(128, 9)
    dimg = torch.from_numpy(img).cuda()
    p = fic.params("mns", 32, 4, 8.0)
    st = fic.Stream(128, 128, p)
    side = torch.cuda.Stream()
    x = torch.zeros(16, device="cuda")
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
        x.add_(1)
        rc = _call(fic, dimg, 128, 128, p, st, side)
    assert rc == -2
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    assert _call(fic, dimg, 128, 128, p, st, torch.cuda.current_stream()) == 0
    want = fic.fic_encode(dimg, p).to_host()
    got = st.to_host()
    assert np.array_equal(got["records"].view(np.uint8), want["records"].view(np.uint8))
