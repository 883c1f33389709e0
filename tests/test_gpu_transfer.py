"""fic_records_to_host: each stream's records, as many as its info block
counts, and its info block land in page-locked host memory without a round
trip to the host; nothing past the count is written, and host pointers the
device cannot address (or misaligned ones) are rejected before anything is
enqueued."""
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


def _encode(fic, imgs, thr):
    d = [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]
    plan = fic.EncodePlan(d, [fic.params("mns", 32, 4, t) for t in thr])
    plan.run()
    torch.cuda.synchronize()
    return plan.outs


def test_records_and_info_reach_host(fic):
    imgs = [im for _, im in synth.scenes512_images()[:3]] + [synth.gaussian_scene(160, 5, 96)]
    sts = _encode(fic, imgs, [4.0, 8.0, 16.0, 8.0])
    h_rec = [torch.full((16 * s.capacity,), 0xA5, dtype=torch.uint8).pin_memory() for s in sts]
    h_info = [torch.full((fic.INFO_WORDS,), -7, dtype=torch.int32).pin_memory() for _ in sts]
    for rep in range(2):
        fic.records_to_host(sts, h_rec, h_info)
        torch.cuda.synchronize()
        for s, r, i in zip(sts, h_rec, h_info):
            want = s.to_host()
            n = len(want["records"])
            assert n > 0
            assert np.array_equal(r[: 16 * n].numpy(), want["records"].view(np.uint8))
            assert np.all(r[16 * n:].numpy() == 0xA5)  # nothing past the count is written
            assert np.array_equal(i.numpy(), s.info.cpu().numpy())


def test_more_streams_than_one_launch_holds(fic):
    imgs = [synth.gaussian_scene(64, 100 + k) for k in range(70)]
    sts = _encode(fic, imgs, [8.0] * 70)
    h_rec = [torch.zeros(16 * s.capacity, dtype=torch.uint8).pin_memory() for s in sts]
    fic.records_to_host(sts, h_rec)  # without info blocks
    torch.cuda.synchronize()
    for s, r in zip(sts, h_rec):
        want = s.to_host()["records"].view(np.uint8)
        assert np.array_equal(r[: want.size].numpy(), want)


def test_unaddressable_host_memory_is_rejected(fic):
    sts = _encode(fic, [synth.gaussian_scene(64, 3)], [8.0])
    L = fic.lib()
    Sa = (fic.fic.StreamC * 1)(sts[0].c)
    # pageable memory: rejected, unless the device addresses the host's page
    # tables (as on systems with a coherent CPU-GPU link), where the copy is valid
    pageable = np.ones(16 * sts[0].capacity + 16, dtype=np.uint8)  # pages written by the host first
    ptr = (ctypes.c_void_p * 1)(pageable.ctypes.data)
    rc = L.fic_records_to_host(Sa, 1, ptr, None, None)
    assert rc in (0, -2)
    if rc == 0:
        torch.cuda.synchronize()
        want = sts[0].to_host()["records"].view(np.uint8)
        assert np.array_equal(pageable[: want.size], want)
    pinned = torch.zeros(16 * sts[0].capacity + 16, dtype=torch.uint8).pin_memory()
    off = (ctypes.c_void_p * 1)(pinned.data_ptr() + 8)  # not 16-byte aligned
    assert L.fic_records_to_host(Sa, 1, off, None, None) == -2
    assert L.fic_records_to_host(Sa, 0, ptr, None, None) == -2
    with pytest.raises(fic.FicError):
        fic.records_to_host(sts, [torch.zeros(16 * sts[0].capacity, dtype=torch.uint8)])  # not pinned
