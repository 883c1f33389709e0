"""Failure detection on the device: the bounded waits give up and report,
and the context stays usable afterwards (no trap, no hang)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_waits_give_up_and_report():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes

    import paper_1501_02894_gb300 as fic
    never = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(3, dtype=torch.int32, device="cuda")
    rc = fic.lib().fic_selftest_waits(ctypes.c_void_p(never.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == 1 and got[1] == 1 and got[2] > 1000
    # the context still works: a normal encode right after
    img = synth.gaussian_scene(64, 1)
    st = fic.fic_encode(torch.from_numpy(img).cuda(), fic.params("mns", 32, 4, 8.0))
    n, _ = st.info_host()
    assert n > 0
