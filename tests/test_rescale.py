"""Resolution-independent decoding (Section 1): a stream rescaled by 2 or 1/2
keeps its codes and decodes on a finer or coarser grid.  The oracle's
rescale is pinned by exact facts; the device's rescaled stream and decode
must equal the oracle's."""
import numpy as np
import pytest

import synth


def _stream(orc, mode="mns", bmax=16, bmin=4, thr=6.0, N=128, seed=3, **kw):
    img = synth.gaussian_scene(N, seed)
    p = orc.make_params(mode, bmax, bmin, thr, **kw)
    leaves, _, _ = orc.encode(img, p)
    return img, p, leaves


def test_round_trip_is_identity(orc):
    _, p, leaves = _stream(orc)
    up, pu, W2, H2 = orc.rescale(leaves, 128, 128, p, +1)
    assert (W2, H2, pu.bmax, pu.bmin) == (256, 256, 32, 8)
    back, pb, W3, H3 = orc.rescale(up, W2, H2, pu, -1)
    assert (W3, H3, pb.bmax, pb.bmin) == (128, 128, 16, 4)
    assert np.array_equal(back.view(np.uint8), leaves.view(np.uint8))


def test_centred_domains_stay_centred(orc):
    _, p, leaves = _stream(orc, thr=4.0)
    up, pu, W2, H2 = orc.rescale(leaves, 128, 128, p, +1)
    for lf in up:
        B = pu.bmax >> (int(lf["level"]) - 1)
        assert int(lf["dx"]) == orc.centred(int(lf["x"]), B, W2)
        assert int(lf["dy"]) == orc.centred(int(lf["y"]), B, H2)


def test_first_iterate_is_the_upsampled_first_iterate(orc):
    _, p, leaves = _stream(orc)
    up, pu, W2, H2 = orc.rescale(leaves, 128, 128, p, +1)
    x1 = orc.decode(leaves, 128, 128, p, 1)
    x1u = orc.decode(up, W2, H2, pu, 1)
    assert np.array_equal(x1u, np.repeat(np.repeat(x1, 2, axis=0), 2, axis=1))


def test_constant_image_decodes_to_the_constant_at_every_scale(orc):
    img = synth.constant(128, 129)          # 129 = L(64) is on the 7-bit grid
    p = orc.make_params("mns", 16, 8, 6.0)
    leaves, _, _ = orc.encode(img, p)
    up, pu, W2, H2 = orc.rescale(leaves, 128, 128, p, +1)
    down, pd, W3, H3 = orc.rescale(up, W2, H2, pu, -1)
    half, ph, W4, H4 = orc.rescale(leaves, 128, 128, p, -1)
    for sl, ps, w, h in ((up, pu, W2, H2), (down, pd, W3, H3), (half, ph, W4, H4)):
        assert np.all(orc.decode(sl, w, h, ps, 6) == 129)


def test_half_scale_needs_even_geometry(orc):
    _, p, leaves = _stream(orc, bmax=16, bmin=4)
    with pytest.raises(ValueError):
        orc.rescale(leaves, 128, 128, p, -1)   # bmin 2 is below the decoder's smallest block


def test_twice_finer_decode_averages_to_the_decode(orc):
    """The attractor rendered at twice the resolution, averaged over 2x2
    pixels, is close to the attractor at the original resolution."""
    _, p, leaves = _stream(orc, thr=4.0)
    up, pu, W2, H2 = orc.rescale(leaves, 128, 128, p, +1)
    x = orc.decode(leaves, 128, 128, p, 12).astype(np.float64)
    xu = orc.decode(up, W2, H2, pu, 12).astype(np.float64)
    avg = xu.reshape(128, 2, 128, 2).mean(axis=(1, 3))
    assert np.mean(np.abs(avg - x)) < 2.0


@pytest.mark.gpu
@pytest.mark.parametrize("mode,bmax,bmin,shift,kw", [
    ("mns", 16, 4, +1, {}), ("mns", 32, 8, -1, {}), ("nosearch", 16, 8, +1, {}),
    ("local", 16, 4, +1, {}), ("exhaustive", 8, 8, +1, {}), ("mns", 16, 8, -1, {}),
])
def test_device_rescale_and_decode_equal_oracle(orc, mode, bmax, bmin, shift, kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    N = 128
    img = synth.gaussian_scene(N, 11)
    op = orc.make_params(mode, bmax, bmin, 6.0, **kw)
    leaves, split, _ = orc.encode(img, op)
    want, pw, W2, H2 = orc.rescale(leaves, N, N, op, shift)
    st = fic.fic_encode(torch.from_numpy(img).cuda(), fic.params(mode, bmax, bmin, 6.0, **kw))
    rs = fic.rescale(st, shift)
    assert (rs.width, rs.height, rs.params.bmax, rs.params.bmin) == (W2, H2, pw.bmax, pw.bmin)
    got = rs.to_host()
    assert np.array_equal(got["records"].view(np.uint8), want.view(np.uint8))
    assert np.array_equal(got["split"], split)
    dec = fic.fic_decode(rs, 7).cpu().numpy()
    assert np.array_equal(dec, orc.decode(want, W2, H2, pw, 7))
