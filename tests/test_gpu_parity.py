"""GPU parity: the CUDA encoder and decoder (through the C ABI) against the
CPU oracle, record by record, split mask by split mask, pixel by pixel.

Everything here is integer work, so the bar is bit-exact equality.
"""
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


def _pair(fic, orc, mode, bmax, bmin, thr, **kw):
    return fic.params(mode, bmax, bmin, thr, **kw), orc.make_params(mode, bmax, bmin, thr, **kw)


def _assert_stream_equal(got, leaves, split, fits=None):
    rec = got["records"]
    assert len(rec) == len(leaves), f"record count {len(rec)} != {len(leaves)}"
    if len(rec):
        gb, wb = rec.view(np.uint8).reshape(-1, 16), leaves.view(np.uint8).reshape(-1, 16)
        bad = np.nonzero(np.any(gb != wb, axis=1))[0]
        assert bad.size == 0, f"{bad.size} records differ, first at {bad[0]}: got {rec[bad[0]]} want {leaves[bad[0]]}"
    assert np.array_equal(got["split"], split), "split masks differ"
    if fits is not None:
        assert got["fits"] == fits
    # tile offsets: first record of each top-level block, last = count
    offs = got["tile_offsets"]
    assert offs[-1] == len(leaves)


def _check_image(fic, orc, img, mode="mns", bmax=32, bmin=4, thr=8.0, iters=10, **kw):
    H, W = img.shape
    p, op = _pair(fic, orc, mode, bmax, bmin, thr, **kw)
    dimg = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    st = fic.fic_encode(dimg, p)
    got = st.to_host()
    leaves, split, fits = orc.encode(img, op)
    _assert_stream_equal(got, leaves, split, fits)
    tops = got["tile_offsets"]
    tw = W // bmax
    keys = (leaves["y"].astype(np.int64) // bmax) * tw + leaves["x"].astype(np.int64) // bmax
    want_offs = np.searchsorted(keys, np.arange(tw * (H // bmax) + 1), side="left")
    assert np.array_equal(tops.astype(np.int64), want_offs)
    if iters is not None:
        dec = fic.fic_decode(st, iters).cpu().numpy()
        want = orc.decode(leaves, W, H, op, iters)
        assert np.array_equal(dec, want), f"decoded pixels differ at {np.argwhere(dec != want)[:5]}"
    return got


def test_scene_256(fic, orc):
    """256x256 scene seed 0, MNS 16->8->4, RMS 8, decode 10 iterations."""
    _check_image(fic, orc, synth.scene256_image(), "mns", 16, 4, 8.0, iters=10)


@pytest.mark.parametrize("thr", [4.0, 8.0, 12.0, 16.0])
@pytest.mark.parametrize("mode", ["mns", "nosearch"])
def test_scene_512(fic, orc, thr, mode):
    _check_image(fic, orc, synth.gaussian_scene(512, 1), mode, 32, 4, thr, iters=10)


@pytest.mark.parametrize("seed", [101, 102])
def test_voronoi_512(fic, orc, seed):
    _check_image(fic, orc, synth.voronoi(512, seed), "mns", 32, 4, 8.0, iters=8)


@pytest.mark.parametrize("W,H,bmax,bmin", [
    (544, 96, 32, 4),     # 17 x 3 top blocks, ragged rows
    (208, 80, 16, 4),     # 13 top blocks per row: last strip holds one
    (208, 48, 8, 4),      # 26 per row: last strip holds ten
    (64, 64, 32, 4),      # minimum size for bmax 32
    (32, 32, 16, 4),
    (96, 64, 32, 8),      # bmin 8
    (128, 128, 32, 32),   # a single level
    (160, 96, 16, 16),
])
def test_sizes_and_levels(fic, orc, W, H, bmax, bmin):
    img = synth.gaussian_scene(W, 31 + W + H, H=H)
    _check_image(fic, orc, img, "mns", bmax, bmin, 6.0, iters=6)


@pytest.mark.parametrize("value", [0, 7, 129, 255])
def test_constant_images(fic, orc, value):
    got = _check_image(fic, orc, synth.constant(128, value), "mns", 32, 4, 8.0, iters=3)
    assert np.all(got["records"]["level"] == 1)


@pytest.mark.parametrize("thr", [0.0, 255.0, [20.0, 10.0, 5.0, 2.5]])
def test_threshold_extremes_and_per_level(fic, orc, thr):
    _check_image(fic, orc, synth.gaussian_scene(256, 17), "mns", 32, 4, thr, iters=4)


def test_paper_bit_widths(fic, orc):
    """3-bit contrast and 8-bit luminance (the paper's Section 3.3 widths)."""
    _check_image(fic, orc, synth.gaussian_scene(256, 19), "mns", 32, 4, 7.0, s_bits=3, o_bits=8, iters=5)


@pytest.mark.parametrize("s_bits,o_bits", [(1, 1), (7, 8), (4, 6)])
def test_other_codebooks(fic, orc, s_bits, o_bits):
    _check_image(fic, orc, synth.gaussian_scene(128, 23), "mns", 16, 4, 5.0, s_bits=s_bits, o_bits=o_bits,
                 iters=3)


def test_random_noise_image(fic, orc):
    rng = np.random.default_rng(99)
    img = rng.integers(0, 256, size=(256, 256), dtype=np.uint8)
    _check_image(fic, orc, img, "mns", 32, 4, 30.0, iters=5)


def test_batch_matches_single_and_oracle(fic, orc):
    """Mixed sizes in one persistent launch == one launch per image == oracle."""
    sizes = [(256, 256), (512, 512), (128, 384), (64, 64), (1024, 256)]
    imgs = [synth.gaussian_scene(w, 500 + i, H=h) for i, (w, h) in enumerate(sizes)]
    thrs = [8.0, 4.0, 12.0, 8.0, 16.0]
    plist = [fic.params("mns", 32, 4, t) for t in thrs]
    dimgs = [torch.from_numpy(im).cuda() for im in imgs]
    outs = fic.fic_encode_batch(dimgs, plist)
    decs = fic.fic_decode_batch(outs, 7)
    for im, t, st, dec in zip(imgs, thrs, outs, decs):
        got = st.to_host()
        leaves, split, fits = orc.encode(im, orc.make_params("mns", 32, 4, t))
        _assert_stream_equal(got, leaves, split, fits)
        single = fic.fic_encode(torch.from_numpy(im).cuda(), fic.params("mns", 32, 4, t)).to_host()
        assert np.array_equal(single["records"].view(np.uint8), got["records"].view(np.uint8))
        want = orc.decode(leaves, im.shape[1], im.shape[0], orc.make_params("mns", 32, 4, t), 7)
        assert np.array_equal(dec.cpu().numpy(), want)


def test_bench_workload_full_size(fic, orc):
    """The benchmark's launch: ten 512x512 images x four thresholds in one
    batch (40 encodes) and a batched 10-iteration decode, all bit-exact."""
    imgs = [im for _, im in synth.scenes512_images()]
    thrs = [4.0, 8.0, 12.0, 16.0]
    batch = [(im, t) for t in thrs for im in imgs]
    plist = [fic.params("mns", 32, 4, t) for _, t in batch]
    dimgs = [torch.from_numpy(im).cuda() for im, _ in batch]
    plan = fic.EncodePlan(dimgs, plist)
    plan.run()
    dplan = fic.DecodePlan(plan.outs)
    dplan.run(10)
    torch.cuda.synchronize()
    for (im, t), st, dec in zip(batch, plan.outs, dplan.outs):
        op = orc.make_params("mns", 32, 4, t)
        leaves, split, fits = orc.encode(im, op)
        _assert_stream_equal(st.to_host(), leaves, split, fits)
        assert np.array_equal(dec.cpu().numpy(), orc.decode(leaves, 512, 512, op, 10))


def test_deterministic_reruns(fic, orc):
    img = torch.from_numpy(synth.gaussian_scene(512, 3)).cuda()
    p = fic.params("mns", 32, 4, 8.0)
    a = fic.fic_encode(img, p).to_host()
    for _ in range(3):
        b = fic.fic_encode(img, p).to_host()
        assert np.array_equal(a["records"].view(np.uint8), b["records"].view(np.uint8))
        assert np.array_equal(a["split"], b["split"])


def test_decode_zero_and_one_iteration(fic, orc):
    img = synth.gaussian_scene(256, 41)
    p, op = _pair(fic, orc, "mns", 32, 4, 8.0)
    st = fic.fic_encode(torch.from_numpy(img).cuda(), p)
    assert np.all(fic.fic_decode(st, 0).cpu().numpy() == 128)
    leaves, _, _ = orc.encode(img, op)
    assert np.array_equal(fic.fic_decode(st, 1).cpu().numpy(), orc.decode(leaves, 256, 256, op, 1))


def test_host_rejects_bad_arguments(fic):
    img = torch.zeros((100, 100), dtype=torch.uint8, device="cuda")
    with pytest.raises(fic.FicError):
        fic.fic_encode(img, fic.params("mns", 32, 4, 8.0))
    with pytest.raises(fic.FicError):
        fic.fic_encode(torch.zeros((64, 64), dtype=torch.uint8, device="cuda"), fic.params("mns", 32, 2, 8.0))


# ---------------------------------------------------------------------------
# Local search (Section 2): candidates around the centred domain

@pytest.mark.parametrize("thr", [8.0, 4.0])
def test_local_scene_512(fic, orc, thr):
    _check_image(fic, orc, synth.gaussian_scene(512, 1), "local", 32, 4, thr, iters=6)


def test_local_voronoi_512(fic, orc):
    _check_image(fic, orc, synth.voronoi(512, 102), "local", 32, 4, 8.0, iters=4)


@pytest.mark.parametrize("W,H,bmax,bmin,R,S", [
    (544, 96, 32, 4, 16, 4),
    (208, 80, 16, 4, 16, 4),
    (208, 48, 8, 4, 8, 2),
    (64, 64, 32, 4, 16, 2),
    (96, 64, 32, 8, 4, 4),
    (160, 96, 16, 16, 16, 4),
])
def test_local_sizes(fic, orc, W, H, bmax, bmin, R, S):
    img = synth.gaussian_scene(W, 77 + W + H, H=H)
    _check_image(fic, orc, img, "local", bmax, bmin, 6.0, iters=4, local_radius=R, local_step=S)


def test_local_radius_zero_is_nosearch(fic, orc):
    img = torch.from_numpy(synth.gaussian_scene(256, 13)).cuda()
    a = fic.fic_encode(img, fic.params("local", 32, 4, 6.0, local_radius=0)).to_host()
    b = fic.fic_encode(img, fic.params("nosearch", 32, 4, 6.0)).to_host()
    assert np.array_equal(a["records"].view(np.uint8), b["records"].view(np.uint8))
    assert np.array_equal(a["split"], b["split"])


def test_decode_paths_agree(fic, orc):
    """Centred streams decode on 2x2-sum images; a batch that holds a
    local-search stream (or a stream too narrow for the window box) takes the
    pixel path.  Both equal the oracle."""
    a = synth.gaussian_scene(256, 61)
    b = synth.gaussian_scene(256, 62)
    pa, opa = _pair(fic, orc, "mns", 32, 4, 8.0)
    pb, opb = _pair(fic, orc, "local", 32, 4, 8.0)
    sa = fic.fic_encode(torch.from_numpy(a).cuda(), pa)
    sb = fic.fic_encode(torch.from_numpy(b).cuda(), pb)
    want_a = orc.decode(orc.encode(a, opa)[0], 256, 256, opa, 7)
    want_b = orc.decode(orc.encode(b, opb)[0], 256, 256, opb, 7)
    only_centred = fic.fic_decode_batch([sa], 7)[0].cpu().numpy()
    mixed = [t.cpu().numpy() for t in fic.fic_decode_batch([sa, sb], 7)]
    assert np.array_equal(only_centred, want_a)
    assert np.array_equal(mixed[0], want_a) and np.array_equal(mixed[1], want_b)
    for iters in (1, 2, 3):  # first-and-last, first then last, one middle iteration
        got = fic.fic_decode_batch([sa], iters)[0].cpu().numpy()
        assert np.array_equal(got, orc.decode(orc.encode(a, opa)[0], 256, 256, opa, iters))
    # bmax 16 on a 64-pixel-wide image: narrower than the 2x2-sum window box
    c = synth.gaussian_scene(64, 63, H=128)
    pc, opc = _pair(fic, orc, "mns", 16, 4, 6.0)
    sc = fic.fic_encode(torch.from_numpy(c).cuda(), pc)
    assert np.array_equal(fic.fic_decode(sc, 5).cpu().numpy(), orc.decode(orc.encode(c, opc)[0], 64, 128, opc, 5))


@pytest.mark.parametrize("bmax,bmin,side", [(32, 4, 512), (16, 4, 256), (8, 4, 192)])
def test_decode_single_launch_and_per_iteration_launches(fic, orc, bmax, bmin, side):
    """The 2x2-sum iterations after the first run either in one cooperative
    launch (grid barrier between iterations) or one launch per iteration;
    both equal the oracle for every iteration count, including 2 (no
    barrier) and 3 (one barrier), and a batch of several streams."""
    imgs = [synth.gaussian_scene(side, 70 + bmax), synth.voronoi(side, 80 + bmax)]
    p, op = _pair(fic, orc, "mns", bmax, bmin, 6.0)
    sts = [fic.fic_encode(torch.from_numpy(im).cuda(), p) for im in imgs]
    leaves = [orc.encode(im, op)[0] for im in imgs]
    plan = fic.DecodePlan(sts)
    for iters in (1, 2, 3, 4, 9):
        want = [orc.decode(lv, side, side, op, iters) for lv in leaves]
        for single in (1, 0):
            for k in (0, 1):
                plan.set_tuning(dec_single_launch=single, dec_ctas_per_sm=k)
                for o in plan.outs:
                    o.zero_()
                plan.run(iters)
                torch.cuda.synchronize()
                for o, w in zip(plan.outs, want):
                    assert np.array_equal(o.cpu().numpy(), w), (iters, single, k)
    for st in sts:
        st.info_host()  # no device error bit


# ---------------------------------------------------------------------------
# Phase 2 with the other domain reading: quadrants of the parent's domain

@pytest.mark.parametrize("img_fn,bmax,bmin,thr", [
    (lambda: synth.scene256_image(), 16, 4, 8.0),
    (lambda: synth.gaussian_scene(512, 1), 32, 4, 6.0),
    (lambda: synth.gaussian_scene(256, 44), 32, 8, 10.0),
    (lambda: synth.voronoi(256, 101), 16, 4, 4.0),
])
def test_phase2_parent_quadrants(fic, orc, img_fn, bmax, bmin, thr):
    img = img_fn()
    got = _check_image(fic, orc, img, "mns", bmax, bmin, thr, iters=6, phase2_domain=1)
    if bmax == 16 and thr == 8.0:  # this image keeps a phase-2 leaf under the quadrant reading
        assert (got["records"]["phase"] == 2).any()
