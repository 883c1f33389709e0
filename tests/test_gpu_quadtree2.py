"""The paper's own quadtree on the GPU: range blocks from 16 x 16 down to
2 x 2 pixels (Sections 3.3-3.4: four levels, phase 2 at levels 1-3 with the
level-3 sets of Section 3.2), with the paper's 3-bit contrast and 8-bit
luminance codes.  The 2 x 2 blocks' domains (4 x 4 pixels) start at odd
coordinates inside the image.  Streams, split masks, fit counts and decoded
pixels are compared with the oracle, bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PAPER = {"s_bits": 3, "o_bits": 8}


@pytest.fixture(scope="module")
def fic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    fic.lib()
    return fic


def _compare(fic, orc, img, mode, bmax, bmin, thr, iters, **kw):
    H, W = img.shape
    p, op = fic.params(mode, bmax, bmin, thr, **kw), orc.make_params(mode, bmax, bmin, thr, **kw)
    st = fic.fic_encode(torch.from_numpy(np.ascontiguousarray(img)).cuda(), p)
    got = st.to_host()
    leaves, split, fits = orc.encode(img, op)
    assert got["records"].shape == leaves.shape, (len(got["records"]), len(leaves))
    gb, wb = got["records"].view(np.uint8).reshape(-1, 16), leaves.view(np.uint8).reshape(-1, 16)
    bad = np.nonzero(np.any(gb != wb, axis=1))[0]
    assert bad.size == 0, f"{bad.size} records differ, first {got['records'][bad[0]]} vs {leaves[bad[0]]}"
    assert np.array_equal(got["split"], split)
    assert got["fits"] == fits
    tw = W // bmax
    keys = (leaves["y"].astype(np.int64) // bmax) * tw + leaves["x"].astype(np.int64) // bmax
    assert np.array_equal(got["tile_offsets"].astype(np.int64),
                          np.searchsorted(keys, np.arange(tw * (H // bmax) + 1), side="left"))
    if iters:
        dec = fic.fic_decode(st, iters).cpu().numpy()
        want = orc.decode(leaves, W, H, op, iters)
        assert np.array_equal(dec, want), f"decoded pixels differ at {np.argwhere(dec != want)[:5]}"
    return leaves


@pytest.mark.parametrize("mode", ["mns", "nosearch"])
@pytest.mark.parametrize("thr", [4.0, 8.0, 16.0])
def test_paper_quadtree_scene_256(fic, orc, mode, thr):
    leaves = _compare(fic, orc, synth.scene256_image(), mode, 16, 2, thr, 10, **PAPER)
    if thr <= 8.0:
        assert (leaves["level"] == 4).any()  # 2 x 2 leaves present


@pytest.mark.parametrize("img_kind", ["scene", "voronoi"])
def test_paper_quadtree_512(fic, orc, img_kind):
    img = synth.gaussian_scene(512, 1) if img_kind == "scene" else synth.voronoi(512, 101)
    leaves = _compare(fic, orc, img, "mns", 16, 2, 8.0, 8, **PAPER)
    assert (leaves["phase"] == 2).any() and (leaves["level"] == 4).any()


@pytest.mark.parametrize("W,H,bmax", [(80, 48, 8), (144, 96, 16), (48, 32, 16), (272, 160, 8)])
def test_quadtree2_sizes(fic, orc, W, H, bmax):
    img = synth.gaussian_scene(W, W + H, H=H)
    _compare(fic, orc, img, "mns", bmax, 2, 5.0, 6)


def test_quadtree2_default_codebooks_and_per_level_thresholds(fic, orc):
    img = synth.gaussian_scene(256, 21)
    _compare(fic, orc, img, "mns", 16, 2, [10.0, 8.0, 6.0, 4.0], 7)


def test_quadtree2_parent_domain_reading(fic, orc):
    _compare(fic, orc, synth.gaussian_scene(256, 22), "mns", 16, 2, 6.0, 5, phase2_domain=1, **PAPER)


def test_quadtree2_mixed_batch(fic, orc):
    """2 x 2 and 4 x 4 last levels in one launch, encoded and decoded as a
    batch: each image equals its own oracle encode and decode."""
    specs = [(256, 31, 2, 8.0), (128, 32, 4, 6.0), (192, 33, 2, 12.0), (64, 34, 8, 4.0)]
    imgs = [synth.gaussian_scene(n, seed) for n, seed, _, _ in specs]
    plist = [fic.params("mns", 16, bmin, t, **PAPER) for (_, _, bmin, t) in specs]
    d = [torch.from_numpy(im).cuda() for im in imgs]
    plan = fic.EncodePlan(d, plist)
    plan.run()
    dplan = fic.DecodePlan(plan.outs)
    dplan.run(6)
    torch.cuda.synchronize()
    for i, (im, (_, _, bmin, t)) in enumerate(zip(imgs, specs)):
        op = orc.make_params("mns", 16, bmin, t, **PAPER)
        leaves, split, fits = orc.encode(im, op)
        got = plan.outs[i].to_host()
        assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8)), i
        assert np.array_equal(got["split"], split) and got["fits"] == fits, i
        want = orc.decode(leaves, im.shape[1], im.shape[0], op, 6)
        assert np.array_equal(dplan.outs[i].cpu().numpy(), want), i


def test_quadtree2_constant_image_decodes_exactly(fic, orc):
    img = np.full((64, 64), 130, np.uint8)
    leaves = _compare(fic, orc, img, "mns", 16, 2, 4.0, 3, **PAPER)
    assert len(leaves) == 16  # every 16 x 16 block accepted at level 1
