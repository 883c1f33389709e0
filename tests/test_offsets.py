"""Position statistics of Section 2 (Figs. 2, 3): histograms of x_d - x_r and
y_d - y_r over a stream's records; the oracle's counts are pinned on planted
leaves, the device's counts must equal the oracle's."""
import numpy as np
import pytest

import synth


def test_oracle_histogram_planted(orc):
    W, H = 64, 32
    lv = np.zeros(5, dtype=orc.LEAF_DTYPE)
    for i, (x, y, dx, dy) in enumerate([(0, 0, 0, 0), (8, 0, 0, 0), (56, 24, 0, 16), (8, 8, 40, 0), (0, 16, 8, 8)]):
        lv[i]["x"], lv[i]["y"], lv[i]["dx"], lv[i]["dy"] = x, y, dx, dy
    hx, hy = orc.offset_histogram(lv, W, H)
    assert hx.shape == (2 * W,) and hy.shape == (2 * H,)
    want_x = np.zeros(2 * W, dtype=np.int64)
    for off in (0, -8, -56, 32, 8):
        want_x[off + W] += 1
    want_y = np.zeros(2 * H, dtype=np.int64)
    for off in (0, 0, -8, -8, -8):
        want_y[off + H] += 1
    assert np.array_equal(hx, want_x) and np.array_equal(hy, want_y)


def test_oracle_histogram_exhaustive_finds_planted_offset(orc):
    """A range planted as an affine copy of a known domain: the exhaustive
    search's record for it lands in the planted bins."""
    from test_oracle_pins import _plant
    from fractions import Fraction as F
    rng = np.random.default_rng(7)
    img = np.clip(synth.gaussian_scene(64, 8).astype(int) + rng.integers(-40, 40, (64, 64)), 0, 255).astype(np.uint8)
    x, y, dx, dy = 48, 8, 4, 36
    _plant(img, x, y, 8, dx, dy, 0, F(3, 4) - F(1, 32), 120)
    p = orc.make_params("exhaustive", 8, 8, 8.0, dom_step=4, isometries=1)
    leaves, _, _ = orc.encode(img, p)
    lf = leaves[(leaves["x"] == x) & (leaves["y"] == y)][0]
    assert (int(lf["dx"]), int(lf["dy"])) == (dx, dy)
    hx, hy = orc.offset_histogram(leaves, 64, 64)
    assert hx.sum() == hy.sum() == leaves.size == 64
    assert hx[dx - x + 64] >= 1 and hy[dy - y + 64] >= 1


@pytest.mark.gpu
@pytest.mark.parametrize("mode,engine", [("exhaustive", 0), ("exhaustive", 1), ("mns", 0), ("local", 0)])
def test_device_histogram_equals_oracle(orc, mode, engine):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    img = synth.gaussian_scene(128, 81)
    if mode == "exhaustive":
        p = fic.params(mode, 8, 8, 8.0, engine=engine)
        op = orc.make_params(mode, 8, 8, 8.0)
    else:
        p = fic.params(mode, 32, 4, 8.0)
        op = orc.make_params(mode, 32, 4, 8.0)
    st = fic.fic_encode(torch.from_numpy(img).cuda(), p)
    hx, hy = fic.offset_histogram(st)
    leaves, _, _ = orc.encode(img, op)
    wx, wy = orc.offset_histogram(leaves, 128, 128)
    assert np.array_equal(hx.cpu().numpy().astype(np.int64), wx)
    assert np.array_equal(hy.cpu().numpy().astype(np.int64), wy)
