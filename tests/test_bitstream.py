"""Bitstream of the stored parameters (Section 3.3) with Technique 2's level
ids (Section 3.4): the oracle's writer and reader are pinned against the bit
accounting and each other; the device writer and reader must produce the
oracle's words and records."""
import numpy as np
import pytest

import synth

CASES = [
    ("mns", 32, 4, 8.0, 512, {}),
    ("mns", 16, 4, 6.0, 256, {}),
    ("mns", 32, 8, 12.0, 256, {}),
    ("nosearch", 32, 4, 8.0, 256, {}),
    ("mns", 16, 2, 7.0, 64, {"s_bits": 3, "o_bits": 8}),   # the paper's widths and sizes
    ("local", 32, 4, 8.0, 256, {}),
    ("exhaustive", 8, 8, 8.0, 128, {}),
    ("exhaustive", 8, 8, 8.0, 96, {"dom_step": 2, "isometries": 3}),
]


def _encode(orc, mode, bmax, bmin, thr, N, kw, seed=5):
    img = synth.gaussian_scene(N, seed)
    p = orc.make_params(mode, bmax, bmin, thr, **kw)
    leaves, split, _ = orc.encode(img, p)
    return p, leaves, split


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-{c[4]}" for c in CASES])
@pytest.mark.parametrize("t2", [True, False])
def test_oracle_round_trip_and_bit_count(orc, case, t2):
    mode, bmax, bmin, thr, N, kw = case
    p, leaves, split = _encode(orc, mode, bmax, bmin, thr, N, kw)
    words, tile_bits, nbits = orc.serialize(leaves, N, N, p, t2)
    assert nbits == orc.bits(leaves, N, N, p, technique2=t2)      # the Section 3.3/3.4 accounting
    back, split2, tile_bits2 = orc.parse(words, nbits, N, N, p, t2)
    assert np.array_equal(back.view(np.uint8), leaves.view(np.uint8))
    assert np.array_equal(split2, split)
    assert np.array_equal(tile_bits2, tile_bits)
    assert tile_bits[0] == 0 and tile_bits[-1] == nbits and np.all(np.diff(tile_bits.astype(np.int64)) > 0)


def test_technique2_saves_exactly_the_implied_level_bits(orc):
    p, leaves, _ = _encode(orc, "mns", 32, 4, 4.0, 256, {})
    _, _, with_t2 = orc.serialize(leaves, 256, 256, p, True)
    _, _, without = orc.serialize(leaves, 256, 256, p, False)
    last = leaves[leaves["level"] == 4]
    implied = int(np.sum(~(((last["x"] // 4) % 2 == 0) & ((last["y"] // 4) % 2 == 0))))
    assert without - with_t2 == 2 * implied  # 2 level bits each (4 levels)
    assert implied == 3 * (len(last) // 4) and len(last) % 4 == 0


def test_field_layout_of_one_leaf(orc):
    """One phase-1 leaf at level 1 of a 1-level stream (no level bits, no
    phase bit): k then q, least-significant bit first."""
    p = orc.make_params("nosearch", 32, 32, 8.0)
    lv = np.zeros(4, dtype=orc.LEAF_DTYPE)
    for i, (x, y) in enumerate([(0, 0), (32, 0), (0, 32), (32, 32)]):
        lv[i]["x"], lv[i]["y"], lv[i]["level"], lv[i]["phase"] = x, y, 1, 1
        lv[i]["dx"], lv[i]["dy"] = orc.centred(x, 32, 64), orc.centred(y, 32, 64)
    lv[0]["k"], lv[0]["q"] = 0b10011, 0b1010101
    words, tile_bits, nbits = orc.serialize(lv, 64, 64, p, True)
    assert nbits == 4 * 12 and list(tile_bits) == [0, 12, 24, 36, 48]
    assert int(words[0]) & 0xFFF == 0b1010101_10011


def test_malformed_streams_rejected(orc):
    p, leaves, _ = _encode(orc, "mns", 32, 4, 8.0, 128, {})
    words, _, nbits = orc.serialize(leaves, 128, 128, p, True)
    with pytest.raises(ValueError):
        orc.parse(words, nbits - 5, 128, 128, p, True)       # truncated
    bad = words.copy()
    bad[0] ^= 0x3  # first leaf's level field: level 4 at the first cell is valid, so flip to an impossible tiling
    try:
        back, _, _ = orc.parse(bad, nbits, 128, 128, p, True)
        assert not np.array_equal(back.view(np.uint8), leaves.view(np.uint8))
    except ValueError:
        pass


# ---------------------------------------------------------------------------
# Device writer and reader against the oracle

GPU_CASES = list(CASES)  # the paper's 16 -> 2 quadtree included


@pytest.fixture(scope="module")
def fic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    fic.lib()
    return fic


@pytest.mark.gpu
@pytest.mark.parametrize("case", GPU_CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-{c[4]}" for c in GPU_CASES])
@pytest.mark.parametrize("t2", [True, False])
def test_device_bitstream_equals_oracle(fic, orc, case, t2):
    import torch
    mode, bmax, bmin, thr, N, kw = case
    img = synth.gaussian_scene(N, 5)
    op = orc.make_params(mode, bmax, bmin, thr, **kw)
    p = fic.params(mode, bmax, bmin, thr, **kw)
    leaves, split, _ = orc.encode(img, op)
    want_words, want_index, nbits = orc.serialize(leaves, N, N, op, t2)
    st = fic.fic_encode(torch.from_numpy(img).cuda(), p)
    words, index = fic.serialize(st, t2)
    torch.cuda.synchronize()
    idx = index.cpu().numpy().view(np.uint64)
    assert np.array_equal(idx, want_index)
    w = words.cpu().numpy().view(np.uint32)
    nw = (nbits + 31) // 32
    assert np.array_equal(w[:nw], want_words) and not w[nw:].any()
    back = fic.parse(words, index, N, N, p, t2)
    got = back.to_host()
    assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8))
    assert np.array_equal(got["split"], split)
    assert np.array_equal(got["tile_offsets"], st.to_host()["tile_offsets"])
    # the oracle's words read by the device
    back2 = fic.parse(torch.from_numpy(want_words.view(np.int32).copy()).cuda(),
                      torch.from_numpy(want_index.view(np.int64).copy()).cuda(), N, N, p, t2)
    assert np.array_equal(back2.to_host()["records"].view(np.uint8), leaves.view(np.uint8))


@pytest.mark.gpu
def test_device_parse_rejects_malformed(fic, orc):
    import torch
    img = synth.gaussian_scene(128, 9)
    p = fic.params("mns", 32, 4, 8.0)
    st = fic.fic_encode(torch.from_numpy(img).cuda(), p)
    words, index = fic.serialize(st)
    bad_index = index.clone()
    bad_index[1] -= 3  # block 0 ends early: its leaves overrun
    back = fic.parse(words, bad_index, 128, 128, p)
    with pytest.raises(fic.FicError) as e:
        back.info_host()
    assert e.value.code == -2


@pytest.mark.gpu
def test_device_batch_equals_per_stream_and_oracle(fic, orc):
    """Every case's stream written and read back in one batched call (the
    case list mixes modes, quadtrees, codebooks and sizes): words, index and
    records equal the oracle's, and the per-stream calls' results."""
    import torch
    sts, want = [], []
    for (mode, bmax, bmin, thr, N, kw) in CASES:
        img = synth.gaussian_scene(N, 5)
        op = orc.make_params(mode, bmax, bmin, thr, **kw)
        leaves, split, _ = orc.encode(img, op)
        want.append((leaves, split, orc.serialize(leaves, N, N, op, True)))
        sts.append(fic.fic_encode(torch.from_numpy(img).cuda(), fic.params(mode, bmax, bmin, thr, **kw)))
    got = fic.serialize_batch(sts, True)
    back = fic.parse_batch([(w, ix, st.width, st.height, st.params) for (w, ix), st in zip(got, sts)], True)
    torch.cuda.synchronize()
    for (words, index), st, b, (leaves, split, (ww, wi, nbits)) in zip(got, sts, back, want):
        assert np.array_equal(index.cpu().numpy().view(np.uint64), wi)
        w = words.cpu().numpy().view(np.uint32)
        nw = (nbits + 31) // 32
        assert np.array_equal(w[:nw], ww) and not w[nw:].any()
        one_w, one_ix = fic.serialize(st, True)
        assert torch.equal(one_w, words) and torch.equal(one_ix, index)
        h = b.to_host()
        assert np.array_equal(h["records"].view(np.uint8), leaves.view(np.uint8))
        assert np.array_equal(h["split"], split)
