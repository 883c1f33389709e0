"""The oracle against the numbers the paper prints (tests/golden/paper_values.json,
each entry with its section)."""
import json
import os
from fractions import Fraction as F

import numpy as np
import pytest

import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def round_half_up(x):
    return (F(x) + F(1, 2)).__floor__()


@pytest.mark.parametrize("case", GOLD["pool_counts"]["cases"])
def test_pool_counts(orc, case):
    N, n = case["N"], case["n"]
    assert orc.count_ranges(N, N, n) == case["ranges"]
    assert orc.count_domains(N, N, n, 1) == case["domains"]


def test_local_candidates(orc):
    g = GOLD["local_candidates"]
    b = g["range_side"]
    img = synth.gaussian_scene(256, 4)
    p = orc.make_params("local", b, b, 8.0)
    assert orc.count_candidates(img, p, 128, 128, b) == g["count"]


@pytest.mark.parametrize("level", ["1", "2", "3"])
def test_phase2_contrast_sets(orc, level):
    lo, hi = GOLD["phase2_contrast_sets"]["levels"][level]
    lv = int(level)
    # fixed point c = round(128 s)
    assert orc.phase2_contrast(lv, 0) == round_half_up(F(str(lo)) * 128)
    assert orc.phase2_contrast(lv, 1) == round_half_up(F(str(hi)) * 128)


@pytest.mark.parametrize("level", ["1", "2", "3"])
def test_phase2_difference_bits(orc, level):
    assert orc.phase2_mbits(int(level)) == GOLD["phase2_difference_bits"]["levels"][level]


def test_phase1_bits(orc):
    g = GOLD["phase1_bits"]
    p = orc.make_params("mns", 16, 2, 8.0, s_bits=g["s_bits"], o_bits=g["o_bits"])
    lv = np.zeros(1, dtype=orc.LEAF_DTYPE)
    lv[0]["level"], lv[0]["phase"] = 1, 1
    assert orc.bits(lv, 64, 64, p) == g["total"]


def _last_level_groups(orc, groups, W):
    lv = np.zeros(4 * groups, dtype=orc.LEAF_DTYPE)
    per_row = W // 8
    for gi in range(groups):
        gx, gy = (gi % per_row) * 8, (gi // per_row) * 8
        for c in range(4):
            lv[4 * gi + c]["x"], lv[4 * gi + c]["y"] = gx + (c & 1) * 4, gy + (c >> 1) * 4
            lv[4 * gi + c]["level"], lv[4 * gi + c]["phase"] = 4, 1
    return lv


def test_technique2_lena(orc):
    g = GOLD["technique2_lena"]
    p = orc.make_params("mns", 32, 4, 8.0)
    lv = _last_level_groups(orc, g["leaves"] // 4, 1024)
    payload = g["leaves"] * (5 + 7)
    assert orc.bits(lv, 1024, 1024, p, technique2=False) - payload == g["bits_without"]
    assert orc.bits(lv, 1024, 1024, p, technique2=True) - payload == g["bits_with"]


def test_technique2_baboon(orc):
    g = GOLD["technique2_baboon"]
    p = orc.make_params("mns", 32, 4, 8.0)
    lv = _last_level_groups(orc, g["leaves"] // 4, 2048)
    payload = g["leaves"] * (5 + 7)
    assert (orc.bits(lv, 2048, 2048, p, technique2=False) - payload) / 8 == g["bytes_without"]
    with_t2 = (orc.bits(lv, 2048, 2048, p, technique2=True) - payload) / 8
    assert abs(with_t2 - g["bytes_with_approx"]) / g["bytes_with_approx"] < 0.05


def test_compression_ratio_arithmetic():
    g = GOLD["compression_ratio_baboon"]
    # kbytes = image bytes / ratio / 1024, as printed (rounded to the paper's precision)
    assert round(g["image_bytes"] / g["ratio_nosearch"] / 1024) == g["kbytes_nosearch"]
    assert abs(g["image_bytes"] / g["ratio_mns"] / 1024 - g["kbytes_mns"]) < 0.5
