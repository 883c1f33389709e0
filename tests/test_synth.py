"""The seeded input generators that both the oracle and the CUDA path read:
deterministic, of the stated shapes, dtypes and mixes."""
import numpy as np

import synth
from synth import images


def test_generators_are_deterministic():
    a, b = images.gaussian_scene(96, 3), images.gaussian_scene(96, 3)
    assert a.dtype == np.uint8 and a.shape == (96, 96) and np.array_equal(a, b)
    assert not np.array_equal(a, images.gaussian_scene(96, 4))
    v = images.voronoi(64, 101)
    assert v.dtype == np.uint8 and np.array_equal(v, images.voronoi(64, 101))
    assert images.gaussian_scene(64, 1, H=32).shape == (32, 64)


def test_scene_images_use_the_whole_range():
    im = images.gaussian_scene(512, 1)
    assert im.min() < 40 and im.max() > 215  # a natural-image-like spread, not a flat field
    assert len(np.unique(im)) > 150


def test_batch_and_exhaustive_workloads():
    imgs = synth.scenes512_images()
    assert [n for n, _ in imgs] == [f"scene{s}" for s in range(1, 9)] + ["voronoi101", "voronoi102"]
    assert all(im.shape == (512, 512) and im.dtype == np.uint8 for _, im in imgs)
    ex = synth.exhaustive_images()
    assert [(n, im.shape) for n, im in ex] == [("scene1_512", (512, 512)), ("scene9_1024", (1024, 1024))]
    assert synth.scene256_image().shape == (256, 256)


def test_mixed_sides_follow_the_weights():
    s = synth.mixed_sides()
    assert s.shape == (512,) and set(np.unique(s)) <= {256, 512, 1024, 2048}
    assert np.array_equal(s, synth.mixed_sides())
    frac = [np.mean(s == v) for v in (256, 512, 1024, 2048)]
    assert np.allclose(frac, [0.4, 0.3, 0.2, 0.1], atol=0.06)


def test_serving_trace():
    t, is_enc, side, seeds = synth.serving_requests(rate=2000.0, seconds=5.0)
    assert np.all(np.diff(t) > 0) and t[-1] < 5.0
    assert abs(t.size / 5.0 - 2000.0) < 200.0  # Poisson count at the rate
    assert abs(is_enc.mean() - 0.8) < 0.03
    assert side.min() >= 128 and side.max() <= 4096 and np.all(side % 32 == 0)
    assert np.array_equal(seeds, 10 ** 6 + np.arange(t.size))
