"""Launch mappings of the batched kernels: every mapping the autotuner may
pick writes the same streams and images (equal to the oracle), and the
autotuner keeps one of its candidates."""
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


@pytest.fixture(scope="module")
def batch(orc):
    """Mixed sizes like the batched workload (sides 256..1024), with the
    oracle's streams and 8-iteration decodes."""
    sides = [256, 512, 1024, 256, 512, 256]
    imgs = [synth.gaussian_scene(s, 1000 + i) for i, s in enumerate(sides)]
    op = orc.make_params("mns", 32, 4, 8.0)
    want = []
    for im in imgs:
        leaves, split, fits = orc.encode(im, op)
        want.append((leaves, split, orc.decode(leaves, im.shape[1], im.shape[0], op, 8)))
    return imgs, want


def _check(fic, plan, dplan, want):
    torch.cuda.synchronize()
    for st, dec, (leaves, split, img) in zip(plan.outs, dplan.outs, want):
        got = st.to_host()
        assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8))
        assert np.array_equal(got["split"], split)
        assert np.array_equal(dec.cpu().numpy(), img)


def test_every_mapping_gives_the_same_output(fic, batch):
    imgs, want = batch
    p = fic.params("mns", 32, 4, 8.0)
    plan = fic.EncodePlan([torch.from_numpy(im).cuda() for im in imgs], p)
    plan.run()
    dplan = fic.DecodePlan(plan.outs)
    for warps, kmax in ((8, 3), (4, 4)):
        for k in range(0, kmax + 1):
            for dyn, fp in ((0, 0), (1, 0), (0, 1), (1, 1)):
                plan.set_tuning(enc_warps=warps, enc_ctas_per_sm=k, enc_dynamic=dyn, enc_fused_pack=fp)
                for st in plan.outs:  # stale results must not survive
                    st.records.zero_()
                plan.run()
                plan.run()  # the dynamic counter is reset between runs
                dplan.set_tuning(dec_ctas_per_sm=1 + (k % 4), dec_single_launch=(k + dyn) % 2)
                dplan.run(8)
                _check(fic, plan, dplan, want)


def test_autotune_picks_a_candidate_and_stays_exact(fic, batch):
    imgs, want = batch
    p = fic.params("mns", 32, 4, 8.0)
    plan = fic.EncodePlan([torch.from_numpy(im).cuda() for im in imgs], p)
    res = plan.autotune(reps=3)
    assert len(res["trials"]) == 2 * 2 * 3 + 2 * 2 * 4
    assert res["best"] == plan.tuning
    assert res["best_ms"] == pytest.approx(min(t["ms"] for t in res["trials"]), rel=1e-4)
    dplan = fic.DecodePlan(plan.outs)
    dres = dplan.autotune(8, reps=3)
    assert len(dres["trials"]) == 8 and 1 <= dres["best"]["dec_ctas_per_sm"] <= 4
    assert {t["dec_single_launch"] for t in dres["trials"]} == {0, 1}
    plan.run()
    dplan.run(8)
    _check(fic, plan, dplan, want)


def test_bad_tuning_rejected(fic):
    img = torch.from_numpy(synth.gaussian_scene(128, 3)).cuda()
    plan = fic.EncodePlan([img], fic.params("mns", 32, 4, 8.0))
    with pytest.raises(fic.FicError):
        plan.set_tuning(enc_warps=6)
    with pytest.raises(fic.FicError):
        plan.set_tuning(enc_dynamic=2)
    with pytest.raises(fic.FicError):
        plan.set_tuning(dec_single_launch=2)
    lplan = fic.EncodePlan([img], fic.params("local", 32, 4, 8.0))
    with pytest.raises(fic.FicError):
        lplan.autotune()
