"""Autotuner cache logic (CPU) and, on a GPU, that every knob setting gives
the same judge results (the knobs change speed only)."""
import json

import numpy as np
import pytest

from paper_2310_09467_gb300 import autotune


def test_batch_key_and_cache_round_trip(tmp_path):
    k1 = autotune.batch_key([(2040, 2040), (1300, 1300), (2040, 2040)], [15, 13, 15], 26, False)
    k2 = autotune.batch_key([(1300, 1300), (2040, 2040), (2040, 2040)], [13, 15, 15], 26, False)
    assert k1 == k2 == "1300x1300p13*1,2040x2040p15*2|K26|T0"
    path = str(tmp_path / "t.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({k1: {"emit_tile_lenslets": 8, "chain_range_bytes": 16384, "judge_frames_per_launch": 2}}, path)
    assert autotune.load_cache(path)[k1]["chain_range_bytes"] == 16384
    open(path, "w").write("not json")
    assert autotune.load_cache(path) == {}
    c = list(autotune.candidates(8))
    assert len(c) == 3 * 4 * 2 and all(set(x) == {"emit_tile_lenslets", "chain_range_bytes",
                                                   "judge_frames_per_launch"} for x in c)


@pytest.mark.gpu
def test_every_knob_setting_gives_the_same_scores(tmp_path):
    from paper_2310_09467_gb300 import build, lfc, synth
    build.build()
    frs = [synth.beads(390, 390, 15, peak=200.0, seed=1), synth.cells(390, 375, 15, seed=2)]
    plan = lfc.Plan(390, 390, 15, max_frames=2)
    ds = [lfc.to_device_frame(f) for f in frs]
    ref_c, ref_s = plan.judge(ds, 15)
    ref_s = ref_s.cpu().numpy().copy()
    for knobs in autotune.candidates(plan.get_tuning()["judge_frames_per_launch"]):
        plan.set_tuning(**knobs)
        c, s = plan.judge(ds, 15)
        assert np.array_equal(s.cpu().numpy(), ref_s), knobs
        assert np.array_equal(c.cpu().numpy(), ref_c.cpu().numpy())
    best, timings = autotune.autotune(plan, ds, 15, path=str(tmp_path / "tune.json"))
    assert best in [t[1] for t in timings]
    assert json.load(open(tmp_path / "tune.json"))
    again, t2 = autotune.autotune(plan, ds, 15, path=str(tmp_path / "tune.json"))
    assert again == best and t2 is None
