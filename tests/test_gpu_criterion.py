"""Quality of the entropy criterion on 2040 x 2040 frames of the benchmark's
kinds (the paper's Sec. 3 claim that the criterion of Eq. (1) picks the
predictor with the best compression ratio, Fig. 4b-4d). Every default id is
compressed for real by the library. Measured facts guarded here:
  * on the cell field, where prediction helps, the judge picks the smallest
    container exactly;
  * on every frame the judge's ranking of the 26 ids agrees with the true
    container sizes (Spearman >= 0.5) and its pick is within 10 % of the
    smallest container (on bead frames, where no prediction is best, the
    judge still picks a predictor: the paper's claim is not reproduced there);
  * the judge's pick equals that of the same bigram entropy taken on the real
    BWT of each block (the full-BWT judge) or is within 1 % of it in size, so
    the first-byte sort of Sec. 2.1.2 is not what costs the ratio."""
import pytest

from paper_2310_09467_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2310_09467_gb300 import build, lfc
    build.build()
    return lfc


@pytest.mark.parametrize("kind", ["beads2000", "cells500", "vessel300"])
def test_judge_pick_against_true_sizes(L, kind):
    from paper_2310_09467_gb300 import criterion
    W = H = 2040
    p = 15
    if kind == "beads2000":
        fr = synth.beads(W, H, p, peak=2000.0, seed=103)
    elif kind == "cells500":
        fr = synth.cells(W, H, p, level=500.0, seed=104)
    else:
        fr = synth.VesselSeries(W, H, p, seed=105).frame(0)
    plan = L.Plan(W, H, p)
    res = criterion.study_frame(plan, L, fr, p, L.default_ids())
    s = criterion.summarize(res, fr.nbytes)
    if kind == "cells500":
        assert s["judge_pick"] == s["true_pick"]
    assert s["spearman_judge_vs_size"] >= 0.5
    assert s["judge_gap_pct"] <= 10.0
    sizes = dict(zip(res["ids"], res["sizes"]))
    assert sizes[s["judge_pick"]] <= 1.01 * sizes[s["full_bwt_pick"]]
    plan.close()
