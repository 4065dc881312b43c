"""What the trained proposal network gains over the exhaustive judge: trained
by the library's own kernels on frames labelled by the exhaustive judge, on
held-out 2040 x 2040 frames it keeps the compressed size within 0.5 % (top-3)
while compressing more frames per second (top-1)."""
import pytest

from paper_2310_09467_gb300 import synth

pytestmark = pytest.mark.gpu


def test_learned_proposal_keeps_ratio_and_gains_speed():
    from paper_2310_09467_gb300 import build, learn, lfc
    build.build()
    tr = learn.make_frames(synth.training_fields(6, 2, 3, seed0=30000), draws=2, seed0=0)
    te = learn.make_frames(synth.training_fields(2, 1, 1, seed0=40000), draws=1, seed0=900000)
    plan = lfc.Plan(2040, 2040, 15, max_frames=8)
    class_ids = sorted([0x00, 0x40] + [f | (d << 4) | (o << 6) for o in (0, 1) for d in (0, 1, 2) for f in (4, 5, 6, 7)])
    labels = learn.labels_for(plan, tr, 15, class_ids)
    net = lfc.Cnn(len(class_ids), 16, seed=2)
    hist = learn.train(net, tr, labels, 15, epochs=25, batch=16, lr=2e-3)
    assert hist[-1] < 0.6 * hist[0]
    res = learn.evaluate(plan, net, class_ids, te, 15, settings=((1, 0.0), (3, 0.0)), reps=2)
    assert res["top3_tau0.0"]["ratio_loss_pct"] <= 0.5
    assert res["top1_tau0.0"]["speedup"] > 1.05
