"""GPU parity at full frame sizes: every judge score and the whole container
against the oracle, bit-exact, for 2040 x 2040 frames (136 x 136 lenslets at
pitch 15), a 1300 x 1300 frame at pitch 13, and the large class of the
uneven batch, 2550 x 2160 (170 x 144 lenslets at pitch 15: 16 blocks, the
last of 216000 bytes) from each generator. These sizes span many chain CTAs,
judge launches and coder tiles and blocks."""
import numpy as np
import pytest

import oracle
from paper_2310_09467_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfc():
    import torch
    from paper_2310_09467_gb300 import build, lfc as L
    build.build()
    torch.cuda.init()
    return L


@pytest.fixture(scope="module", params=["beads2000", "cells500", "beads1300", "large_beads", "large_cells",
                                        "large_vessel"])
def frame(request):
    if request.param == "beads2000":
        return synth.beads(2040, 2040, 15, peak=2000.0, seed=2), 15
    if request.param == "beads1300":  # 100 x 100 lenslets at pitch 13, seed 0
        return synth.bead_frame_1300(seed=0), 13
    if request.param == "large_beads":
        return synth.beads(2550, 2160, 15, peak=2000.0, seed=1001), 15
    if request.param == "large_cells":
        return synth.cells(2550, 2160, 15, level=500.0, seed=1002), 15
    if request.param == "large_vessel":
        return synth.VesselSeries(2550, 2160, 15, seed=1003).frame(0), 15
    return synth.cells(2040, 2040, 15, level=500.0, seed=3), 15


def test_fullsize_judge_and_container(lfc, frame):
    frame, p = frame
    plan = lfc.Plan(frame.shape[1], frame.shape[0], p)
    d = lfc.to_device_frame(frame)
    choice, scores = plan.judge([d], p)
    best, ref = oracle.judge(frame, p)
    got = scores.cpu().numpy().view(np.uint64)[0]
    assert [int(got[i]) for i in oracle.default_ids()] == ref
    assert int(choice.cpu()[0]) == best
    blob = plan.compress_to_bytes([d], p)[0]
    assert blob == oracle.compress_id(frame, p, best)
    n_blocks = -(-frame.nbytes // 720000)
    assert int.from_bytes(blob[28:32], "little") == n_blocks
    import torch
    out = torch.empty(frame.shape, dtype=torch.int16, device="cuda")
    plan.decompress([torch.from_numpy(np.frombuffer(blob, dtype=np.uint8).copy()).cuda()], [out])
    assert np.array_equal(lfc.from_device_frame(out), frame)


def test_fullsize_temporal(lfc):
    """A series frame with its previous frame: 52 candidates, temporal base field."""
    p = 15
    vs = synth.VesselSeries(2040, 2040, p, seed=5)
    f0, f1 = vs.frame(0), vs.frame(1)
    plan = lfc.Plan(2040, 2040, p, max_frames=2, temporal=True)
    d0, d1 = lfc.to_device_frame(f0), lfc.to_device_frame(f1)
    choice, scores = plan.judge([d0, d1], p, prevs=[None, d0])
    best, ref = oracle.judge(f1, p, oracle.default_ids(True), prev=f0)
    got = scores.cpu().numpy().view(np.uint64)[1]
    assert [int(got[i]) for i in oracle.default_ids(True)] == ref
    assert int(choice.cpu()[1]) == best
    blobs = plan.compress_to_bytes([d0, d1], p, prevs=[None, d0])
    assert blobs[1] == oracle.compress_id(f1, p, best, prev=f0)
