"""GPU parity of the planar byte layout (id bit 3: every high byte of the
stream, then every low byte; Sec. 2.1.2 / Fig. 2c) against the CPU oracle:
entropy scores and choices over the default ids and their planar twins,
containers chosen by the judge or given by the caller, temporal frames and
decoding (the allocation-free judge's planar case is in test_zz_no_alloc.py).
All bit-exact."""
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


def _frames():
    return [
        (synth.beads(195, 195, 13, peak=2000.0, seed=0), 13),
        (synth.cells(210, 195, 15, seed=3), 15),
        (synth.beads(340, 260, 20, peak=500.0, seed=7), 20),   # > 256 output columns per tile
        (synth.cells(96, 102, 3, seed=8), 3),                  # odd widths: scalar store paths
        (synth.beads(480, 240, 15, peak=300.0, seed=13), 15),  # 32 lenslets a row: vector-store paths
    ]


def _ids():
    return sorted(oracle.default_ids() + oracle.planar_ids())


@pytest.mark.parametrize("k", range(5))
def test_judge_and_container_with_planar_ids(lfc, k):
    fr, p = _frames()[k]
    ids = _ids()
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, candidate_ids=ids, block_bytes=20000)
    d = lfc.to_device_frame(fr)
    choice, scores = plan.judge([d], p)
    best, ref = oracle.judge(fr, p, ids)
    got = scores.cpu().numpy().view(np.uint64)[0]
    assert [int(got[i]) for i in ids] == ref
    assert int(choice.cpu()[0]) == best
    blob = plan.compress_to_bytes([d], p)[0]
    assert blob == oracle.compress_id(fr, p, best, block_bytes=20000)
    assert np.array_equal(oracle.decompress(blob), fr)


def test_planar_only_set_and_given_ids(lfc):
    import torch
    fr, p = _frames()[0]
    ids = oracle.planar_ids()
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, max_frames=2, candidate_ids=ids, block_bytes=20000)
    d = lfc.to_device_frame(fr)
    blob = plan.compress_to_bytes([d], p)[0]
    best, _ = oracle.judge(fr, p, ids)
    assert best & 8 and blob == oracle.compress_id(fr, p, best, block_bytes=20000)
    for cid in (0x08, 0x4C, 0x2F, 0x6E):
        choice = torch.tensor([cid, cid], dtype=torch.uint8, device="cuda")
        out, sizes, offs = plan.compress([d, d], p, choice=choice)
        sz, host = sizes.cpu().numpy(), out.cpu().numpy()
        ref = oracle.compress_id(fr, p, cid, block_bytes=20000)
        for i in range(2):
            assert host[offs[i]:offs[i] + sz[i]].tobytes() == ref, (hex(cid), i)


def test_planar_temporal(lfc):
    vs = synth.VesselSeries(180, 180, 15, seed=11)
    frs = [vs.frame(k) for k in range(3)]
    ids = sorted(oracle.default_ids(True) + oracle.planar_ids(True))
    plan = lfc.Plan(180, 180, 15, max_frames=3, temporal=True, candidate_ids=ids, block_bytes=30000)
    ds = [lfc.to_device_frame(x) for x in frs]
    blobs = plan.compress_to_bytes(ds, 15, prevs=[None, ds[0], ds[1]])
    for i, blob in enumerate(blobs):
        pv = frs[i - 1] if i else None
        use = ids if pv is not None else [c for c in ids if not c >> 7]
        best, _ = oracle.judge(frs[i], 15, use, prev=pv)
        assert blob == oracle.compress_id(frs[i], 15, best, prev=pv, block_bytes=30000)


@pytest.mark.parametrize("k", range(5))
def test_decode_planar_containers(lfc, k):
    import torch
    fr, p = _frames()[k]
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, block_bytes=20000)
    for cid in (0x08, 0x4C, 0x2D, 0x6F, 0x5E):
        ref = oracle.compress_id(fr, p, cid, block_bytes=20000)
        out = torch.empty(fr.shape, dtype=torch.int16, device="cuda")
        plan.decompress([torch.from_numpy(np.frombuffer(ref, dtype=np.uint8).copy()).cuda()], [out])
        assert np.array_equal(lfc.from_device_frame(out), fr), hex(cid)

