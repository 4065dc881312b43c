"""lfc_compress_host: host frames in, host containers out (the call a user
with frames in host memory makes). Its containers equal lfc_compress's and
the oracle's, with the judge, with given ids and with temporal frames."""
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


def _blobs(out, sizes, offs):
    o = out.numpy() if hasattr(out, "numpy") else out
    return [o[offs[i]:offs[i] + int(sizes[i])].tobytes() for i in range(len(offs))]


def test_host_round_trip_matches_device_and_oracle(lfc):
    import torch
    frs = [synth.beads(390, 260, 13, peak=200.0, seed=5), synth.cells(390, 260, 13, seed=6)]
    plan = lfc.Plan(390, 260, 13, max_frames=2, block_bytes=20000)
    host = [torch.from_numpy(f.view(np.int16)).pin_memory() for f in frs]
    out, sizes, offs = plan.compress_host(host, 13)
    got = _blobs(out, sizes, offs)
    dev = plan.compress_to_bytes([lfc.to_device_frame(f) for f in frs], 13)
    assert got == dev
    for f, b in zip(frs, got):
        best, _ = oracle.judge(f, 13)
        assert b == oracle.compress_id(f, 13, best, block_bytes=20000)
    # pageable numpy frames and given ids
    out2, sizes2, offs2 = plan.compress_host(frs, 13, choice=[0x47, 0x6E])
    got2 = _blobs(out2, sizes2, offs2)
    assert got2 == [oracle.compress_id(frs[0], 13, 0x47, block_bytes=20000),
                    oracle.compress_id(frs[1], 13, 0x6E, block_bytes=20000)]


def test_host_temporal(lfc):
    vs = synth.VesselSeries(180, 180, 15, seed=11)
    frs = [vs.frame(k) for k in range(3)]
    plan = lfc.Plan(180, 180, 15, max_frames=3, temporal=True, block_bytes=30000)
    out, sizes, offs = plan.compress_host(frs, 15, prevs=[None, frs[0], frs[1]])
    for i, b in enumerate(_blobs(out, sizes, offs)):
        pv = frs[i - 1] if i else None
        best, _ = oracle.judge(frs[i], 15, prev=pv)
        assert b == oracle.compress_id(frs[i], 15, best, prev=pv, block_bytes=30000)


def test_host_rejects_small_output(lfc):
    import torch
    fr = synth.beads(195, 195, 13, peak=2000.0, seed=0)
    plan = lfc.Plan(195, 195, 13, block_bytes=20000)
    with pytest.raises(lfc.LfcError) as ei:
        plan.compress_host([fr], 13, out=torch.empty(100, dtype=torch.uint8))
    assert ei.value.status == 2  # LFC_ERR_CAPACITY
