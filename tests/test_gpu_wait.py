"""Bounded device waits of the suffix sort's radix passes (each tile waits
for the digit counts of its block's earlier tiles). A fault injected from
the host makes the first tile of the first block never publish its counts:
the block's other tiles then wait on a flag that nothing sets, give up after
the plan's wait budget and the call returns LFC_ERR_TIMEOUT (a status, never
a trap). The plan and the GPU stay usable: the next call's container equals
the oracle's. The same fault in a replayed batch is reported by
lfc_plan_device_status."""
import time

import numpy as np
import pytest

import oracle
from paper_2310_09467_gb300 import synth

pytestmark = pytest.mark.gpu

W = H = 1020  # 2 MB: blocks of 720000 bytes, each many 4096-element tiles
P = 15


@pytest.fixture(scope="module")
def L():
    from paper_2310_09467_gb300 import build, lfc
    build.build()
    return lfc


def test_sort_wait_gives_up_and_plan_recovers(L):
    fr = synth.beads(W, H, P, peak=2000.0, seed=5)
    plan = L.Plan(W, H, P)
    plan.set_tuning(wait_budget_ms=200)
    assert plan.get_tuning()["wait_budget_ms"] == 200
    d = L.to_device_frame(fr)
    plan.inject_fault(1)
    t0 = time.time()
    with pytest.raises(L.LfcError) as ei:
        plan.compress_to_bytes([d], P)
    assert ei.value.status == 5  # LFC_ERR_TIMEOUT
    assert time.time() - t0 < 60
    assert plan.device_status() == 5  # the sticky word saw it too; reading clears it
    assert plan.device_status() == 0
    best, _ = oracle.judge(fr, P)
    ref = oracle.compress_id(fr, P, best)
    for _ in range(2):
        assert plan.compress_to_bytes([d], P)[0] == ref
    plan.close()


def test_batch_wait_timeout_reported_by_device_status(L):
    import torch
    fr = synth.cells(W, H, P, level=500.0, seed=6)
    plan = L.Plan(W, H, P)
    plan.set_tuning(wait_budget_ms=200)
    d = L.to_device_frame(fr)
    batch = plan.batch([d], P)
    plan.inject_fault(1)
    batch.launch()
    assert plan.device_status() == 5
    batch.launch()
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    best, _ = oracle.judge(fr, P)
    assert batch.to_bytes()[0] == oracle.compress_id(fr, P, best)
    batch.close()
    plan.close()
