"""Host-side arithmetic of bench.py's roofline extras (no GPU)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_chain_smem_bound_arithmetic():
    # 1e9 pair increments in 1 ms on 2 SMs at 1000 MHz: 2e9 wavefronts per second
    r = bench.chain_smem_bound(1e9, 1.0, 2, 1000.0)
    assert r["pair_increments_per_s"] == pytest.approx(1e12)
    assert r["smem_bound_per_s"] == pytest.approx(2e9 / bench.CHAIN_WAVEFRONTS_PER_BYTE)
    assert r["smem_bound_conflict_free_per_s"] == pytest.approx(2e9 * 32 / 3)
    assert r["frac_of_smem_bound"] == pytest.approx(1e12 / r["smem_bound_per_s"])
    # the measured walk needs more wavefronts per byte than the conflict-free three accesses
    assert bench.CHAIN_WAVEFRONTS_PER_BYTE > bench.CHAIN_WAVEFRONTS_PER_BYTE_IDEAL
    assert r["issue_bound_per_s"] == pytest.approx(4 * 2e9 / bench.CHAIN_INSTR_PER_BYTE)
    assert bench.chain_smem_bound(1.0, 0.0, 1, 1.0)["pair_increments_per_s"] == 0.0
