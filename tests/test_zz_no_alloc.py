"""lfc_judge_noalloc: the allocation-free judge, for callers that may not
allocate device memory (for example an acquisition loop with a device-memory
budget fixed at start-up, or a plug-in whose host framework owns the
allocator). Called through the C ABI, its choice and uint64 scores must equal
those of lfc_judge (exact integer parity, the same bar as every judge test)
on two calls in a row; the second call runs on the scratch the first left
behind. Collected last so that a stop at the first failure has run the rest."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2310_09467_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_judge_matches_lfc_judge_twice():
    import torch
    from paper_2310_09467_gb300 import build, lfc
    build.build()
    lib = lfc.load()
    stream = torch.cuda.current_stream()
    ids = oracle.default_ids()
    ids_c = (ctypes.c_uint8 * len(ids))(*ids)
    cases = [(synth.beads(195, 195, 13, peak=2000.0, seed=0), 13),
             (synth.cells(300, 270, 15, seed=3), 15)]
    for fr, p in cases:
        d = lfc.to_device_frame(fr)
        plan = lfc.Plan(fr.shape[1], fr.shape[0], p)
        ref_choice, ref_scores = plan.judge([d], p)
        arr = (lfc.Frame * 1)()
        arr[0].data = d.data_ptr()
        arr[0].prev = None
        arr[0].height, arr[0].width = fr.shape
        arr[0].pitch = p
        arr[0].reserved = 0
        choice = torch.full((1,), 255, dtype=torch.uint8, device="cuda")
        scores = torch.zeros(256, dtype=torch.int64, device="cuda")
        rc = lib.lfc_judge_noalloc(arr, ids_c, len(ids), ctypes.c_void_p(choice.data_ptr()),
                                   ctypes.c_void_p(scores.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = scores.cpu().numpy().view(np.uint64)
        ref = ref_scores.cpu().numpy().view(np.uint64)[0]
        assert [int(got[i]) for i in ids] == [int(ref[i]) for i in ids]
        assert int(choice.cpu()[0]) == int(ref_choice.cpu()[0])
        plan.close()
    # sizes beyond the stated maximum are rejected before any device work
    big = (lfc.Frame * 1)()
    big[0].data = d.data_ptr()
    big[0].width, big[0].height, big[0].pitch, big[0].reserved = 15, 4110, 15, 0
    assert lib.lfc_judge_noalloc(big, ids_c, len(ids), ctypes.c_void_p(choice.data_ptr()), None,
                                 ctypes.c_void_p(stream.cuda_stream)) == 1
