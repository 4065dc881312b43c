"""lfc_judge_noalloc: the allocation-free judge, for callers that may not
allocate device memory (for example an acquisition loop with a device-memory
budget fixed at start-up, or a plug-in whose host framework owns the
allocator). Called through the C ABI, its choice and uint64 scores must equal
those of lfc_judge and of the oracle (exact integer parity, the same bar as
every judge test) on calls in a row; each later call runs on the scratch the
earlier one left behind. Collected last so that a stop at the first failure
has run the rest."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2310_09467_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _frame_struct(lfc, d, shape, p, prev=None):
    arr = (lfc.Frame * 1)()
    arr[0].data = d.data_ptr()
    arr[0].prev = None if prev is None else prev.data_ptr()
    arr[0].height, arr[0].width = shape
    arr[0].pitch = p
    arr[0].reserved = 0
    return arr


def _call(lib, torch, arr, ids):
    ids_c = (ctypes.c_uint8 * len(ids))(*ids)
    choice = torch.full((1,), 255, dtype=torch.uint8, device="cuda")
    scores = torch.zeros(256, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.lfc_judge_noalloc(arr, ids_c, len(ids), ctypes.c_void_p(choice.data_ptr()),
                               ctypes.c_void_p(scores.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    got = scores.cpu().numpy().view(np.uint64)
    return int(choice.cpu()[0]), [int(got[i]) for i in ids]


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
        arr = _frame_struct(lfc, d, fr.shape, p)
        ch, got = _call(lib, torch, arr, ids)
        ref = ref_scores.cpu().numpy().view(np.uint64)[0]
        assert got == [int(ref[i]) for i in ids]
        assert ch == int(ref_choice.cpu()[0])
        plan.close()
    # sizes beyond the stated maximum are rejected before any device work
    choice = torch.full((1,), 255, dtype=torch.uint8, device="cuda")
    for w, h, p in [(15, 4110, 15), (2670, 30, 15)]:
        big = _frame_struct(lfc, d, (h, w), p)
        assert lib.lfc_judge_noalloc(big, ids_c, len(ids), ctypes.c_void_p(choice.data_ptr()), None,
                                     ctypes.c_void_p(stream.cuda_stream)) == 1


def test_noalloc_judge_matches_oracle_at_full_size():
    """2040 x 2040 beads (16 segments of 128 rows), a 2550 x 2160 cell frame
    (170 x 144 lenslets, width near the 2656 limit) and a series frame with
    its previous frame over all 52 ids (temporal ids read the previous
    frame), against the oracle's scores, two calls in a row each."""
    import torch
    from paper_2310_09467_gb300 import build, lfc
    build.build()
    lib = lfc.load()
    vs = synth.VesselSeries(2040, 2040, 15, seed=7)
    f0 = vs.frame(0)
    cases = [(synth.beads(2040, 2040, 15, peak=2000.0, seed=2), None, oracle.default_ids()),
             (synth.cells(2550, 2160, 15, level=500.0, seed=11), None, oracle.default_ids()),
             (vs.frame(1), f0, oracle.default_ids(True))]
    for fr, prev, ids in cases:
        best, ref = oracle.judge(fr, 15, ids, prev=prev)
        d = lfc.to_device_frame(fr)
        dp = None if prev is None else lfc.to_device_frame(prev)
        arr = _frame_struct(lfc, d, fr.shape, 15, dp)
        for _ in range(2):
            ch, got = _call(lib, torch, arr, ids)
            assert got == ref
            assert ch == best


_RESET_SCRIPT = r'''
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2310_09467_gb300 import lfc, synth
lib = lfc.load()
rt = ctypes.CDLL("libcudart.so.13")   # the runtime liblfc is linked against
rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
rt.cudaFree.argtypes = [ctypes.c_void_p]

def ck(rc, what):
    if rc != 0:
        raise SystemExit("%s returned %d" % (what, rc))

fr, p = synth.cells(300, 270, 15, seed=3), 15
ids = oracle.default_ids()
best, ref = oracle.judge(fr, p, ids)
ids_c = (ctypes.c_uint8 * len(ids))(*ids)
for rnd in range(3):
    d, ch, sc = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    ck(rt.cudaMalloc(ctypes.byref(d), fr.nbytes), "cudaMalloc")
    ck(rt.cudaMalloc(ctypes.byref(ch), 16), "cudaMalloc")
    ck(rt.cudaMalloc(ctypes.byref(sc), 256 * 8), "cudaMalloc")
    ck(rt.cudaMemcpy(d, fr.ctypes.data, fr.nbytes, 1), "cudaMemcpy")
    f = lfc.Frame()
    f.data, f.prev, f.width, f.height, f.pitch, f.reserved = d.value, None, fr.shape[1], fr.shape[0], p, 0
    ck(lib.lfc_judge_noalloc(ctypes.byref(f), ids_c, len(ids), ch, sc, None), "lfc_judge_noalloc")
    ck(rt.cudaDeviceSynchronize(), "cudaDeviceSynchronize")
    got = np.zeros(256, dtype=np.uint64)
    c = np.zeros(1, dtype=np.uint8)
    ck(rt.cudaMemcpy(got.ctypes.data, sc, 256 * 8, 2), "cudaMemcpy")
    ck(rt.cudaMemcpy(c.ctypes.data, ch, 1, 2), "cudaMemcpy")
    if [int(got[i]) for i in ids] != ref or int(c[0]) != best:
        raise SystemExit("round %d: scores differ from the oracle" % rnd)
    for ptr in (d, ch, sc):
        ck(rt.cudaFree(ptr), "cudaFree")
    if rnd < 2:
        ck(rt.cudaDeviceReset(), "cudaDeviceReset")   # the next call runs in a new context
print("ok")
'''


def test_noalloc_judge_planar_ids():
    """The default ids and their planar twins (id bit 3: the judged string
    is 2H rows of W high bytes, then W low bytes), against the oracle:
    vector-width and odd-width frames, and 600 rows (5 segments)."""
    import torch
    from paper_2310_09467_gb300 import build, lfc
    build.build()
    lib = lfc.load()
    ids = sorted(oracle.default_ids() + oracle.planar_ids())
    for fr, p in ((synth.beads(195, 195, 13, peak=2000.0, seed=0), 13), (synth.cells(96, 102, 3, seed=8), 3),
                  (synth.beads(300, 600, 15, peak=200.0, seed=21), 15)):
        best, ref = oracle.judge(fr, p, ids)
        d = lfc.to_device_frame(fr)
        ch, got = _call(lib, torch, _frame_struct(lfc, d, fr.shape, p), ids)
        assert got == ref
        assert ch == best


def test_noalloc_judge_after_device_reset():
    """The scratch array is re-created (zeroed, possibly elsewhere) when the
    device's context is: calls after cudaDeviceReset must still find it and
    rebuild its log2 table. Runs in a process of its own that uses the CUDA
    runtime directly (no torch, whose state a reset would invalidate)."""
    from paper_2310_09467_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", _RESET_SCRIPT, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
