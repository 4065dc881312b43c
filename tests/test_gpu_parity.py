"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

All of the path is integer work, so every comparison is bit-exact: symbol
streams, uint64 entropy scores, chosen ids, bzip2 stream bytes and whole
containers. Sizes span several tiles, CTAs and blocks with ragged tails.
"""
import bz2

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
        (synth.beads(150, 135, 15, peak=20.0, seed=1), 15),
        (synth.cells(210, 195, 15, seed=3), 15),
        (synth.beads(390, 260, 13, peak=200.0, seed=5), 13),
        (synth.beads(340, 260, 20, peak=500.0, seed=7), 20),   # 340 output columns per 17-lenslet row: > 256 threads
        (synth.cells(96, 102, 3, seed=8), 3),
        (synth.beads(480, 240, 15, peak=300.0, seed=13), 15),  # 32 lenslets a row: vector-store paths
    ]


def test_symbols_all_ids(lfc):
    rng = np.random.default_rng(0)
    p = 5
    fr = rng.integers(0, 65536, (7 * p, 9 * p), dtype=np.uint16)
    fr[0, :3] = [0, 65535, 0]
    prev = rng.integers(0, 65536, fr.shape, dtype=np.uint16)
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, temporal=True)
    d, dp = lfc.to_device_frame(fr), lfc.to_device_frame(prev)
    for cid in range(256):
        if not oracle.id_valid(cid):
            continue
        pv = prev if cid >> 7 else None
        got = plan.symbols(d, p, cid, prev=dp if pv is not None else None).cpu().numpy().view(np.uint16)
        assert np.array_equal(got, oracle.symbols(fr, p, cid, prev=pv)), cid


@pytest.mark.parametrize("k", range(7))
def test_judge_scores_and_choice(lfc, k):
    fr, p = _frames()[k]
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p)
    choice, scores = plan.judge([lfc.to_device_frame(fr)], p)
    ids = oracle.default_ids()
    best, ref = oracle.judge(fr, p, ids)
    got = scores.cpu().numpy().view(np.uint64)[0]
    assert [int(got[i]) for i in ids] == ref
    assert int(choice.cpu()[0]) == best


def test_judge_batch_uneven_and_temporal(lfc):
    vs = synth.VesselSeries(180, 165, 15, seed=4)
    f0, f1 = vs.frame(0), vs.frame(1)
    other = synth.beads(195, 195, 13, peak=2000.0, seed=9)
    plan = lfc.Plan(195, 195, 13, max_frames=3, temporal=True)
    ds = [lfc.to_device_frame(x) for x in (f0, f1, other)]
    pitches = [15, 15, 13]
    choice, scores = plan.judge(ds, pitches, prevs=[None, ds[0], None])
    sc = scores.cpu().numpy().view(np.uint64)
    ch = choice.cpu().numpy()
    for i, (fr, pv, p) in enumerate([(f0, None, 15), (f1, f0, 15), (other, None, 13)]):
        ids = oracle.default_ids(pv is not None)
        best, ref = oracle.judge(fr, p, ids, prev=pv)
        assert [int(sc[i][c]) for c in ids] == ref, i
        assert int(ch[i]) == best


def _coder_inputs():
    rng = np.random.default_rng(7)
    yield [b"a"]
    yield [b"ab", b"abab" * 3, b"\x00" * 1000, bytes(range(256)) * 3]
    yield [bytes(rng.integers(0, 256, 5000, dtype=np.uint8)), bytes(rng.integers(0, 3, 70001, dtype=np.uint8))]
    yield [bytes(np.repeat(rng.integers(0, 256, 3000, dtype=np.uint8), rng.integers(1, 300, 3000))[:300000])]
    yield [b"aaaabbbb" * 90000]                                   # 720000 -> 900000 after RLE1
    yield [bytes(rng.integers(0, 256, 720000, dtype=np.uint8)), b"xyz" * 240000]
    yield [bytes(rng.integers(0, 2, 250000, dtype=np.uint8) * 255)]
    # last columns b^8192 a^8192 and z^8192 x^8192 y^8192: zero MTF runs that fill whole
    # 4096-position tiles and end exactly at a tile boundary
    yield [b"ab" * 8192, b"xyz" * 8192]
    # input runs filling whole RLE1 tiles and ending on tile boundaries
    yield [b"a" * 8192 + b"b" * 5000 + b"c" * 4096 + bytes(range(256)) * 4, b"\x07" * 12288]


@pytest.mark.parametrize("case", range(9))
def test_bzip2_encode_bytes_identical(lfc, case):
    blocks = list(_coder_inputs())[case]
    plan = lfc.Plan(195, 195, 13, max_frames=4)
    got = plan.bzip2_encode_bytes(blocks)
    for g, b in zip(got, blocks):
        assert g == oracle.bz2_stream(b)
        assert bz2.decompress(g) == b


@pytest.mark.parametrize("case", range(9))
def test_bwt_blocks_identical(lfc, case):
    """lfc_bwt_blocks: the coder's RLE1 + full rotation sort on its own, last
    column and origin row of every block equal to the oracle's."""
    import torch
    blocks = list(_coder_inputs())[case]
    plan = lfc.Plan(195, 195, 13, max_frames=4)
    buf = b"".join(blocks)
    data = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda()
    offs = np.cumsum([0] + [len(b) for b in blocks])[:-1]
    L, ln, orig = plan.bwt_blocks(data, offs, [len(b) for b in blocks])
    L, ln, orig = L.cpu().numpy(), ln.cpu().numpy(), orig.cpu().numpy()
    for i, b in enumerate(blocks):
        r = oracle.rle1(b)
        refL, refo = oracle.bwt(r)
        assert int(ln[i]) == r.size
        assert np.array_equal(L[i, :r.size], refL)
        assert int(orig[i]) == refo


@pytest.mark.parametrize("k", range(7))
def test_compress_container_identical(lfc, k):
    fr, p = _frames()[k]
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, block_bytes=20000)
    blob = plan.compress_to_bytes([lfc.to_device_frame(fr)], p)[0]
    best, _ = oracle.judge(fr, p)
    assert blob == oracle.compress_id(fr, p, best, block_bytes=20000)
    assert np.array_equal(oracle.decompress(blob), fr)


def test_compress_batch_temporal(lfc):
    vs = synth.VesselSeries(180, 180, 15, seed=11)
    frs = [vs.frame(k) for k in range(3)]
    plan = lfc.Plan(180, 180, 15, max_frames=3, temporal=True, block_bytes=30000)
    ds = [lfc.to_device_frame(x) for x in frs]
    blobs = plan.compress_to_bytes(ds, 15, prevs=[None, ds[0], ds[1]])
    for i, blob in enumerate(blobs):
        pv = frs[i - 1] if i else None
        best, _ = oracle.judge(frs[i], 15, prev=pv)
        assert blob == oracle.compress_id(frs[i], 15, best, prev=pv, block_bytes=30000)
        assert np.array_equal(oracle.decompress(blob, prev=pv), frs[i])


def _dev_bytes(blob):
    import torch
    return torch.from_numpy(np.frombuffer(blob, dtype=np.uint8).copy()).cuda()


@pytest.mark.parametrize("k", range(7))
def test_decompress_round_trip(lfc, k):
    import torch
    fr, p = _frames()[k]
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, block_bytes=20000)
    blob = plan.compress_to_bytes([lfc.to_device_frame(fr)], p)[0]
    out = torch.empty(fr.shape, dtype=torch.int16, device="cuda")
    plan.decompress([_dev_bytes(blob)], [out])
    assert np.array_equal(lfc.from_device_frame(out), fr)
    # the GPU decoder also reads the oracle's containers of every id
    for cid in (0, 0x44, 0x27, 0x66):
        ref = oracle.compress_id(fr, p, cid, block_bytes=20000)
        out2 = torch.empty(fr.shape, dtype=torch.int16, device="cuda")
        plan.decompress([_dev_bytes(ref)], [out2])
        assert np.array_equal(lfc.from_device_frame(out2), fr), cid


def test_decompress_temporal_chain(lfc):
    import torch
    vs = synth.VesselSeries(180, 180, 15, seed=12)
    frs = [vs.frame(k) for k in range(3)]
    plan = lfc.Plan(180, 180, 15, max_frames=3, temporal=True, block_bytes=30000)
    ds = [lfc.to_device_frame(x) for x in frs]
    blobs = plan.compress_to_bytes(ds, 15, prevs=[None, ds[0], ds[1]])
    outs = [torch.empty(frs[0].shape, dtype=torch.int16, device="cuda") for _ in range(3)]
    plan.decompress([_dev_bytes(b) for b in blobs], outs, prevs=[None, outs[0], outs[1]])
    for o, f in zip(outs, frs):
        assert np.array_equal(lfc.from_device_frame(o), f)


def test_decompress_rejects_corruption(lfc):
    """Host-side fault injection: flipped and truncated bytes give CORRUPT
    (or, for a flip in padding bits, the exact frame), never a fault."""
    import torch
    fr, p = _frames()[1]
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, block_bytes=20000)
    blob = plan.compress_to_bytes([lfc.to_device_frame(fr)], p)[0]
    rng = np.random.default_rng(3)
    for pos in list(rng.integers(0, len(blob), 40)) + [0, 8, 12, 20, 24, 28, 32, 36, 40, 44]:
        t = bytearray(blob)
        t[pos] ^= 1 << int(rng.integers(0, 8))
        out = torch.zeros(fr.shape, dtype=torch.int16, device="cuda")
        try:
            plan.decompress([_dev_bytes(bytes(t))], [out])
        except lfc.LfcError as e:
            assert e.status in (1, 2, 3), e
            continue
        assert np.array_equal(lfc.from_device_frame(out), fr), pos
    out = torch.zeros(fr.shape, dtype=torch.int16, device="cuda")
    with pytest.raises(lfc.LfcError):
        plan.decompress([_dev_bytes(blob[:-7])], [out])
    small = torch.zeros(10, dtype=torch.int16, device="cuda")
    with pytest.raises(lfc.LfcError) as ei:
        plan.decompress([_dev_bytes(blob)], [small])
    assert ei.value.status == 2


def test_compress_given_choice(lfc):
    """Caller-chosen ids skip the judge: the chosen stream is emitted directly."""
    import torch
    fr, p = _frames()[0]
    plan = lfc.Plan(fr.shape[1], fr.shape[0], p, max_frames=2, block_bytes=20000)
    d = lfc.to_device_frame(fr)
    for cid in (0x00, 0x44, 0x27):
        choice = torch.tensor([cid, cid], dtype=torch.uint8, device="cuda")
        out, sizes, offs = plan.compress([d, d], p, choice=choice)
        sz, host = sizes.cpu().numpy(), out.cpu().numpy()
        ref = oracle.compress_id(fr, p, cid, block_bytes=20000)
        for i in range(2):
            assert host[offs[i]:offs[i] + sz[i]].tobytes() == ref, (cid, i)
