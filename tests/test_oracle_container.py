"""Oracle container: lossless round trip (Supp. S2 claim, Sec. 3), header
with the 8-bit predictor id (Sec. 2.1.4), block split (Sec. 2.1.3), temporal
frames, and host-side fault injection (flipped and truncated bytes)."""
import bz2
import struct

import numpy as np
import pytest

import oracle
from paper_2310_09467_gb300 import synth


def _frames():
    return [
        (synth.beads(195, 195, 13, peak=2000.0, seed=0), 13),
        (synth.beads(150, 135, 15, peak=20.0, seed=1), 15),
        (synth.cells(210, 195, 15, seed=3), 15),
    ]


@pytest.mark.parametrize("k", range(3))
def test_round_trip_and_streams(k):
    fr, p = _frames()[k]
    blob, cid = oracle.compress(fr, p, block_bytes=20000)
    W, H, pp, cid2 = oracle.container_info(blob)
    assert (W, H, pp, cid2) == (fr.shape[1], fr.shape[0], p, cid)
    assert np.array_equal(oracle.decompress(blob), fr)
    # every block is a standalone bzip2 stream of the chosen symbol stream
    nb = struct.unpack_from("<I", blob, 28)[0]
    sizes = struct.unpack_from("<%dI" % nb, blob, 40)
    S = oracle.stream_bytes(oracle.symbols(fr, p, cid)).tobytes()
    o = 40 + 4 * nb
    got = b""
    for s in sizes:
        got += bz2.decompress(blob[o:o + s])
        o += s
    assert got == S and o == len(blob)


def test_temporal_round_trip():
    vs = synth.VesselSeries(180, 180, 15, seed=4)
    f0, f1 = vs.frame(0), vs.frame(1)
    blob, cid = oracle.compress(f1, 15, prev=f0, block_bytes=30000)
    assert np.array_equal(oracle.decompress(blob, prev=f0), f1)
    for c in oracle.default_ids(True):
        if c >> 7:
            b = oracle.compress_id(f1, 15, c, prev=f0, block_bytes=30000)
            assert np.array_equal(oracle.decompress(b, prev=f0), f1)


def test_fault_injection_detected():
    fr, p = _frames()[1]
    blob = oracle.compress_id(fr, p, 0x47, block_bytes=20000)
    rng = np.random.default_rng(0)
    for pos in list(rng.integers(40, len(blob), 25)) + [0, 8, 20, 28, 36]:
        t = bytearray(blob)
        t[pos] ^= 1 << int(rng.integers(0, 8))
        try:
            out = oracle.decompress(bytes(t))
        except ValueError:
            continue
        # a flip that still decodes may only touch padding bits
        assert np.array_equal(out, fr), "undetected corruption at %d" % pos
    with pytest.raises(ValueError):
        oracle.decompress(blob[: len(blob) - 10])


def _payload(blob):
    """Concatenated block payloads, each decoded by the stock bzip2 decoder."""
    nb = struct.unpack_from("<I", blob, 28)[0]
    sizes = struct.unpack_from("<%dI" % nb, blob, 40)
    o = 40 + 4 * nb
    got = b""
    for s in sizes:
        got += bz2.decompress(blob[o:o + s])
        o += s
    return got


def _planes(z):
    z = np.asarray(z, dtype=np.uint16).ravel()
    return (z >> 8).astype(np.uint8).tobytes() + (z & 0xFF).astype(np.uint8).tobytes()


def test_planar_layout_codes_the_byte_planes():
    """Id bit 3 (Fig. 2c: each 16-bit value split into its high and low 8
    bits): the coded string is every high byte in stream order, then every
    low byte. Without prediction those are the frame's own byte planes; the
    (lo, hi) layout codes the frame's little-endian bytes."""
    fr, p = _frames()[0]
    X = fr.astype(np.uint16).ravel()
    blob = oracle.compress_id(fr, p, oracle.make_id(0, planar=1), block_bytes=20000)
    assert _payload(blob) == _planes(X)
    assert np.array_equal(oracle.decompress(blob), fr)
    blob0 = oracle.compress_id(fr, p, 0, block_bytes=20000)
    assert _payload(blob0) == X.astype("<u2").tobytes()
    # view-major raw symbols are the frame's pixels in mosaic order
    Nx, Ny = fr.shape[1] // p, fr.shape[0] // p
    mosaic = fr.reshape(Ny, p, Nx, p).transpose(1, 0, 3, 2).reshape(fr.shape)
    blobv = oracle.compress_id(fr, p, oracle.make_id(0, ordering=1, planar=1), block_bytes=20000)
    assert _payload(blobv) == _planes(mosaic)


@pytest.mark.parametrize("k", range(3))
def test_planar_predicted_round_trip(k):
    """A predicted planar id codes the planes of the same symbols as its
    (lo, hi) twin, and decodes back to the frame."""
    fr, p = _frames()[k]
    for cid in (oracle.make_id(5, 2, 1), oracle.make_id(7, 1, 0), oracle.make_id(4, 0, 1)):
        z = oracle.symbols(fr, p, cid)
        assert np.array_equal(oracle.symbols(fr, p, cid | 8), z)
        blob = oracle.compress_id(fr, p, cid | 8, block_bytes=20000)
        assert oracle.container_info(blob)[3] == cid | 8
        assert _payload(blob) == _planes(z)
        assert np.array_equal(oracle.decompress(blob), fr)


def test_planar_temporal_round_trip():
    vs = synth.VesselSeries(180, 180, 15, seed=4)
    f0, f1 = vs.frame(0), vs.frame(1)
    for cid in (oracle.make_id(0, temporal=1, planar=1), oracle.make_id(6, 2, 1, temporal=1, planar=1)):
        b = oracle.compress_id(f1, 15, cid, prev=f0, block_bytes=30000)
        assert np.array_equal(oracle.decompress(b, prev=f0), f1)


def test_realign_inverse_and_ids():
    z = np.random.default_rng(5).integers(0, 65536, 1001).astype(np.uint16)
    for planar in (False, True):
        assert np.array_equal(oracle.unrealign(oracle.stream_bytes(z, planar), planar), z)
    assert oracle.stream_bytes(z, True).tobytes() == _planes(z)
    assert all(oracle.id_valid(c) for c in oracle.planar_ids(True))
    assert not oracle.id_valid(oracle.make_id(0, 1, planar=1))  # f = 0 stays in domain 0
