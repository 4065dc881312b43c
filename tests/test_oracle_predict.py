"""Oracle pins for the prediction part (Sec. 2.1.1) and the orderings.

Pins: hand-computed lossless-JPEG values (tests/golden/predictor_2x2.txt),
closed-form residuals on planes and lenslet-periodic frames, the sub-aperture
mosaic property of the view-major ordering, and exact round trips.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "predictor_2x2.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([int(v) for v in line.split()])
    return out


@pytest.mark.parametrize("row", _rows())
def test_jpeg_predictor_golden(row):
    A, B, C, X, f, _pred, sym = row
    frame = np.array([[C, B], [A, X]], dtype=np.uint16)
    z = oracle.symbols(frame, 2, oracle.make_id(f, 0, 0, 0))
    assert int(z[3]) == sym
    # boundary rule: origin predicts 0, first row from the left, first column from the top
    def zz(d):
        d = ((d + 32768) % 65536) - 32768
        return 2 * d if d >= 0 else -2 * d - 1
    assert int(z[0]) == zz(C)
    assert int(z[1]) == zz(B - C)
    assert int(z[2]) == zz(A - C)


def test_none_is_raw():
    rng = np.random.default_rng(1)
    fr = rng.integers(0, 65536, (12, 18), dtype=np.uint16)
    assert np.array_equal(oracle.symbols(fr, 3, 0), fr.ravel())


@pytest.mark.parametrize("p", [3, 5])
def test_view_major_is_subaperture_mosaic(p):
    rng = np.random.default_rng(p)
    Ny, Nx = 4, 6
    fr = rng.integers(0, 65536, (Ny * p, Nx * p), dtype=np.uint16)
    z = oracle.symbols(fr, p, oracle.make_id(0, 0, 1, 0)).reshape(Ny * p, Nx * p)
    for v in range(p):
        for u in range(p):
            tile = z[v * Ny:(v + 1) * Ny, u * Nx:(u + 1) * Nx]
            assert np.array_equal(tile, fr[v::p, u::p])  # sub-aperture image of view (u, v)
    assert np.array_equal(np.sort(z.ravel()), np.sort(fr.ravel()))


def _zz(d):
    d = ((np.asarray(d, dtype=np.int64) + 32768) % 65536) - 32768
    return np.where(d >= 0, 2 * d, -2 * d - 1)


@pytest.mark.parametrize("f", [4, 5, 6, 7])
def test_intra_constant_frame(f):
    p, c = 5, 1234
    fr = np.full((3 * p, 4 * p), c, dtype=np.uint16)
    z = oracle.symbols(fr, p, oracle.make_id(f, 0, 0, 0)).reshape(fr.shape)
    exp = np.zeros(fr.shape, dtype=np.int64)
    exp[::p, ::p] = 2 * c  # lenslet origins predict 0
    assert np.array_equal(z, exp)


def test_intra_plane_exact_for_a_plus_b_minus_c():
    p = 6
    y, x = np.mgrid[0:3 * p, 0:2 * p]
    fr = (1000 + 7 * (x % p) + 3 * (y % p)).astype(np.uint16)
    z = oracle.symbols(fr, p, oracle.make_id(4, 0, 0, 0)).reshape(fr.shape)
    v, u = y % p, x % p
    exp = np.where((v == 0) & (u == 0), _zz(fr.astype(np.int64)),
                   np.where(v == 0, _zz(7), np.where(u == 0, _zz(3), 0)))
    assert np.array_equal(z, exp)


@pytest.mark.parametrize("f", [4, 5, 6, 7])
def test_inter_periodic_frame(f):
    p = 4
    rng = np.random.default_rng(f)
    lens = rng.integers(0, 65536, (p, p), dtype=np.uint16)
    fr = np.tile(lens, (3, 5))
    z = oracle.symbols(fr, p, oracle.make_id(f, 1, 0, 0)).reshape(fr.shape)
    exp = np.zeros(fr.shape, dtype=np.int64)
    exp[:p, :p] = _zz(lens.astype(np.int64))  # first lenslet predicts 0
    assert np.array_equal(z, exp)


@pytest.mark.parametrize("f", [4, 5, 6, 7])
def test_phase_periodic_frame(f):
    """Identical lenslets: the intra residual field is lenslet-periodic, so the
    second (inter) stage leaves only the first lenslet's intra residuals."""
    p = 4
    rng = np.random.default_rng(10 + f)
    lens = rng.integers(0, 65536, (p, p), dtype=np.uint16)
    fr = np.tile(lens, (3, 4))
    zp = oracle.symbols(fr, p, oracle.make_id(f, 2, 0, 0)).reshape(fr.shape)
    zi = oracle.symbols(fr, p, oracle.make_id(f, 0, 0, 0)).reshape(fr.shape)
    exp = np.zeros(fr.shape, dtype=zi.dtype)
    exp[:p, :p] = zi[:p, :p]
    assert np.array_equal(zp, exp)


def test_temporal_zero_motion():
    p = 3
    rng = np.random.default_rng(5)
    prev = rng.integers(0, 65536, (2 * p, 3 * p), dtype=np.uint16)
    for f, d in [(0, 0), (4, 0), (5, 1), (7, 2)]:
        z = oracle.symbols(prev, p, oracle.make_id(f, d, 0, 1), prev=prev)
        assert not z.any()
    # pure temporal, f = 0: symbol is the zigzagged frame difference
    cur = rng.integers(0, 65536, prev.shape, dtype=np.uint16)
    z = oracle.symbols(cur, p, oracle.make_id(0, 0, 0, 1), prev=prev)
    assert np.array_equal(z, _zz(cur.astype(np.int64) - prev.astype(np.int64)).ravel())


def test_invalid_ids_rejected():
    assert not oracle.id_valid(0x10)   # f = 0 needs domain 0
    assert not oracle.id_valid(0x08)   # f = 8 undefined
    assert not oracle.id_valid(0x34)   # domain 3 undefined
    assert len(oracle.default_ids()) == 26
    assert len(oracle.default_ids(True)) == 52
    assert all(oracle.id_valid(i) for i in oracle.default_ids(True))


@pytest.mark.parametrize("p,Ny,Nx", [(3, 4, 5), (5, 3, 3), (13, 2, 3)])
def test_round_trip_all_ids(p, Ny, Nx):
    rng = np.random.default_rng(p * 100 + Nx)
    fr = rng.integers(0, 65536, (Ny * p, Nx * p), dtype=np.uint16)
    fr[0, :4] = [0, 65535, 0, 65535]
    fr[-1, -3:] = 65535
    prev = rng.integers(0, 65536, fr.shape, dtype=np.uint16)
    for cid in range(256):
        if not oracle.id_valid(cid):
            continue
        pv = prev if (cid >> 7) & 1 else None
        z = oracle.symbols(fr, p, cid, prev=pv)
        back = oracle.inverse_symbols(z, fr.shape[1], fr.shape[0], p, cid, prev=pv)
        assert np.array_equal(back, fr), cid
