"""Oracle pins for the prediction part (Sec. 2.1.1) and the orderings.

Pins: hand-computed lossless-JPEG values (tests/golden/predictor_2x2.txt),
hand-computed inter-lenslet and phase-space symbols of a frame whose left and
top neighbouring lenslets differ (tests/golden/predictor_inter_phase_2x2.txt),
closed-form residuals on planes, lenslet-periodic frames and lenslet ramps,
the sub-aperture mosaic property of the view-major ordering, and exact round
trips.
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
    assert oracle.id_valid(0x08)       # bit 3 is the planar byte layout, not part of f
    assert not oracle.id_valid(0x18)   # f = 0 needs domain 0 in either layout
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


GOLDEN_IP = os.path.join(os.path.dirname(__file__), "golden", "predictor_inter_phase_2x2.txt")


def _inter_phase_golden():
    frame, syms = [], []
    for line in open(GOLDEN_IP):
        parts = line.split()
        if not parts or parts[0].startswith("#"):
            continue
        if parts[0] == "frame":
            frame.append([int(v) for v in parts[1:]])
        elif parts[0] == "sym":
            syms.append((int(parts[1]), int(parts[2]), [int(v) for v in parts[3:]]))
    return np.array(frame, dtype=np.uint16), syms


@pytest.mark.parametrize("case", range(4))
def test_inter_phase_golden_orientation(case):
    """Hand-computed symbols of a 2x2-lenslet frame whose left and top
    neighbouring lenslets differ, so that swapping A (left lenslet) and B (top
    lenslet), or the x - p and y - p strides, changes the result."""
    frame, syms = _inter_phase_golden()
    f, dom, exp = syms[case]
    z = oracle.symbols(frame, 2, oracle.make_id(f, dom, 0, 0))
    assert [int(v) for v in z] == exp
    back = oracle.inverse_symbols(z, 4, 4, 2, oracle.make_id(f, dom, 0, 0))
    assert np.array_equal(back, frame)


def _lenslet_ramp(p, Ny, Nx, c0, a, b):
    """Frame constant inside each lenslet, a linear ramp across lenslets:
    X = c0 + a s + b t for lenslet column s and row t."""
    t = np.arange(Ny * p)[:, None] // p
    s = np.arange(Nx * p)[None, :] // p
    return (c0 + a * s + b * t).astype(np.uint16)


def _ramp_interior_residual(f, a, b):
    # A = X - a (left lenslet), B = X - b (top lenslet), C = X - a - b.
    return {1: a, 2: b, 3: a + b, 4: 0, 5: a - (a // 2), 6: b - (b // 2), 7: -((-(a + b)) // 2)}[f]


@pytest.mark.parametrize("f", range(1, 8))
@pytest.mark.parametrize("a,b", [(7, -3), (-5, 12)])
def test_inter_lenslet_ramp_closed_form(f, a, b):
    """Closed form on a lenslet ramp: first lenslet row predicts from the left
    lenslet (residual a), first lenslet column from the top one (residual b),
    inside the grid the predictor function of (A, B, C) = (X - a, X - b,
    X - a - b). The residuals are the same at every view (u, v)."""
    p, Ny, Nx = 3, 4, 5
    fr = _lenslet_ramp(p, Ny, Nx, 1000, a, b)
    z = oracle.symbols(fr, p, oracle.make_id(f, 1, 0, 0)).reshape(fr.shape)
    t = np.arange(Ny * p)[:, None] // p + np.zeros((1, Nx * p), dtype=np.int64)
    s = np.arange(Nx * p)[None, :] // p + np.zeros((Ny * p, 1), dtype=np.int64)
    d = np.where((t == 0) & (s == 0), fr.astype(np.int64),
                 np.where(t == 0, a, np.where(s == 0, b, _ramp_interior_residual(f, a, b))))
    assert np.array_equal(z, _zz(d))


@pytest.mark.parametrize("f", range(1, 8))
@pytest.mark.parametrize("a,b", [(7, -3), (-5, 12)])
def test_phase_space_ramp_closed_form(f, a, b):
    """Phase space on the same ramp: inside a lenslet every intra residual is 0
    except the origin view's, which is the pixel itself; the second (inter)
    stage therefore leaves the inter-lenslet closed form at view (0, 0) and 0
    at every other view."""
    p, Ny, Nx = 3, 4, 5
    fr = _lenslet_ramp(p, Ny, Nx, 1000, a, b)
    z = oracle.symbols(fr, p, oracle.make_id(f, 2, 0, 0)).reshape(fr.shape)
    zi = oracle.symbols(fr, p, oracle.make_id(f, 1, 0, 0)).reshape(fr.shape)
    origin = (np.arange(Ny * p)[:, None] % p == 0) & (np.arange(Nx * p)[None, :] % p == 0)
    assert np.array_equal(z, np.where(origin, zi, 0))
