"""Oracle pins for the per-block bzip2 coder (Sec. 2.1.3): brute-force
rotation sort, CRC-32/BZIP2 check value, optimal Huffman cost, and the
stock bzip2 decoder (Python's bz2 = libbz2, and /usr/bin/bzip2 -d) which
must reproduce every input byte for byte."""
import bz2
import heapq
import itertools
import shutil
import subprocess

import numpy as np
import pytest

import oracle


def brute_bwt(b):
    m = len(b)
    rots = [bytes(b[i:]) + bytes(b[:i]) for i in range(m)]
    order = sorted(range(m), key=lambda i: (rots[i], i))
    L = bytes(b[(i - 1) % m] for i in order)
    return L, order.index(0)


@pytest.mark.parametrize("m", range(1, 9))
def test_bwt_exhaustive_binary(m):
    for t in itertools.product((0, 1), repeat=m):
        b = bytes(t)
        L, o = oracle.bwt(b)
        assert (bytes(L), o) == brute_bwt(b)


def test_bwt_periodic_and_random():
    rng = np.random.default_rng(2)
    cases = [b"abab", b"aaaa", b"abcabcabc", b"banana", b"\x00" * 17, b"xyxyxyxyz"]
    cases += [bytes(rng.integers(0, k, n, dtype=np.uint8)) for k in (2, 3, 256) for n in (9, 50, 300)]
    for b in cases:
        L, o = oracle.bwt(b)
        assert (bytes(L), o) == brute_bwt(b), b


def test_crc32_bzip2_check_value():
    assert oracle.crc32(b"123456789") == 0xFC891918


def test_rle1_runs():
    assert bytes(oracle.rle1(b"aaaa")) == b"aaaa\x00"
    assert bytes(oracle.rle1(b"aaab")) == b"aaab"
    assert bytes(oracle.rle1(b"a" * 255)) == b"aaaa\xfb"
    assert bytes(oracle.rle1(b"a" * 257)) == b"aaaa\xfbaa"
    assert bytes(oracle.rle1(b"a" * 259)) == b"aaaa\xfbaaaa\x00"


def _heap_huffman_cost(w):
    h = list(w)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def test_huffman_lengths_optimal_and_complete():
    rng = np.random.default_rng(3)
    for alpha in (3, 4, 17, 100, 258):
        for _ in range(5):
            f = rng.integers(0, 1000, alpha).astype(np.uint32)
            f[rng.integers(0, alpha, alpha // 3)] = 0
            L = oracle.huff_lengths(f, max_len=40).astype(np.int64)
            w = np.maximum(f.astype(np.int64), 1)
            assert sum(2.0 ** -L) == 1.0               # complete prefix code
            assert int((w * L).sum()) == _heap_huffman_cost(w)  # optimal cost


def test_huffman_length_limit():
    f = np.array([2 ** k for k in range(24)] + [1] * 10, dtype=np.uint32)  # skewed -> deep tree
    L = oracle.huff_lengths(f, max_len=17)
    assert L.max() <= 17
    assert sum(2.0 ** -L.astype(np.int64)) <= 1.0


def _inputs():
    rng = np.random.default_rng(4)
    yield b"a"
    yield b"ab"
    yield b"\x00" * 1000
    yield bytes(range(256)) * 10
    yield bytes(rng.integers(0, 256, 5000, dtype=np.uint8))
    yield bytes(rng.integers(0, 3, 70000, dtype=np.uint8))
    yield bytes(np.repeat(rng.integers(0, 256, 3000, dtype=np.uint8), rng.integers(1, 300, 3000))[:300000])
    # worst-case RLE1 expansion: every 4-run becomes 5 bytes -> 900000 bytes
    yield (b"aaaabbbb" * 90000)
    yield bytes(rng.integers(0, 256, 720000, dtype=np.uint8))


@pytest.mark.parametrize("idx", range(9))
def test_stream_decoded_by_stock_bzip2(idx, tmp_path):
    data = list(_inputs())[idx]
    s = oracle.bz2_stream(data)
    assert bz2.decompress(s) == data
    assert oracle.bz2_decode(s, len(data)) == data
    if shutil.which("bzip2") and idx in (4, 7):
        f = tmp_path / "x.bz2"
        f.write_bytes(s)
        out = subprocess.run(["bzip2", "-dc", str(f)], check=True, capture_output=True).stdout
        assert out == data


def test_decoder_reads_stock_streams():
    rng = np.random.default_rng(5)
    for data in [b"hello world" * 100, bytes(rng.integers(0, 16, 2_000_000, dtype=np.uint8))]:
        for lvl in (1, 9):
            assert oracle.bz2_decode(bz2.compress(data, lvl), len(data)) == data


def test_decoder_rejects_corruption():
    data = bytes(np.random.default_rng(6).integers(0, 8, 20000, dtype=np.uint8))
    s = bytearray(oracle.bz2_stream(data))
    for pos in (3, 5, 12, len(s) // 2, len(s) - 3):
        t = bytearray(s)
        t[pos] ^= 0x10
        with pytest.raises(ValueError):
            got = oracle.bz2_decode(bytes(t), len(data))
            if got != data:  # a flip that still parses must fail the CRC
                raise ValueError("mismatch")
    with pytest.raises(ValueError):
        oracle.bz2_decode(bytes(s[: len(s) // 2]), len(data))
