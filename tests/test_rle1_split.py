"""The GPU decoder's split of inverse RLE1 across threads, modelled in plain
Python on the oracle's RLE1 output: a position q is a sync point when bytes
q-2 and q-1 differ and bytes q-5 .. q-2 are not all equal (byte q-1 is then a
literal that starts a run), every thread decodes from the first sync point of
its chunk to the next thread's, and the pieces concatenate to the input. Also
checks that no piece reads a count byte past its end."""
import numpy as np
import pytest

import oracle


def _decode_piece(blk, a, b, same, last, out):
    i = a
    while i < b:
        v = blk[i]
        out.append(v)
        same = same + 1 if v == last else 1
        last = v
        if same == 4:
            assert i + 1 < len(blk)
            out.extend([v] * blk[i + 1])
            i += 1
            same, last = 0, -1
        i += 1
    return i


def _sync(blk, q):
    return q >= 5 and blk[q - 1] != blk[q - 2] and not (blk[q - 5] == blk[q - 4] == blk[q - 3] == blk[q - 2])


def split_decode(blk, threads):
    m = len(blk)
    ch = max(8, -(-m // threads))
    starts = []
    for t in range(threads):
        s0, e0 = t * ch, min(m, (t + 1) * ch)
        if s0 >= m:
            starts.append(m)
        elif t == 0:
            starts.append(0)
        else:
            starts.append(next((q for q in range(max(s0, 5), e0) if _sync(blk, q)), m))
    out = []
    for t, p in enumerate(starts):
        if p >= m:
            continue
        end = next((q for q in starts[t + 1:] if q < m), m)
        same, last = (0, -1) if t == 0 else (1, blk[p - 1])
        assert _decode_piece(blk, p, end, same, last, out) == end  # never past the next piece
    return bytes(out)


def _runs(rng, n, alphabet):
    data = []
    while len(data) < n:
        data += [int(rng.integers(0, alphabet))] * int(rng.choice([1, 1, 2, 3, 4, 5, 7, 8, 255, 256, 259, 600]))
    return np.array(data[:n], dtype=np.uint8)


@pytest.mark.parametrize("alphabet", [1, 2, 3, 256])
def test_split_inverse_rle1(alphabet):
    rng = np.random.default_rng(alphabet)
    for n in (0, 1, 5, 37, 1000, 20000):
        data = _runs(rng, n, alphabet)
        blk = list(oracle.rle1(data))
        for threads in (1, 3, 64, 1024):
            assert split_decode(blk, threads) == data.tobytes()
