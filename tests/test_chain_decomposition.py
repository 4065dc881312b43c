"""The pair-chain decomposition the judge kernels use, checked on the CPU
against the oracle's judge histogram (Sec. 2.1.2, Eq. (1)).

The judge-BWT's last column lists, per first byte b, the predecessors of
b's occurrences in stream order, so its bigram histogram counts the pairs
(predecessor of one occurrence of b, predecessor of the next one) plus one
pair at each boundary between non-empty buckets. The GPU splits a stream
into segments (CTAs) of warp ranges of lane sub-ranges, walks each
sub-range with a private table of last predecessors, and stitches lanes,
warps, segments and buckets back together in order. This model follows
that split (10 warps, 32 lanes) in plain Python; if the stitching were
wrong, a pair would be lost or invented at some boundary, and the counts
would differ from the oracle's on these streams, which put boundaries
everywhere (sub-ranges of 1..64 bytes, values absent from whole lanes)."""
import numpy as np
import pytest

import oracle

NONE = -1
WARPS, LANES = 10, 32


def walk(S, lo, hi, hist):
    """One lane: pairs inside [lo, hi); returns (first, last) per value."""
    n = len(S)
    last = [NONE] * 256
    first = [NONE] * 256
    if hi > lo:
        prev = int(S[lo - 1]) if lo > 0 else int(S[n - 1])  # cyclic predecessor
        for k in range(lo, hi):
            b = int(S[k])
            if last[b] == NONE:
                first[b] = prev
            else:
                hist[last[b], prev] += 1
            last[b] = prev
            prev = b
    return first, last


def stitch(parts, hist):
    """Join (first, last) tables in order; pairs across the joins."""
    first = [NONE] * 256
    last = [NONE] * 256
    for b in range(256):
        cur = NONE
        for f, l in parts:
            if l[b] == NONE:
                continue
            if cur != NONE:
                hist[cur, f[b]] += 1
            else:
                first[b] = f[b]
            cur = l[b]
        last[b] = cur
    return first, last


def model_hist(S, range_bytes):
    n = len(S)
    hist = np.zeros((256, 256), np.int64)
    sub = range_bytes // LANES
    seg_bytes = WARPS * range_bytes
    segs = []
    for seg in range(-(-n // seg_bytes)):
        warps = []
        for w in range(WARPS):
            ra = (seg * WARPS + w) * range_bytes
            lanes = []
            for lane in range(LANES):
                lo = min(n, ra + lane * sub)
                lanes.append(walk(S, lo, min(n, lo + sub), hist))
            warps.append(stitch(lanes, hist))
        segs.append(stitch(warps, hist))
    first, last = stitch(segs, hist)
    # bucket boundaries: last predecessor of b, first of the next present value
    present = [b for b in range(256) if last[b] != NONE]
    for b, nb in zip(present, present[1:]):
        hist[last[b], first[nb]] += 1
    return hist


def streams():
    rng = np.random.default_rng(7)
    yield rng.integers(0, 256, 3000, dtype=np.uint8)                  # every value, short lanes
    yield rng.integers(0, 3, 5000, dtype=np.uint8)                    # few values, long chains
    yield (rng.geometric(0.3, 9000) % 256).astype(np.uint8)           # skewed, like residual bytes
    yield np.zeros(700, np.uint8)                                     # one bucket
    yield np.repeat(rng.integers(0, 256, 60, dtype=np.uint8), 37)      # runs crossing lanes
    yield np.array([9], np.uint8)                                     # single byte
    yield rng.integers(0, 256, 37, dtype=np.uint8)                    # ragged, mostly empty lanes


@pytest.mark.parametrize("range_bytes", [32, 512, 2048])
@pytest.mark.parametrize("case", range(7))
def test_chain_split_matches_oracle(case, range_bytes):
    S = list(streams())[case]
    ref = np.asarray(oracle.judge_hist(S), dtype=np.int64).reshape(256, 256)
    assert np.array_equal(model_hist(S, range_bytes), ref)


def test_chain_split_total():
    # n - 1 pairs: one per adjacent entries of the n-entry last column
    S = np.random.default_rng(3).integers(0, 40, 4000, dtype=np.uint8)
    assert model_hist(S, 512).sum() == len(S) - 1
