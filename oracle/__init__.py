"""CPU oracle for the PC-bzip2 compression path (ctypes over lfc_oracle.c).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package. The CUDA library never imports, links or calls it, and this package
never imports the CUDA library.

Every function here is a thin marshalling layer over the plain C oracle in
``lfc_oracle.c``; the arithmetic lives there, with the paper passage each step
follows. The exact compressed bytes (Huffman table partition, refinement and
tie rules) are choices the paper and the bzip2 format leave free: parity
unpinned beyond stock-decoder acceptance and the properties the tests check.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liblfc_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liblfc_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC", _SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, u32, u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "lfc_orc_id_valid": (i32, [i32]),
        "lfc_orc_symbols": (i32, [P, P, i32, i32, i32, i32, P]),
        "lfc_orc_inverse_symbols": (i32, [P, P, i32, i32, i32, i32, P]),
        "lfc_orc_judge_last": (None, [P, i64, P]),
        "lfc_orc_bigram": (None, [P, i64, P]),
        "lfc_orc_log2_fx": (u64, [u32]),
        "lfc_orc_score": (u64, [P]),
        "lfc_orc_judge": (i32, [P, P, i32, i32, i32, P, i32, P]),
        "lfc_orc_crc32": (u32, [P, i64]),
        "lfc_orc_rle1": (i64, [P, i64, P]),
        "lfc_orc_bwt": (i32, [P, i64, P, P]),
        "lfc_orc_mtf_rle2": (i64, [P, i64, P, P, P]),
        "lfc_orc_huff_lengths": (None, [P, i32, i32, P]),
        "lfc_orc_bz2_stream": (i64, [P, i64, P, i64]),
        "lfc_orc_bz2_decode": (i64, [P, i64, P, i64]),
        "lfc_orc_compress_id": (i64, [P, P, i32, i32, i32, i32, i32, P, i64]),
        "lfc_orc_compress": (i64, [P, P, i32, i32, i32, P, i32, i32, P, i64, P]),
        "lfc_orc_container_info": (i32, [P, i64, P, P, P, P]),
        "lfc_orc_realign": (None, [P, i64, i32, P]),
        "lfc_orc_unrealign": (None, [P, i64, i32, P]),
        "lfc_orc_decompress": (i32, [P, i64, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u16(a):
    return np.ascontiguousarray(a, dtype=np.uint16)


def _u8(a):
    if isinstance(a, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(a), dtype=np.uint8).copy()
    return np.ascontiguousarray(a, dtype=np.uint8)


# ----------------------------------------------------------------- candidates
def id_valid(cid: int) -> bool:
    return bool(_load().lfc_orc_id_valid(int(cid)))


def make_id(f: int, domain: int = 0, ordering: int = 0, temporal: int = 0, planar: int = 0) -> int:
    """Candidate id bit layout: f | planar << 3 | domain << 4 | ordering << 6 | temporal << 7."""
    return f | (planar << 3) | (domain << 4) | (ordering << 6) | (temporal << 7)


def planar_ids(temporal: bool = False) -> list[int]:
    """The default set with the planar byte layout (bit 3) instead."""
    return [c | 8 for c in default_ids(temporal)]


def default_ids(temporal: bool = False) -> list[int]:
    """Default candidate set: f in {0, 4, 5, 6, 7} (none plus the four
    multi-neighbour lossless-JPEG functions), three domains (f = 0 only once),
    two orderings; doubled with the temporal flag for series frames."""
    ids = []
    for t in ([0, 1] if temporal else [0]):
        for o in (0, 1):
            ids.append(make_id(0, 0, o, t))
            for d in (0, 1, 2):
                for f in (4, 5, 6, 7):
                    ids.append(make_id(f, d, o, t))
    return sorted(ids)


# ---------------------------------------------------------------- prediction
def symbols(frame, pitch: int, cid: int, prev=None) -> np.ndarray:
    """Symbol stream (uint16, stream order) of ``frame`` under candidate ``cid``."""
    X = _u16(frame)
    H, W = X.shape
    P = None if prev is None else _u16(prev)
    out = np.empty(H * W, dtype=np.uint16)
    rc = _load().lfc_orc_symbols(_ptr(X), _ptr(P), W, H, pitch, cid, _ptr(out))
    if rc != 0:
        raise ValueError("lfc_orc_symbols rejected the arguments (rc=%d)" % rc)
    return out


def inverse_symbols(stream, W: int, H: int, pitch: int, cid: int, prev=None) -> np.ndarray:
    Z = _u16(stream)
    P = None if prev is None else _u16(prev)
    out = np.empty((H, W), dtype=np.uint16)
    rc = _load().lfc_orc_inverse_symbols(_ptr(Z), _ptr(P), W, H, pitch, cid, _ptr(out))
    if rc != 0:
        raise ValueError("lfc_orc_inverse_symbols rejected the arguments (rc=%d)" % rc)
    return out


def stream_bytes(sym: np.ndarray, planar: bool = False) -> np.ndarray:
    """Realign uint16 symbols to bytes (lfc_orc_realign): (lo, hi) per
    symbol, or planar (all high bytes, then all low bytes)."""
    z = _u16(sym).ravel()
    out = np.empty(2 * z.size, dtype=np.uint8)
    _load().lfc_orc_realign(_ptr(z), z.size, 1 if planar else 0, _ptr(out))
    return out


def unrealign(S, planar: bool = False) -> np.ndarray:
    S = _u8(S)
    z = np.empty(S.size // 2, dtype=np.uint16)
    _load().lfc_orc_unrealign(_ptr(S), z.size, 1 if planar else 0, _ptr(z))
    return z


# --------------------------------------------------------------------- judge
def judge_last(S) -> np.ndarray:
    S = _u8(S)
    L = np.empty_like(S)
    _load().lfc_orc_judge_last(_ptr(S), S.size, _ptr(L))
    return L


def bigram(L) -> np.ndarray:
    L = _u8(L)
    h = np.empty(65536, dtype=np.uint32)
    _load().lfc_orc_bigram(_ptr(L), L.size, _ptr(h))
    return h


def judge_hist(S) -> np.ndarray:
    return bigram(judge_last(S))


def log2_fx(c: int) -> int:
    return int(_load().lfc_orc_log2_fx(int(c)))


def score(hist) -> int:
    h = np.ascontiguousarray(hist, dtype=np.uint32)
    assert h.size == 65536
    return int(_load().lfc_orc_score(_ptr(h)))


def judge(frame, pitch: int, ids=None, prev=None):
    """Returns (best id, scores as a list of ints in ``ids`` order)."""
    X = _u16(frame)
    H, W = X.shape
    if ids is None:
        ids = default_ids(prev is not None)
    ids_a = np.asarray(ids, dtype=np.uint8)
    P = None if prev is None else _u16(prev)
    sc = np.zeros(len(ids_a), dtype=np.uint64)
    best = _load().lfc_orc_judge(_ptr(X), _ptr(P), W, H, pitch, _ptr(ids_a), len(ids_a), _ptr(sc))
    if best < 0:
        raise ValueError("lfc_orc_judge rejected the arguments (rc=%d)" % best)
    return int(best), [int(v) for v in sc]


# --------------------------------------------------------------------- bzip2
def crc32(data) -> int:
    d = _u8(data)
    return int(_load().lfc_orc_crc32(_ptr(d), d.size))


def rle1(data) -> np.ndarray:
    d = _u8(data)
    out = np.empty(d.size + d.size // 4 + 8, dtype=np.uint8)
    m = _load().lfc_orc_rle1(_ptr(d), d.size, _ptr(out))
    return out[:m].copy()


def bwt(block):
    """Returns (L, origPtr) of the full rotation sort of ``block``."""
    b = _u8(block)
    L = np.empty_like(b)
    orig = ctypes.c_int64(0)
    rc = _load().lfc_orc_bwt(_ptr(b), b.size, _ptr(L), ctypes.byref(orig))
    if rc != 0:
        raise ValueError("bwt failed")
    return L, int(orig.value)


def mtf_rle2(L):
    """Returns (symbols uint16, in_use[256] uint8, freq[258] uint32)."""
    L = _u8(L)
    sym = np.empty(L.size + 1, dtype=np.uint16)
    in_use = np.empty(256, dtype=np.uint8)
    freq = np.empty(258, dtype=np.uint32)
    n = _load().lfc_orc_mtf_rle2(_ptr(L), L.size, _ptr(sym), _ptr(in_use), _ptr(freq))
    return sym[:n].copy(), in_use, freq


def huff_lengths(freq, max_len: int = 17) -> np.ndarray:
    f = np.ascontiguousarray(freq, dtype=np.uint32)
    out = np.empty(f.size, dtype=np.uint8)
    _load().lfc_orc_huff_lengths(_ptr(f), f.size, max_len, _ptr(out))
    return out


def bz2_stream(data) -> bytes:
    """One standalone one-block bzip2 stream of ``data`` (<= 720000 bytes)."""
    d = _u8(data)
    cap = 64 + 3 * d.size + 20000
    out = np.empty(cap, dtype=np.uint8)
    n = _load().lfc_orc_bz2_stream(_ptr(d), d.size, _ptr(out), cap)
    if n < 0:
        raise ValueError("bz2_stream failed (rc=%d)" % n)
    return out[:n].tobytes()


def bz2_decode(stream, cap: int) -> bytes:
    s = _u8(stream)
    out = np.empty(max(cap, 1), dtype=np.uint8)
    n = _load().lfc_orc_bz2_decode(_ptr(s), s.size, _ptr(out), cap)
    if n < 0:
        raise ValueError("corrupt bzip2 stream (rc=%d)" % n)
    return out[:n].tobytes()


# ----------------------------------------------------------------- container
def max_container_bytes(W: int, H: int, block_bytes: int = 720000) -> int:
    n = 2 * W * H
    nb = (n + block_bytes - 1) // block_bytes
    return 40 + 4 * nb + nb * (64 + 3 * block_bytes + 20000)


def compress_id(frame, pitch: int, cid: int, prev=None, block_bytes: int = 720000) -> bytes:
    X = _u16(frame)
    H, W = X.shape
    P = None if prev is None else _u16(prev)
    cap = max_container_bytes(W, H, block_bytes)
    out = np.empty(cap, dtype=np.uint8)
    n = _load().lfc_orc_compress_id(_ptr(X), _ptr(P), W, H, pitch, cid, block_bytes, _ptr(out), cap)
    if n < 0:
        raise ValueError("compress failed (rc=%d)" % n)
    return out[:n].tobytes()


def compress(frame, pitch: int, ids=None, prev=None, block_bytes: int = 720000):
    """Judge over ``ids`` and compress with the winner. Returns (bytes, id)."""
    X = _u16(frame)
    H, W = X.shape
    if ids is None:
        ids = default_ids(prev is not None)
    ids_a = np.asarray(ids, dtype=np.uint8)
    P = None if prev is None else _u16(prev)
    cap = max_container_bytes(W, H, block_bytes)
    out = np.empty(cap, dtype=np.uint8)
    chosen = ctypes.c_int(-1)
    n = _load().lfc_orc_compress(_ptr(X), _ptr(P), W, H, pitch, _ptr(ids_a), len(ids_a),
                                 block_bytes, _ptr(out), cap, ctypes.byref(chosen))
    if n < 0:
        raise ValueError("compress failed (rc=%d)" % n)
    return out[:n].tobytes(), int(chosen.value)


def container_info(blob):
    b = _u8(blob)
    W, H, p, cid = (ctypes.c_int() for _ in range(4))
    rc = _load().lfc_orc_container_info(_ptr(b), b.size, ctypes.byref(W), ctypes.byref(H),
                                        ctypes.byref(p), ctypes.byref(cid))
    if rc != 0:
        raise ValueError("not an LFC1 container")
    return W.value, H.value, p.value, cid.value


def decompress(blob, prev=None) -> np.ndarray:
    b = _u8(blob)
    W, H, _, _ = container_info(b)
    out = np.empty((H, W), dtype=np.uint16)
    P = None if prev is None else _u16(prev)
    rc = _load().lfc_orc_decompress(_ptr(b), b.size, _ptr(P), _ptr(out))
    if rc != 0:
        raise ValueError("corrupt container")
    return out
