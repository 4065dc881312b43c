"""Python binding of liblfc (include/lfc.h): argument marshalling only.

Every step of the compression path runs in the CUDA library; this module
passes device pointers (``tensor.data_ptr()``), sizes and the current CUDA
stream. It never computes any part of the method itself, and it has no CPU
fallback: if ``liblfc.so`` is missing it raises.

Frames are 2-D CUDA tensors of 2-byte elements (int16 or uint16 views of the
uint16 counts), row-major, height x width.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "liblfc.so")

LFC_OK = 0
STATUS = {0: "LFC_OK", 1: "LFC_ERR_INVALID_ARG", 2: "LFC_ERR_CAPACITY", 3: "LFC_ERR_CORRUPT",
          4: "LFC_ERR_CUDA", 5: "LFC_ERR_TIMEOUT", 6: "LFC_ERR_UNIMPLEMENTED", 7: "LFC_ERR_NOMEM"}

# every symbol include/lfc.h declares
EXPORTS = ["lfc_plan_create", "lfc_plan_destroy", "lfc_plan_last_error", "lfc_judge", "lfc_symbols",
           "lfc_max_compressed_bytes", "lfc_compress", "lfc_bzip2_encode", "lfc_max_stream_bytes",
           "lfc_plan_block_capacity", "lfc_decompress", "lfc_status_string", "lfc_plan_set_timing",
           "lfc_plan_timing", "lfc_plan_launch_count", "lfc_judge_noalloc", "lfc_plan_bwt_counters",
           "lfc_batch_create", "lfc_batch_launch", "lfc_batch_destroy",
           "lfc_plan_set_tuning", "lfc_plan_get_tuning",
           "lfc_cnn_create", "lfc_cnn_destroy", "lfc_cnn_last_error", "lfc_cnn_param_count", "lfc_cnn_set_params",
           "lfc_cnn_get_params", "lfc_cnn_thumbnails", "lfc_cnn_set_thumbnails", "lfc_cnn_forward", "lfc_cnn_backward",
           "lfc_cnn_adam_step", "lfc_plan_set_proposal", "lfc_propose", "lfc_plan_device_status",
           "lfc_plan_inject_fault", "lfc_bwt_blocks", "lfc_compress_host"]

STAGES = ["judge_hist", "judge_score", "emit", "crc", "rle1", "bwt_sort8", "bwt_refine", "bwt_out", "mtf",
          "huffman", "pack", "container", "judge_emit", "bwt_keys"]


class LfcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("max_frames", ctypes.c_int32), ("candidate_mask", ctypes.c_uint64 * 4),
                ("temporal", ctypes.c_int32), ("keyframe_interval", ctypes.c_int32),
                ("block_bytes", ctypes.c_int32), ("topk", ctypes.c_int32), ("tau", ctypes.c_float)]


class Tuning(ctypes.Structure):
    _fields_ = [("emit_tile_lenslets", ctypes.c_int32), ("chain_range_bytes", ctypes.c_int32),
                ("judge_frames_per_launch", ctypes.c_int32), ("wait_budget_ms", ctypes.c_int32)]


class Frame(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("prev", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("pitch", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None


def load():
    """Load liblfc.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO_PATH):
        raise RuntimeError("liblfc.so not built (%s): run __graft_entry__.build()" % SO_PATH)
    lib = ctypes.CDLL(SO_PATH)
    P, i32, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
    sig = {
        "lfc_plan_create": (i32, [ctypes.POINTER(Config), P, ctypes.POINTER(P)]),
        "lfc_plan_destroy": (None, [P]),
        "lfc_plan_last_error": (ctypes.c_char_p, [P]),
        "lfc_judge": (i32, [P, ctypes.POINTER(Frame), i32, P, P]),
        "lfc_symbols": (i32, [P, ctypes.POINTER(Frame), i32, P]),
        "lfc_max_compressed_bytes": (sz, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
        "lfc_compress": (i32, [P, ctypes.POINTER(Frame), i32, P, P, sz, P]),
        "lfc_compress_host": (i32, [P, ctypes.POINTER(Frame), i32, P, P, sz, P]),
        "lfc_bzip2_encode": (i32, [P, P, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_uint32), i32, P, sz, P]),
        "lfc_max_stream_bytes": (sz, [ctypes.c_int32]),
        "lfc_plan_block_capacity": (i32, [P]),
        "lfc_decompress": (i32, [P, ctypes.POINTER(P), ctypes.POINTER(u64), i32, ctypes.POINTER(P),
                                 ctypes.POINTER(u64), ctypes.POINTER(P)]),
        "lfc_status_string": (ctypes.c_char_p, [i32]),
        "lfc_plan_set_timing": (i32, [P, i32]),
        "lfc_plan_timing": (i32, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32]),
        "lfc_plan_launch_count": (ctypes.c_int64, [P]),
        "lfc_plan_bwt_counters": (i32, [P, ctypes.POINTER(ctypes.c_int64), i32]),
        "lfc_batch_create": (i32, [P, ctypes.POINTER(Frame), i32, P, P, sz, P, ctypes.POINTER(P)]),
        "lfc_batch_launch": (i32, [P]),
        "lfc_plan_set_tuning": (i32, [P, ctypes.POINTER(Tuning)]),
        "lfc_plan_get_tuning": (i32, [P, ctypes.POINTER(Tuning)]),
        "lfc_cnn_create": (i32, [i32, i32, ctypes.c_uint64, P, ctypes.POINTER(P)]),
        "lfc_cnn_destroy": (None, [P]),
        "lfc_cnn_last_error": (ctypes.c_char_p, [P]),
        "lfc_cnn_param_count": (sz, [P]),
        "lfc_cnn_set_params": (i32, [P, P, sz]),
        "lfc_cnn_get_params": (i32, [P, P, P, sz]),
        "lfc_cnn_thumbnails": (i32, [P, ctypes.POINTER(Frame), i32, P]),
        "lfc_cnn_set_thumbnails": (i32, [P, P, i32]),
        "lfc_cnn_forward": (i32, [P, i32, P]),
        "lfc_cnn_backward": (i32, [P, i32, P, P]),
        "lfc_cnn_adam_step": (i32, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "lfc_plan_set_proposal": (i32, [P, P, ctypes.POINTER(ctypes.c_uint8), i32, i32, ctypes.c_float]),
        "lfc_propose": (i32, [P, ctypes.POINTER(Frame), i32, P]),
        "lfc_batch_destroy": (None, [P]),
        "lfc_judge_noalloc": (i32, [ctypes.POINTER(Frame), ctypes.POINTER(ctypes.c_uint8), i32, P, P, P]),
        "lfc_plan_device_status": (i32, [P]),
        "lfc_plan_inject_fault": (i32, [P, i32]),
        "lfc_bwt_blocks": (i32, [P, P, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_uint32), i32, P, sz, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def max_compressed_bytes(width: int, height: int, block_bytes: int = 0) -> int:
    return int(load().lfc_max_compressed_bytes(width, height, block_bytes))


def max_stream_bytes(block_bytes: int) -> int:
    return int(load().lfc_max_stream_bytes(block_bytes))


def default_ids(temporal=False):
    """The plan's default candidate ids (include/lfc.h id layout): f in
    {0, 4, 5, 6, 7} x domains 0-2 (f = 0 only in domain 0) x 2 orderings, 26
    ids ascending; with ``temporal`` also the same 26 with bit 7 set."""
    ids = sorted([o << 6 for o in (0, 1)] + [f | (d << 4) | (o << 6) for o in (0, 1) for d in (0, 1, 2)
                                              for f in (4, 5, 6, 7)])
    return ids + [i | 0x80 for i in ids] if temporal else ids


def mask_from_ids(ids):
    m = [0, 0, 0, 0]
    for i in ids:
        m[i >> 6] |= 1 << (i & 63)
    return m


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Plan:
    """One plan = workspace for frames up to width x height, max_frames per call."""

    def __init__(self, width, height, pitch, max_frames=1, candidate_ids=None, temporal=False,
                 block_bytes=0, keyframe_interval=16, stream=None):
        torch = _torch()
        self.lib = load()
        cfg = Config()
        cfg.width, cfg.height, cfg.pitch, cfg.max_frames = width, height, pitch, max_frames
        m = mask_from_ids(candidate_ids) if candidate_ids else [0, 0, 0, 0]
        for i in range(4):
            cfg.candidate_mask[i] = m[i]
        cfg.temporal = 1 if temporal else 0
        cfg.keyframe_interval = keyframe_interval
        cfg.block_bytes = block_bytes
        cfg.topk, cfg.tau = 0, 0.0
        self.cfg = cfg
        self.block_bytes = block_bytes or 720000
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = self.lib.lfc_plan_create(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != LFC_OK:
            raise LfcError(rc, "lfc_plan_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lfc_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != LFC_OK:
            msg = self.lib.lfc_plan_last_error(self.h)
            raise LfcError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def set_timing(self, enable=True):
        self._check(self.lib.lfc_plan_set_timing(self.h, 1 if enable else 0), "lfc_plan_set_timing")

    def timing(self):
        """Accumulated device milliseconds and span counts per stage (synchronises)."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        sp = (ctypes.c_int64 * n)()
        self._check(self.lib.lfc_plan_timing(self.h, ms, sp, n), "lfc_plan_timing")
        return {k: (ms[i], sp[i]) for i, k in enumerate(STAGES)}

    def set_tuning(self, emit_tile_lenslets=0, chain_range_bytes=0, judge_frames_per_launch=0, wait_budget_ms=0):
        t = Tuning(emit_tile_lenslets, chain_range_bytes, judge_frames_per_launch, wait_budget_ms)
        self._check(self.lib.lfc_plan_set_tuning(self.h, ctypes.byref(t)), "lfc_plan_set_tuning")

    def inject_fault(self, fault=1):
        """Test hook (lfc_plan_inject_fault): 1 = the next suffix sort's first
        tile withholds its look-back status, so its waiters time out."""
        self._check(self.lib.lfc_plan_inject_fault(self.h, fault), "lfc_plan_inject_fault")

    def device_status(self):
        """LFC status of the plan's bounded device waits since the last check
        (lfc_plan_device_status); synchronises the plan's stream."""
        return int(self.lib.lfc_plan_device_status(self.h))

    def get_tuning(self):
        t = Tuning()
        self._check(self.lib.lfc_plan_get_tuning(self.h, ctypes.byref(t)), "lfc_plan_get_tuning")
        return {"emit_tile_lenslets": t.emit_tile_lenslets, "chain_range_bytes": t.chain_range_bytes,
                "judge_frames_per_launch": t.judge_frames_per_launch, "wait_budget_ms": t.wait_budget_ms}

    def launch_count(self):
        return int(self.lib.lfc_plan_launch_count(self.h))

    def bwt_counters(self):
        """(calls, rounds, input bytes coded, tied elements over rounds, tied per round)."""
        buf = (ctypes.c_int64 * 36)()
        k = self.lib.lfc_plan_bwt_counters(self.h, buf, 36)
        v = list(buf[:k])
        return {"calls": v[0], "rounds": v[1], "input_bytes": v[2], "tied_total": v[3],
                "tied_per_round": [x for x in v[4:] if x]}

    @property
    def block_capacity(self):
        return int(self.lib.lfc_plan_block_capacity(self.h))

    @staticmethod
    def _frames(frames, pitch, prevs=None):
        arr = (Frame * len(frames))()
        for i, f in enumerate(frames):
            assert f.is_cuda and f.dim() == 2 and f.element_size() == 2 and f.is_contiguous()
            arr[i].data = f.data_ptr()
            pv = None if prevs is None else prevs[i]
            arr[i].prev = pv.data_ptr() if pv is not None else None
            arr[i].height, arr[i].width = f.shape
            arr[i].pitch = pitch if isinstance(pitch, int) else pitch[i]
            arr[i].reserved = 0
        return arr

    # ------------------------------------------------------------- calls
    def judge(self, frames, pitch, prevs=None, choice=None, scores=None):
        """Returns (choice uint8[n], scores int64[n, 256] holding uint64 bits)."""
        torch = _torch()
        n = len(frames)
        arr = self._frames(frames, pitch, prevs)
        if choice is None:
            choice = torch.empty(n, dtype=torch.uint8, device=frames[0].device)
        if scores is None:
            scores = torch.zeros((n, 256), dtype=torch.int64, device=frames[0].device)
        self._check(self.lib.lfc_judge(self.h, arr, n, _ptr(choice), _ptr(scores)), "lfc_judge")
        return choice, scores

    def symbols(self, frame, pitch, cid, prev=None, out=None):
        torch = _torch()
        arr = self._frames([frame], pitch, None if prev is None else [prev])
        if out is None:
            out = torch.empty(frame.numel(), dtype=torch.int16, device=frame.device)
        self._check(self.lib.lfc_symbols(self.h, arr, cid, _ptr(out)), "lfc_symbols")
        return out

    def slots(self, frames):
        offs, o = [], 0
        for f in frames:
            offs.append(o)
            o += max_compressed_bytes(f.shape[1], f.shape[0], self.block_bytes)
        return offs, o

    def compress_host(self, frames, pitch, prevs=None, choice=None, out=None, sizes=None):
        """lfc_compress_host: frames (and prevs) are CPU uint16/int16 tensors or
        arrays (pinned memory copies fastest); returns (out host uint8 buffer,
        sizes uint64[n] host, slot offsets)."""
        import numpy as np
        torch = _torch()

        def host(x):
            if isinstance(x, np.ndarray):
                x = torch.from_numpy(np.ascontiguousarray(x))
            assert not x.is_cuda and x.dim() == 2 and x.element_size() == 2 and x.is_contiguous()
            return x
        frames = [host(f) for f in frames]
        prevs = None if prevs is None else [None if p is None else host(p) for p in prevs]
        n = len(frames)
        arr = (Frame * n)()
        for i, f in enumerate(frames):
            arr[i].data = f.data_ptr()
            pv = None if prevs is None else prevs[i]
            arr[i].prev = pv.data_ptr() if pv is not None else None
            arr[i].height, arr[i].width = f.shape
            arr[i].pitch = pitch if isinstance(pitch, int) else pitch[i]
            arr[i].reserved = 0
        offs, total = self.slots(frames)
        if out is None:
            out = torch.empty(total, dtype=torch.uint8)
        if sizes is None:
            sizes = np.zeros(n, dtype=np.uint64)
        ch = None
        if choice is not None:
            ch = np.ascontiguousarray(np.asarray(choice, dtype=np.uint8))
        rc = self.lib.lfc_compress_host(self.h, arr, n, ch.ctypes.data_as(ctypes.c_void_p) if ch is not None else None,
                                        _ptr(out), out.numel(), sizes.ctypes.data_as(ctypes.c_void_p))
        self._check(rc, "lfc_compress_host")
        return out, sizes, offs

    def compress(self, frames, pitch, prevs=None, choice=None, out=None, sizes=None):
        """Compress on the device. Returns (out uint8 buffer, sizes int64[n], slot offsets)."""
        torch = _torch()
        n = len(frames)
        arr = self._frames(frames, pitch, prevs)
        offs, total = self.slots(frames)
        if out is None:
            out = torch.empty(total, dtype=torch.uint8, device=frames[0].device)
        if sizes is None:
            sizes = torch.empty(n, dtype=torch.int64, device=frames[0].device)
        rc = self.lib.lfc_compress(self.h, arr, n, _ptr(choice), _ptr(out), out.numel(), _ptr(sizes))
        self._check(rc, "lfc_compress")
        return out, sizes, offs

    def set_proposal(self, cnn, class_ids, topk, tau):
        ids = (ctypes.c_uint8 * len(class_ids))(*class_ids)
        self._check(self.lib.lfc_plan_set_proposal(self.h, cnn.h if cnn else None, ids, len(class_ids), topk, tau),
                    "lfc_plan_set_proposal")

    def propose(self, frames, pitch):
        torch = _torch()
        arr = self._frames(frames, pitch)
        masks = torch.zeros((len(frames), 4), dtype=torch.int64, device=frames[0].device)
        self._check(self.lib.lfc_propose(self.h, arr, len(frames), _ptr(masks)), "lfc_propose")
        return masks

    def batch(self, frames, pitch, prevs=None, choice=None, out=None, sizes=None):
        """Capture lfc_compress on these frame buffers as a CUDA graph."""
        return Batch(self, frames, pitch, prevs, choice, out, sizes)

    def compress_to_bytes(self, frames, pitch, prevs=None, choice=None):
        out, sizes, offs = self.compress(frames, pitch, prevs, choice)
        sz = sizes.cpu().numpy()
        host = out.cpu().numpy()
        return [host[o:o + int(s)].tobytes() for o, s in zip(offs, sz)]

    def bzip2_encode(self, data, offsets, sizes_in, out=None, stride=None):
        """Device bytes ``data`` (uint8 tensor) split at offsets/sizes -> streams."""
        torch = _torch()
        nb = len(offsets)
        offs = (ctypes.c_uint64 * nb)(*[int(o) for o in offsets])
        szs = (ctypes.c_uint32 * nb)(*[int(s) for s in sizes_in])
        if stride is None:
            stride = max_stream_bytes(max(int(s) for s in sizes_in))
        if out is None:
            out = torch.empty(nb * stride, dtype=torch.uint8, device=data.device)
        ss = torch.empty(nb, dtype=torch.int32, device=data.device)
        rc = self.lib.lfc_bzip2_encode(self.h, _ptr(data), offs, szs, nb, _ptr(out), stride, _ptr(ss))
        self._check(rc, "lfc_bzip2_encode")
        return out, ss, stride

    def bzip2_encode_bytes(self, blocks):
        torch = _torch()
        buf = b"".join(blocks)
        data = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda()
        offs, o = [], 0
        for b in blocks:
            offs.append(o)
            o += len(b)
        out, ss, stride = self.bzip2_encode(data, offs, [len(b) for b in blocks])
        host = out.cpu().numpy()
        sz = ss.cpu().numpy()
        return [host[i * stride:i * stride + int(sz[i])].tobytes() for i in range(len(blocks))]

    def bwt_blocks(self, data, offsets, sizes_in):
        """Device bytes ``data`` split at offsets/sizes -> (L columns as a
        uint8 tensor of n x stride, lengths, origin rows) of RLE1 + BWT."""
        torch = _torch()
        nb = len(offsets)
        offs = (ctypes.c_uint64 * nb)(*[int(o) for o in offsets])
        szs = (ctypes.c_uint32 * nb)(*[int(s) for s in sizes_in])
        stride = 900000
        L = torch.empty(nb * stride, dtype=torch.uint8, device=data.device)
        ln = torch.empty(nb, dtype=torch.int32, device=data.device)
        orig = torch.empty(nb, dtype=torch.int32, device=data.device)
        rc = self.lib.lfc_bwt_blocks(self.h, _ptr(data), offs, szs, nb, _ptr(L), stride, _ptr(ln), _ptr(orig))
        self._check(rc, "lfc_bwt_blocks")
        return L.view(nb, stride), ln, orig

    def decompress(self, blobs, outs, prevs=None):
        """blobs: list of uint8 CUDA tensors (one container each); outs: frame tensors."""
        n = len(blobs)
        ins = (ctypes.c_void_p * n)(*[b.data_ptr() for b in blobs])
        szs = (ctypes.c_uint64 * n)(*[b.numel() for b in blobs])
        os_ = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        ob = (ctypes.c_uint64 * n)(*[o.numel() * o.element_size() for o in outs])
        pv = None
        if prevs is not None:
            pv = (ctypes.c_void_p * n)(*[(p.data_ptr() if p is not None else None) for p in prevs])
        rc = self.lib.lfc_decompress(self.h, ins, szs, n, os_, ob, pv)
        self._check(rc, "lfc_decompress")
        return outs


class Cnn:
    """The proposal network (lfc_cnn_*): thumbnails, forward, backward, Adam."""

    def __init__(self, n_classes, max_batch, seed=0, stream=None):
        torch = _torch()
        self.lib = load()
        self.K = n_classes
        self.max_batch = max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = self.lib.lfc_cnn_create(n_classes, max_batch, seed, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != LFC_OK:
            raise LfcError(rc, "lfc_cnn_create")
        self.h = h
        self.n_params = int(self.lib.lfc_cnn_param_count(h))

    def _check(self, rc, what):
        if rc != LFC_OK:
            msg = self.lib.lfc_cnn_last_error(self.h)
            raise LfcError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lfc_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.n_params
        self._check(self.lib.lfc_cnn_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size), "set_params")

    def get_params(self, grads=False):
        p = np.empty(self.n_params, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32) if grads else None
        self._check(self.lib.lfc_cnn_get_params(self.h, p.ctypes.data_as(ctypes.c_void_p),
                                                None if g is None else g.ctypes.data_as(ctypes.c_void_p),
                                                self.n_params), "get_params")
        return (p, g) if grads else p

    def thumbnails(self, frames, pitch, want=False):
        torch = _torch()
        arr = Plan._frames(frames, pitch)
        out = torch.empty((len(frames), 2, 256, 256), dtype=torch.float32, device=frames[0].device) if want else None
        self._check(self.lib.lfc_cnn_thumbnails(self.h, arr, len(frames), _ptr(out)), "thumbnails")
        return out

    def set_thumbnails(self, thumbs):
        self._check(self.lib.lfc_cnn_set_thumbnails(self.h, _ptr(thumbs.contiguous()), thumbs.shape[0]), "set_thumbnails")

    def forward(self, n):
        torch = _torch()
        probs = torch.empty((n, self.K), dtype=torch.float32, device="cuda")
        self._check(self.lib.lfc_cnn_forward(self.h, n, _ptr(probs)), "forward")
        return probs

    def backward(self, labels):
        torch = _torch()
        n = labels.numel()
        loss = torch.empty(n, dtype=torch.float32, device="cuda")
        self._check(self.lib.lfc_cnn_backward(self.h, n, _ptr(labels), _ptr(loss)), "backward")
        return loss

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.lfc_cnn_adam_step(self.h, lr, beta1, beta2, eps), "adam_step")

    def flat_from_dict(self, P):
        keys = ["w0", "b0", "w1", "b1", "w2", "b2", "w3", "b3", "wl", "bl"]
        return np.concatenate([np.asarray(P[k], dtype=np.float64).reshape(-1) for k in keys]).astype(np.float32)

    def dict_from_flat(self, flat):
        shapes = [("w0", (3, 3, 2, 32)), ("b0", (32,)), ("w1", (3, 3, 32, 32)), ("b1", (32,)),
                  ("w2", (3, 3, 32, 32)), ("b2", (32,)), ("w3", (3, 3, 32, 32)), ("b3", (32,)),
                  ("wl", (32, self.K)), ("bl", (self.K,))]
        out, o = {}, 0
        for k, shp in shapes:
            n = int(np.prod(shp))
            out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
            o += n
        return out


class Batch:
    """One captured compress call (lfc_batch_*): launch() replays it."""

    def __init__(self, plan, frames, pitch, prevs=None, choice=None, out=None, sizes=None):
        torch = _torch()
        self.plan = plan
        self.frames = frames
        n = len(frames)
        self.arr = plan._frames(frames, pitch, prevs)
        self.offs, total = plan.slots(frames)
        self.out = out if out is not None else torch.empty(total, dtype=torch.uint8, device=frames[0].device)
        self.sizes = sizes if sizes is not None else torch.empty(n, dtype=torch.int64, device=frames[0].device)
        h = ctypes.c_void_p()
        rc = plan.lib.lfc_batch_create(plan.h, self.arr, n, _ptr(choice), _ptr(self.out), self.out.numel(),
                                       _ptr(self.sizes), ctypes.byref(h))
        plan._check(rc, "lfc_batch_create")
        self.h = h

    def launch(self):
        self.plan._check(self.plan.lib.lfc_batch_launch(self.h), "lfc_batch_launch")

    def to_bytes(self):
        sz = self.sizes.cpu().numpy()
        host = self.out.cpu().numpy()
        return [host[o:o + int(s)].tobytes() for o, s in zip(self.offs, sz)]

    def close(self):
        if getattr(self, "h", None):
            self.plan.lib.lfc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def to_device_frame(arr: np.ndarray, device="cuda"):
    """uint16 numpy frame -> contiguous int16 CUDA tensor holding the same bits."""
    torch = _torch()
    a = np.ascontiguousarray(arr, dtype=np.uint16).view(np.int16)
    return torch.from_numpy(a.copy()).to(device)


def from_device_frame(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint16)
