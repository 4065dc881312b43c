"""fp64 CPU oracle of the learned candidate proposal.

TEST INFRASTRUCTURE: only tests/, the smoke check and bench.py's baseline
legs use it. The paper only motivates this part (Sec. 4: the time of the
two-dimensional entropy criterion is to be reduced); the network below is this
library's design, written plainly in numpy fp64:

  thumbnail  2 x 256 x 256: channel 0 the raw lenslet layout, channel 1 the
             view-major mosaic; each is averaged over bs x bs blocks
             (bs = ceil(max(W, H) / 256), edge blocks over their valid
             pixels), mapped by log1p(max(v - 100, 0)) / 8, zero-padded;
  conv1      2 -> C, 3 x 3, zero padding 1, bias, ReLU;
  conv2..4   C -> C, same;
  pool       mean over all 256 x 256 positions;
  linear     C -> K logits, bias; softmax; cross-entropy with the label.

The network's stated precision is BF16 weights and activations with FP32
accumulation. ``forward`` and ``backward`` take an optional ``act_round``
applied where a BF16 network stores a tensor: every convolution's output
after its ReLU and, going back, every convolution's pre-activation gradient
after its ReLU mask. With ``bf16`` there (and BF16-rounded inputs and
weights) the fp64 oracle differs from a BF16/FP32 implementation only by the
FP32 accumulation order; without it, it is the exact fp64 network.

Pins: finite differences of the loss (all parameters, tiny sizes), the
convolution against scipy.signal.correlate, softmax-CE gradient in closed form,
the BF16 rounding against hand-worked bit patterns.
"""
from __future__ import annotations

import math

import numpy as np

THUMB = 256


def bf16(a) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as fp64.
    BF16 keeps the sign, the 8-bit exponent and the top 7 mantissa bits of an
    IEEE-754 binary32 value; the value is first taken to binary32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    keep_odd = (u >> 16) & 1
    u = ((u + 0x7FFF + keep_odd) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def block_mean(img: np.ndarray, bs: int) -> np.ndarray:
    H, W = img.shape
    th, tw = -(-H // bs), -(-W // bs)
    out = np.zeros((th, tw))
    for by in range(th):
        for bx in range(tw):
            blk = img[by * bs:(by + 1) * bs, bx * bs:(bx + 1) * bs]
            out[by, bx] = blk.mean()
    return out


def view_major(frame: np.ndarray, p: int) -> np.ndarray:
    """out[v*Ny + t, u*Nx + s] = in[t*p + v, s*p + u]."""
    H, W = frame.shape
    Ny, Nx = H // p, W // p
    return frame.reshape(Ny, p, Nx, p).transpose(1, 0, 3, 2).reshape(H, W)


def thumbnail(frame: np.ndarray, p: int) -> np.ndarray:
    H, W = frame.shape
    bs = -(-max(H, W) // THUMB)
    out = np.zeros((2, THUMB, THUMB))
    for c, img in enumerate((frame.astype(np.float64), view_major(frame, p).astype(np.float64))):
        m = block_mean(img, bs)
        out[c, :m.shape[0], :m.shape[1]] = np.log1p(np.maximum(m - 100.0, 0.0)) / 8.0
    return out


def init_params(C: int, K: int, seed: int = 0, cin: int = 2) -> dict:
    """He-normal convolution weights, zero biases (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    P = {}
    chans = [cin, C, C, C, C]
    for l in range(4):
        fan = chans[l] * 9
        P["w%d" % l] = rng.normal(0, math.sqrt(2.0 / fan), (3, 3, chans[l], chans[l + 1]))
        P["b%d" % l] = np.zeros(chans[l + 1])
    P["wl"] = rng.normal(0, math.sqrt(1.0 / C), (C, K))
    P["bl"] = np.zeros(K)
    return P


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [Cin, H, W], w [3, 3, Cin, Cout] -> [Cout, H, W]; zero padding 1:
    y[co, i, j] = b[co] + sum_{ky, kx, ci} x[ci, i + ky - 1, j + kx - 1] w[ky, kx, ci, co]."""
    Cin, H, W = x.shape
    xp = np.zeros((Cin, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[3], H, W)) + b[:, None, None]
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("chw,cd->dhw", xp[:, ky:ky + H, kx:kx + W], w[ky, kx])
    return y


def forward(P: dict, x: np.ndarray, act_round=None):
    """x [2, H, W] -> (logits [K], cache). act_round, if given, is applied to
    every convolution's output after its ReLU."""
    acts = [x]
    h = x
    for l in range(4):
        h = np.maximum(conv3x3(h, P["w%d" % l], P["b%d" % l]), 0.0)
        if act_round is not None:
            h = act_round(h)
        acts.append(h)
    g = h.mean(axis=(1, 2))
    logits = g @ P["wl"] + P["bl"]
    return logits, (acts, g)


def softmax(z: np.ndarray) -> np.ndarray:
    e = np.exp(z - z.max())
    return e / e.sum()


def loss(P: dict, x: np.ndarray, label: int) -> float:
    logits, _ = forward(P, x)
    return float(-np.log(softmax(logits)[label]))


def backward(P: dict, x: np.ndarray, label: int, act_round=None):
    """Gradients of the cross-entropy loss with respect to every parameter.
    act_round, if given, is applied to the stored activations (as in
    forward) and to every pre-activation gradient after the ReLU mask."""
    logits, (acts, g) = forward(P, x, act_round)
    dz = softmax(logits)
    dz[label] -= 1.0                                   # d loss / d logits
    G = {"wl": np.outer(g, dz), "bl": dz.copy()}
    dg = P["wl"] @ dz
    h = acts[4]
    dh = np.broadcast_to(dg[:, None, None] / (h.shape[1] * h.shape[2]), h.shape).copy()
    for l in range(3, -1, -1):
        dpre = dh * (acts[l + 1] > 0)                  # through the ReLU
        if act_round is not None:
            dpre = act_round(dpre)
        xin = acts[l]
        Cin, H, W = xin.shape
        xp = np.zeros((Cin, H + 2, W + 2))
        xp[:, 1:-1, 1:-1] = xin
        w = P["w%d" % l]
        dw = np.zeros_like(w)
        for ky in range(3):
            for kx in range(3):
                dw[ky, kx] = np.einsum("chw,dhw->cd", xp[:, ky:ky + H, kx:kx + W], dpre)
        G["w%d" % l] = dw
        G["b%d" % l] = dpre.sum(axis=(1, 2))
        # input gradient: correlation with the flipped, transposed kernel
        dpp = np.zeros((dpre.shape[0], H + 2, W + 2))
        dpp[:, 1:-1, 1:-1] = dpre
        dx = np.zeros_like(xin)
        for ky in range(3):
            for kx in range(3):
                dx += np.einsum("dhw,cd->chw", dpp[:, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W], w[ky, kx])
        dh = dx
    return G
