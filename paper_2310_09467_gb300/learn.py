"""Training and evaluation of the learned candidate proposal.

Labels come from the exhaustive judge (lfc_judge over the plan's 26
candidates); the network (lfc_cnn_*) is trained with its own forward,
backward and Adam kernels; Python only orders the calls. Evaluation compares
lfc_compress with and without the proposal on held-out frames: total
compressed bytes (ratio loss) and frames per second.
"""
from __future__ import annotations

import time

import numpy as np

PHOTON_LEVELS = (20.0, 200.0, 2000.0)


def make_frames(fields, levels=PHOTON_LEVELS, draws=1, seed0=0):
    """Frames on the device: every field at every photon level, ``draws``
    noise draws each. Cells are scaled to level/4 (their unit level is a
    membrane of ~1.3 photons per unit)."""
    from . import synth
    frames = []
    k = 0
    for kind, sub in fields:
        for lv in levels:
            for _ in range(draws):
                scale = lv * (0.25 if kind == "cells" else 1.0)
                frames.append(synth.photons_to_frame_torch(sub, scale, seed0 + k))
                k += 1
    return frames


def make_dataset(plan, net, fields, pitch, class_ids, levels=PHOTON_LEVELS, draws=1, seed0=0, chunk=8):
    """Thumbnails (FP32, n x 2 x 256 x 256, lfc_cnn_thumbnails) and
    exhaustive-judge labels (lfc_judge) of every field x photon level x noise
    draw. Frames are drawn on the device a chunk at a time and dropped once
    judged, so a training set of thousands of 2040 x 2040 frames keeps only
    its thumbnails (0.5 MB each). The plan and the network must take
    ``chunk`` frames per call."""
    import torch

    from . import synth
    pos = {c: i for i, c in enumerate(class_ids)}
    dev_fields = [(kind, torch.as_tensor(sub, dtype=torch.float32, device="cuda")) for kind, sub in fields]
    specs = [(kind, sub, lv) for kind, sub in dev_fields for lv in levels for _ in range(draws)]
    thumbs, labels = [], []
    for i in range(0, len(specs), chunk):
        frames = []
        for j, (kind, sub, lv) in enumerate(specs[i:i + chunk]):
            scale = lv * (0.25 if kind == "cells" else 1.0)
            frames.append(synth.photons_to_frame_torch(sub, scale, seed0 + i + j))
        ch, _ = plan.judge(frames, pitch)
        labels.extend(pos[int(c)] for c in ch.cpu().numpy())
        thumbs.append(net.thumbnails(frames, pitch, want=True))
    return torch.cat(thumbs), torch.tensor(labels, dtype=torch.int32, device="cuda")


def train_thumbs(net, thumbs, labels, epochs=10, batch=32, lr=2e-3, seed=0, log=None):
    """Adam on mean cross-entropy over stored thumbnails (cosine learning
    rate); returns the per-epoch mean losses."""
    import torch
    rng = np.random.default_rng(seed)
    n = thumbs.shape[0]
    hist = []
    step = 0
    total_steps = epochs * max(1, n // batch)
    for ep in range(epochs):
        order = torch.as_tensor(rng.permutation(n), device="cuda")
        losses = []
        for b0 in range(0, n - batch + 1, batch):
            idx = order[b0:b0 + batch]
            net.set_thumbnails(thumbs[idx])
            loss = net.backward(labels[idx])
            cur_lr = lr * 0.5 * (1 + np.cos(np.pi * step / max(1, total_steps)))
            net.adam_step(float(cur_lr))
            losses.append(loss.mean())
            step += 1
        m = float(torch.stack(losses).mean()) if losses else float("nan")
        hist.append(m)
        if log:
            log("epoch %d loss %.4f" % (ep, m))
    return hist


def accuracy_thumbs(net, thumbs, labels, topk=1, batch=32):
    import torch
    hits = 0
    for b0 in range(0, thumbs.shape[0], batch):
        th = thumbs[b0:b0 + batch]
        net.set_thumbnails(th)
        probs = net.forward(th.shape[0])
        top = torch.topk(probs, topk, dim=1).indices
        hits += int((top == labels[b0:b0 + th.shape[0]].long()[:, None]).any(dim=1).sum())
    return hits / thumbs.shape[0]


def proposal_ms_per_frame(plan, frames, pitch, chunk=8, reps=3):
    """Device time of the proposal alone (lfc_propose: thumbnails, the four
    convolutions, pooling, softmax and the candidate masks) per frame, CUDA
    events on the plan's stream."""
    import torch
    st = plan.stream
    for i in range(0, len(frames), chunk):
        plan.propose(frames[i:i + chunk], pitch)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        for i in range(0, len(frames), chunk):
            plan.propose(frames[i:i + chunk], pitch)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / (reps * len(frames))


def labels_for(plan, frames, pitch, class_ids, chunk=8):
    """Exhaustive-judge choice of every frame as a class index."""
    import torch
    pos = {c: i for i, c in enumerate(class_ids)}
    out = []
    for i in range(0, len(frames), chunk):
        ch, _ = plan.judge(frames[i:i + chunk], pitch)
        out.extend(pos[int(c)] for c in ch.cpu().numpy())
    return torch.tensor(out, dtype=torch.int32, device="cuda")


def train(net, frames, labels, pitch, epochs=20, batch=32, lr=2e-3, seed=0, log=None):
    """Adam on mean cross-entropy; returns the per-epoch mean losses."""
    import torch
    rng = np.random.default_rng(seed)
    n = len(frames)
    hist = []
    step = 0
    total_steps = epochs * max(1, n // batch)
    for ep in range(epochs):
        order = rng.permutation(n)
        losses = []
        for b0 in range(0, n - batch + 1, batch):
            idx = order[b0:b0 + batch]
            net.thumbnails([frames[i] for i in idx], pitch)
            lab = labels[torch.as_tensor(idx, device="cuda")]
            loss = net.backward(lab)
            cur_lr = lr * 0.5 * (1 + np.cos(np.pi * step / max(1, total_steps)))
            net.adam_step(float(cur_lr))
            losses.append(loss.mean())
            step += 1
        m = float(torch.stack(losses).mean()) if losses else float("nan")
        hist.append(m)
        if log:
            log("epoch %d loss %.4f" % (ep, m))
    return hist


def accuracy(net, frames, labels, pitch, topk=1, batch=32):
    import torch
    hits = 0
    for b0 in range(0, len(frames), batch):
        fr = frames[b0:b0 + batch]
        net.thumbnails(fr, pitch)
        probs = net.forward(len(fr))
        top = torch.topk(probs, topk, dim=1).indices
        hits += int((top == labels[b0:b0 + len(fr)].long()[:, None]).any(dim=1).sum())
    return hits / len(frames)


def evaluate(plan, net, class_ids, frames, pitch, settings=((1, 0.0), (3, 0.0), (1, 0.5), (3, 0.5)), chunk=8, reps=2):
    """Compressed bytes and frames/s: exhaustive vs each (topk, tau)."""
    import torch

    def run(setting):
        if setting is None:
            plan.set_proposal(None, class_ids, 1, 0.0)
        else:
            plan.set_proposal(net, class_ids, setting[0], setting[1])
        total = 0
        for i in range(0, len(frames), chunk):
            out, sizes, _ = plan.compress(frames[i:i + chunk], pitch)
            total += int(sizes.sum())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for i in range(0, len(frames), chunk):
                plan.compress(frames[i:i + chunk], pitch)
        torch.cuda.synchronize()
        fps = reps * len(frames) / (time.perf_counter() - t0)
        return total, fps

    base_bytes, base_fps = run(None)
    res = {"exhaustive": {"bytes": base_bytes, "fps": base_fps}}
    for s in settings:
        b, f = run(s)
        res["top%d_tau%.1f" % s] = {"bytes": b, "fps": f, "ratio_loss_pct": 100.0 * (b - base_bytes) / base_bytes,
                                    "speedup": f / base_fps}
    plan.set_proposal(None, class_ids, 1, 0.0)
    return res
