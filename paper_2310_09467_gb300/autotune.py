"""Autotuner of the judge's tile shapes (emission tile width, upper bound on
the pair-chain range per warp, frames per judge launch).

The knobs change speed only, never results. For a batch the tuner times
every setting with CUDA events on the plan's stream, keeps the fastest, and
caches it in a JSON file keyed by the batch geometry and candidate count
(default ``~/.cache/lfc/tune.json``; ``LFC_TUNE_CACHE`` overrides).
"""
from __future__ import annotations

import itertools
import json
import os

SPACE = {
    "emit_tile_lenslets": (4, 8, 16),
    "chain_range_bytes": (32768, 65536, 131072, 262144),
}


def cache_path() -> str:
    return os.environ.get("LFC_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "lfc", "tune.json"))


def batch_key(shapes, pitches, n_candidates: int, temporal: bool) -> str:
    """Key of a batch: sorted (W, H, p) counts, candidates per frame, temporal."""
    cnt = {}
    for (h, w), p in zip(shapes, pitches):
        k = "%dx%dp%d" % (w, h, p)
        cnt[k] = cnt.get(k, 0) + 1
    geo = ",".join("%s*%d" % (k, cnt[k]) for k in sorted(cnt))
    return "%s|K%d|T%d" % (geo, n_candidates, 1 if temporal else 0)


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(max_frames_per_launch: int):
    fpl = sorted({max_frames_per_launch, max(1, max_frames_per_launch // 2)})
    for ts, rb, jf in itertools.product(SPACE["emit_tile_lenslets"], SPACE["chain_range_bytes"], fpl):
        yield {"emit_tile_lenslets": ts, "chain_range_bytes": rb, "judge_frames_per_launch": jf}


def autotune(plan, frames, pitch, prevs=None, reps: int = 2, use_cache: bool = True, n_candidates: int = 26,
             path=None):
    """Pick and set the fastest judge knobs for this batch; returns (knobs, timings)."""
    import torch
    pitches = [pitch] * len(frames) if isinstance(pitch, int) else list(pitch)
    key = batch_key([tuple(f.shape) for f in frames], pitches, n_candidates,
                    prevs is not None and any(p is not None for p in prevs))
    cache = load_cache(path) if use_cache else {}
    if key in cache:
        plan.set_tuning(**cache[key])
        return cache[key], None
    default = plan.get_tuning()
    stream = plan.stream
    timings = []
    for knobs in candidates(default["judge_frames_per_launch"]):
        plan.set_tuning(**knobs)
        plan.judge(frames, pitch, prevs=prevs)  # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            plan.judge(frames, pitch, prevs=prevs)
        b.record(stream)
        b.synchronize()
        timings.append((a.elapsed_time(b) / reps, knobs))
    best = min(timings, key=lambda x: x[0])[1]
    plan.set_tuning(**best)
    if use_cache:
        cache[key] = best
        save_cache(cache, path)
    return best, timings
