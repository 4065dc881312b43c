"""Streaming harness: frames arrive at camera rate, are grouped into
micro-batches of a fixed composition and compressed by one CUDA-graph launch
per micro-batch (lfc_batch_*). Latency of a frame = time its container is
ready minus its arrival time.

Host timing: arrivals follow a fixed schedule (t_i = i / fps from the start);
a micro-batch launches as soon as its last frame has arrived and the previous
launch has completed; completion is observed with a CUDA event.
"""
from __future__ import annotations

import statistics
import time


def run_stream(plan, frames_np, pitches, micro: int, fps: float, prevs_fn=None, to_device=None):
    """frames_np: list of uint16 arrays (arrival order); micro-batches are
    consecutive groups of ``micro`` frames and must share one composition.
    Returns a dict with p50/p99/max latency (ms) and achieved frames/s."""
    import torch
    n = len(frames_np) - len(frames_np) % micro
    slots = [torch.empty(frames_np[i].shape, dtype=torch.int16, device="cuda") for i in range(micro)]
    host = [torch.from_numpy(f.view("int16")).pin_memory() for f in frames_np[:n]]
    prevs = prevs_fn(slots) if prevs_fn else None
    batch = plan.batch(slots, pitches[:micro], prevs=prevs)
    stream = plan.stream
    # warm-up launch (graph upload)
    batch.launch()
    torch.cuda.synchronize()
    lat = []
    t0 = time.perf_counter()
    done_ev = None
    for b0 in range(0, n, micro):
        last_arrival = t0 + (b0 + micro - 1) / fps
        while True:  # wait for the last frame of the micro-batch to arrive
            now = time.perf_counter()
            if now >= last_arrival:
                break
            time.sleep(min(0.0005, last_arrival - now))
        if done_ev is not None:
            done_ev.synchronize()
        with torch.cuda.stream(stream):
            for k in range(micro):
                slots[k].copy_(host[b0 + k], non_blocking=True)
        batch.launch()
        done_ev = torch.cuda.Event()
        done_ev.record(stream)
        done_ev.synchronize()
        t_done = time.perf_counter()
        for k in range(micro):
            lat.append(1e3 * (t_done - (t0 + (b0 + k) / fps)))
    total = time.perf_counter() - t0
    batch.close()
    lat_sorted = sorted(lat)
    return {"frames": n, "micro_batch": micro, "arrival_fps": fps, "p50_ms": statistics.median(lat),
            "p99_ms": lat_sorted[min(len(lat) - 1, int(0.99 * len(lat)))], "max_ms": lat_sorted[-1],
            "achieved_fps": n / total}
