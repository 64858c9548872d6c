"""Continuous-batching serving loop for CTC forced alignment.

Requests arrive over time (an arrival schedule, e.g. Poisson). The loop runs
one Aligner in batched mode: at every tick it submits every request that has
arrived since the previous tick in one ``align_submit_batch`` call and
flushes. The library admits queued requests while their backpointer footprint
fits its budget (the rest wait for memory held by running batches), launches
each admitted group as a new batch on its own streams so it overlaps batches
already on the GPU, and reports completions through non-blocking polls.
Latency of a request = completion seen by the loop - its arrival time.

All alignment work runs in the CUDA library; this module only schedules calls.
"""
from __future__ import annotations

import dataclasses
import gc
import time

import numpy as np

from . import align


@dataclasses.dataclass
class Request:
    arrival_s: float
    log_probs: object          # CUDA float32 [T, C] tensor
    targets: np.ndarray        # int32 [L]
    blank: int = 0
    out: tuple | None = None   # (path, scores, total, states) device tensors; allocated if None
    result: align.Result | None = None
    submitted_s: float = 0.0
    done_s: float = 0.0

    @property
    def cells(self) -> int:
        return int(self.log_probs.shape[0]) * (2 * int(self.targets.size) + 1)


@dataclasses.dataclass
class ServeStats:
    n: int
    makespan_s: float
    cells: int
    cells_per_s: float
    latency_ms: np.ndarray
    p50_ms: float
    p99_ms: float
    max_inflight: int
    max_tick_ms: float = 0.0   # longest iteration of the loop (a host stall shows here)

    def as_dict(self) -> dict:
        return {"requests": self.n, "makespan_s": self.makespan_s, "cells": self.cells,
                "cells_per_s": self.cells_per_s, "p50_ms": self.p50_ms, "p99_ms": self.p99_ms,
                "max_inflight": self.max_inflight, "max_tick_ms": self.max_tick_ms}


def _alloc_out(torch, T: int, device):
    return (torch.empty(T, dtype=torch.int32, device=device), torch.empty(T, dtype=torch.float32, device=device),
            torch.empty(1, dtype=torch.float32, device=device), None)


def serve(aligner: align.Aligner, requests: list[Request], *, tick_s: float = 0.0, clock=time.perf_counter,
          warmup: int = 0, freeze_gc: bool = True) -> ServeStats:
    """Run the arrival schedule to completion. ``aligner`` must be in batched mode.
    Arrival times are relative to the start of the run. The first ``warmup``
    requests are served but excluded from the statistics.

    freeze_gc: move every object that exists when the loop starts to the
    collector's permanent generation for the duration of the run, so that a
    full collection (which otherwise scans every object of the process, e.g.
    all of torch's, for tens of milliseconds) does not stall the loop."""
    import torch

    if freeze_gc:
        gc.freeze()
    try:
        return _serve(aligner, requests, tick_s, clock, warmup, torch)
    finally:
        if freeze_gc:
            gc.unfreeze()


def _serve(aligner, requests, tick_s, clock, warmup, torch) -> ServeStats:
    """The loop of serve()."""
    order = sorted(range(len(requests)), key=lambda i: requests[i].arrival_s)
    for r in requests:
        if r.out is None:
            r.out = _alloc_out(torch, int(r.log_probs.shape[0]), r.log_probs.device)
    pending: list[Request] = []
    nxt = 0
    t0 = clock()
    max_inflight = 0
    max_tick = 0.0
    prev = 0.0
    while nxt < len(order) or pending:
        now = clock() - t0
        max_tick = max(max_tick, now - prev)
        prev = now
        arrived = []
        while nxt < len(order) and requests[order[nxt]].arrival_s <= now:
            arrived.append(requests[order[nxt]])
            nxt += 1
        if arrived:
            res = aligner.submit_batch([(r.log_probs, r.targets, r.blank, r.out) for r in arrived])
            for r, x in zip(arrived, res):
                r.result = x
                r.submitted_s = now
            aligner.flush()
            pending.extend(arrived)
        elif pending:
            aligner.flush()  # admit work that waited for memory
        finished = aligner.poll_done()
        if finished:
            t_done = clock() - t0
            ids = {x.request_id for x in finished}
            still = []
            for r in pending:
                if r.result.request_id in ids:
                    r.done_s = t_done
                else:
                    still.append(r)
            pending = still
        max_inflight = max(max_inflight, len(pending))
        if tick_s > 0:
            time.sleep(tick_s)
        elif not arrived and nxt < len(order) and pending == []:
            # Idle until the next arrival.
            gap = requests[order[nxt]].arrival_s - (clock() - t0)
            if gap > 0:
                time.sleep(min(gap, 0.001))
    kept = [requests[i] for i in order[warmup:]]
    lat = np.array([(r.done_s - r.arrival_s) * 1e3 for r in kept])
    t_first = min(r.arrival_s for r in kept)
    t_last = max(r.done_s for r in kept)
    cells = sum(r.cells for r in kept)
    span = max(t_last - t_first, 1e-9)
    return ServeStats(n=len(kept), makespan_s=span, cells=cells, cells_per_s=cells / span, latency_ms=lat,
                      p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                      max_inflight=max_inflight, max_tick_ms=1e3 * max_tick)


def poisson_requests(batch, rate_per_s: float, seed: int) -> list[Request]:
    """One request per utterance of a synth.Batch, arriving as a Poisson process."""
    rng = np.random.default_rng(seed)
    times = np.cumsum(rng.exponential(1.0 / rate_per_s, size=len(batch)))
    times -= times[0]
    return [Request(float(times[i]), batch.utt(i), batch.targets[i]) for i in range(len(batch))]
