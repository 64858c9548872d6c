#!/usr/bin/env python3
"""Benchmark: CTC forced alignment (Viterbi over the CTC trellis) on GB300.

Headline workload (batch64): 64 utterances, T uniform in 500..3000 frames
(20 ms), C=32 classes, L=round(T/4) targets, FP32 synthetic log-probabilities
(seeded; 3*N(0,1) logits with +4 on a planted feasible path, log_softmax).
One step = the whole hot path (validate, expand, forward max-plus recursion,
2-bit backpointers and anchor rows, final state, backtrack, scores) for the
whole batch. Legs measured the same way, each with its own roofline, in
"legs": plain1 (one utterance, T=200, L=40), longform (one utterance,
T=180000, L=45000, also checkpointed), ragged32 / ragged500 (4096 utterances,
lognormal lengths, C=32 / C=500), and persistent launches of two of them. --workload picks the
headline workload instead (plain1, batch64, longform, ragged32, ragged500).

Metric: trellis cells per second, cells = sum over utterances of T * (2L+1).
  value  : batched launch through the C ABI (one packed align_submit_batch),
           inputs resident in device memory, device time between CUDA events
           on the submitting stream (L2 flushed before every timed step by
           writing a 256 MiB buffer).
  e2e    : same metric through the host-buffer path of align_submit_batch
           (pinned host emissions, host->device and device->host copies inside
           the timed region), host wall clock from the submit to the last poll.
  plain  : one synchronous submit+poll per utterance (reported beside).
  serving: (batch64 only) workload 5 through the continuous-batching loop:
           2,000 requests per offered load after 200 warm-up requests.
With --gpus N > 1 (torchrun), every rank aligns its own copy of the batch (no
data-path collective; weak scaling); value is the sum of cells over ranks
divided by the slowest rank's time.

--impl reference times the CPU oracle (plain C, FP32) on this host's cores on
the same workload, the same input bytes (generated on the GPU when there is
one, as the GPU arm does, then copied to the host) and the same metric (a
bounded sample per step for large workloads).
--profile runs only warm-up + steps batches (no extras) for profilers.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trellis cells/s (T*S)"
WORKLOADS = {
    "batch64": {"cfg": 2, "C": None, "name": "batch64_T500-3000_C32_L=T/4"},
    "plain1": {"cfg": 1, "C": None, "name": "plain1_T200_C32_L40"},
    "longform": {"cfg": 3, "C": None, "name": "longform_T180000_C32_L45000"},
    "ragged32": {"cfg": 4, "C": 32, "name": "ragged4096_lognormal800_C32"},
    "ragged500": {"cfg": 4, "C": 500, "name": "ragged4096_lognormal800_C500"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="batch64", choices=sorted(WORKLOADS))
    ap.add_argument("--no-spans", action="store_true", help="skip the token-span leg")
    ap.add_argument("--no-logits", action="store_true", help="skip the fused log_softmax leg")
    ap.add_argument("--no-sum", action="store_true", help="skip the sum-product (CTC forward) leg")
    ap.add_argument("--no-beam", action="store_true", help="skip the CTC beam-search decoder leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000, help="timed requests per offered load")
    ap.add_argument("--serving-warmup", type=int, default=200, help="warm-up requests before them")
    ap.add_argument("--no-legs", action="store_true", help="skip the long-form and ragged legs")
    ap.add_argument("--leg-steps", type=int, default=10, help="timed steps of each leg")
    ap.add_argument("--profile", action="store_true", help="only warm-up + steps batches, for profilers")
    ap.add_argument("--profile-utts", type=int, default=0, metavar="N",
                    help="with --profile: only the workload's first N utterances (a small capture)")
    ap.add_argument("--profile-beam", type=int, default=0, metavar="N",
                    help="only warm-up + steps decoder calls on a batch of N utterances, for profilers")
    return ap.parse_args()


def input_digest(t, limit_bytes: int = 512 << 20) -> str:
    """SHA-256 of a tensor's bytes (the seeded synthetic inputs of a run), or a
    note when the tensor is too large to copy to the host for it."""
    import hashlib
    nbytes = t.numel() * t.element_size()
    if nbytes > limit_bytes:
        return f"not computed ({nbytes} bytes)"
    return hashlib.sha256(t.detach().cpu().contiguous().numpy().tobytes()).hexdigest()


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_items(batch, max_cells: float):
    """Utterances of the batch (host arrays), the first ones up to max_cells cells.
    A single utterance far larger than that (the hour-long one) is replaced by an
    utterance of the same shape family ten times shorter."""
    T0 = int(batch.offsets[1] - batch.offsets[0])
    c0 = T0 * (2 * len(batch.targets[0]) + 1)
    if len(batch) == 1 and c0 > 10 * max_cells:
        from paper_2310_17864_gb300 import synth
        s = batch.specs[0]
        u = synth.make_utterance(s.seed, s.T // 10, s.C, s.L // 10, s.repeat_frac)
        c = u.T * (2 * u.L + 1)
        return [(u.lp.numpy(), u.targets, c)], c
    lp = batch.lp.cpu().numpy()
    items, cells = [], 0
    for i in range(len(batch)):
        T = int(batch.offsets[i + 1] - batch.offsets[i])
        c = T * (2 * len(batch.targets[i]) + 1)
        if items and cells + c > max_cells:
            break
        items.append((lp[batch.offsets[i]:batch.offsets[i + 1]], batch.targets[i], c))
        cells += c
    return items, cells


def oracle_pass(ex, items):
    import oracle
    # Huge problems (the hour-long utterance) run the oracle's forward-only total.
    list(ex.map(lambda it: oracle.viterbi_f32(it[0], it[1], 0) if it[2] < 4e9
                else oracle.viterbi_total_f32(it[0], it[1], 0), items))


def cpu_oracle_rate(batch, seconds: float) -> dict:
    """The oracle as it stands on all host cores (one utterance per task) over
    repeated passes of a bounded sample of the workload, for about `seconds`."""
    import concurrent.futures as cf

    import oracle
    oracle.lib()
    n = cores()
    items, cells = oracle_items(batch, 2.5e8)
    t0 = time.perf_counter()
    passes = 0
    with cf.ThreadPoolExecutor(max_workers=n) as ex:  # ctypes releases the GIL during the C call
        while True:
            oracle_pass(ex, items)
            passes += 1
            if time.perf_counter() - t0 > seconds or passes >= 1000:
                break
    dt = time.perf_counter() - t0
    return {"value": passes * cells / dt, "unit": "cells/s", "cores": n, "kind": "oracle",
            "sample": f"{passes} pass(es) over the first {len(items)} of {len(batch)} utterances "
                      f"({cells} cells per pass), {n} threads, {dt:.1f} s"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def serving_run(align, serve, synth, autotune, dev: int, n: int, warmup: int, persistent: bool = False) -> dict:
    """Workload 5: Poisson arrivals served by the continuous-batching loop with a
    16 GiB backpointer budget. Saturation = every request arriving at time 0;
    then offered loads of 0.5, 0.8 and 0.95 times the saturation request rate.
    Each run serves `warmup` + `n` requests of the stream; the first `warmup`
    (by arrival) are excluded from its statistics."""
    b = synth.make_batch(synth.specs(5, n=n + warmup), device=f"cuda:{dev}")
    al = align.Aligner(device=dev, batched=True, bp_budget_bytes=16 << 30, persistent=persistent)
    autotune.apply(al)
    try:
        warm = serve.poisson_requests(b, rate_per_s=1e9, seed=1)
        serve.serve(al, warm, warmup=warmup)
        sat_reqs = [serve.Request(0.0, r.log_probs, r.targets) for r in warm]
        sat = serve.serve(al, sat_reqs, warmup=warmup)
        rate_sat = sat.n / sat.makespan_s
        out = {"requests": n, "warmup_requests": warmup,
               "saturation": {**sat.as_dict(), "requests_per_s": rate_sat}, "loads": {}}
        for frac in (0.5, 0.8, 0.95):
            reqs = serve.poisson_requests(b, rate_per_s=frac * rate_sat, seed=int(frac * 100))
            st = serve.serve(al, reqs, warmup=warmup)
            out["loads"][str(frac)] = {**st.as_dict(), "offered_requests_per_s": frac * rate_sat}
        out["persistent_batches"] = al.stats()["persistent_batches"]
        return out
    finally:
        al.close()


def make_workload_batch(wl, device: str, n: int | None = None):
    """The workload's synthetic batch (its first n utterances if n is given)."""
    from paper_2310_17864_gb300 import synth
    return synth.make_batch(synth.specs(wl["cfg"], C=wl["C"], n=n), device=device)


def packed_targets(batch):
    tg = np.concatenate([np.asarray(t, np.int32) for t in batch.targets] + [np.zeros(0, np.int32)])
    tg_off = np.concatenate([[0], np.cumsum([len(t) for t in batch.targets])]).astype(np.int64)
    return tg, tg_off


def reference_arm(args, wl):
    """The oracle, as it stands, on the host cores: same workload, same input
    bytes as the GPU arm (generated with the same device generator when a GPU
    is present, then copied to the host), same metric."""
    import concurrent.futures as cf

    import oracle
    import torch
    gen_dev = "cuda:0" if torch.cuda.is_available() else "cpu"
    batch = make_workload_batch(wl, gen_dev)
    digest = input_digest(batch.lp)
    if gen_dev != "cpu":
        batch.lp = batch.lp.cpu()
    oracle.lib()
    items, cells = oracle_items(batch, 2.5e8)
    n = cores()
    steps = []
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle_pass(ex, items)
            if k >= args.warmup:
                steps.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(steps)
    value = cells / (ms / 1e3)
    sample = (f"first {len(items)} of {len(batch)} utterances ({cells} of {batch.cells} cells) per step, "
              f"{n} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"], "utterances": len(batch), "cells_per_step": cells,
                   "input_sha256": digest, "inputs_generated_on": gen_dev},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": n, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


class DeviceTimer:
    """Device time of one submitted batch between CUDA events on the
    submitting stream. The stream is held by a device-side sleep while the
    host enqueues, so the events time device work only; the hold is calibrated
    to twice the slowest enqueue seen (at least 20 ms). L2 is flushed (256 MiB
    write, above the 129 MB L2) before every step."""

    def __init__(self, torch, stream, flush_buf):
        self.torch, self.stream, self.flush_buf = torch, stream, flush_buf
        self.cycles = 40_000_000
        self.enqueue_max = 0.0
        self.enqueue = []

    def step(self, al, enqueue, finish) -> float:
        torch = self.torch
        self.flush_buf.fill_(1)
        with torch.cuda.stream(self.stream):
            torch.cuda._sleep(self.cycles)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(self.stream)
            h0 = time.perf_counter()
            handle = enqueue()
            al.join(self.stream)
            ev1.record(self.stream)
            h1 = time.perf_counter()
        finish(handle)
        ev1.synchronize()
        self.enqueue.append(h1 - h0)
        self.enqueue_max = max(self.enqueue_max, h1 - h0)
        self.cycles = max(40_000_000, int(2 * self.enqueue_max * 2.0e9))
        return ev0.elapsed_time(ev1)


def roofline_of(batch, ms: float, t_frame_ns: float, peaks: dict, sm_count: int) -> dict:
    """Three lower bounds on one step: HBM bytes at the measured copy
    bandwidth, the per-frame dependency chain of the longest utterance (T_max
    frames at the measured null-work frame time), and ALU issue (6 operations
    per cell at the SM count and clock). The largest binds; frac = bound / time."""
    n = len(batch)
    T_of = [int(batch.offsets[i + 1] - batch.offsets[i]) for i in range(n)]
    cells = batch.cells
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "MEASURED_PEAKS.json" if peaks else "fallback 6800 GB/s"
    # Algorithmic bytes: emissions read once, 2 bits of backpointer per cell
    # written and read back once, outputs (path, scores, total) written.
    em_bytes = int(batch.lp.numel()) * 4
    out_bytes = sum(T * 8 + 4 for T in T_of)
    alg_bytes = em_bytes + 2 * cells * 2 / 8 + out_bytes
    hbm_s = alg_bytes / (hbm_peak * 1e9)
    T_max = max(T_of)
    chain_s = T_max * t_frame_ns * 1e-9
    sm_hz = 2.07e9
    ops_per_cell = 6  # compare + select per candidate (2 or 3) and one add, averaged over blank/label states
    alu_s = cells * ops_per_cell / (sm_count * 128 * sm_hz)
    terms = {"hbm": hbm_s, "latency": chain_s, "alu": alu_s}
    bound = max(terms, key=terms.get)
    if bound == "latency":
        rl = {"bound": "latency", "achieved": T_max / (ms / 1e3), "peak": 1e9 / t_frame_ns, "unit": "frames/s"}
    elif bound == "hbm":
        rl = {"bound": "hbm", "achieved": alg_bytes / (ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s"}
    else:
        rl = {"bound": "alu", "achieved": cells * ops_per_cell / (ms / 1e3) / 1e12,
              "peak": sm_count * 128 * sm_hz / 1e12, "unit": "Top/s"}
    rl.update({"frac": terms[bound] / (ms / 1e3), "traffic": None,
               "terms_us": {k: v * 1e6 for k, v in terms.items()}, "t_frame_ns": t_frame_ns,
               "alg_bytes_per_step": alg_bytes, "hbm_gbs": alg_bytes / (ms / 1e3) / 1e9,
               "hbm_peak_gbs": hbm_peak,
               "peak_source": f"{peak_src} (HBM, of measured); null-work frame probe measured in this run (latency)"})
    return rl


def run_batched(torch, align, autotune, replicas, batch, dev, stream, flush_buf, steps, warmup, dist, clocks=None,
                force_checkpoint=False, persistent=False):
    """Device-timed packed-batch steps of one workload. Returns the step
    times, kernel launches per step, enqueue times and the aligner's budget."""
    n = len(batch)
    C = int(batch.lp.shape[1])
    tg, tg_off = packed_targets(batch)
    TT = int(batch.offsets[-1])
    out = (torch.empty(TT, dtype=torch.int32, device=dev), torch.empty(TT, dtype=torch.float32, device=dev),
           torch.empty(n, dtype=torch.float32, device=dev), None)
    need = sum(align.align_plan(int(batch.offsets[i + 1] - batch.offsets[i]), C, len(batch.targets[i]),
                                budget=1 << 40)["backpointer_bytes"] for i in range(n))
    budget = max(4 << 30, int(1.2 * need) + (256 << 20))
    al = align.Aligner(device=dev, batched=True, stream=stream, bp_budget_bytes=budget,
                       max_inflight=max(8192, 2 * n), force_checkpoint=force_checkpoint, persistent=persistent)
    tuned = autotune.apply(al)
    timer = DeviceTimer(torch, stream, flush_buf)

    def enqueue():
        pr = al.submit_packed(batch.lp, batch.offsets, tg, tg_off, out)
        al.flush()
        return pr

    def finish(pr):
        al.wait_packed(pr)
        assert (pr.status == 0).all(), pr.status[pr.status != 0][:4]

    try:
        for _ in range(warmup):
            timer.step(al, enqueue, finish)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        timer.enqueue = []
        st0 = al.stats()
        times = []
        if clocks is not None:
            with clocks:
                for _ in range(steps):
                    times.append(timer.step(al, enqueue, finish))
        else:
            for _ in range(steps):
                times.append(timer.step(al, enqueue, finish))
        st1 = al.stats()
        torch.cuda.synchronize()
    finally:
        al.close()
    launches = (st1["kernel_launches"] - st0["kernel_launches"]) // max(steps, 1)
    tp = (st1["throughput_batches"] - st0["throughput_batches"]) / max(steps, 1)
    ck = (st1["checkpointed"] - st0["checkpointed"]) / max(steps, 1)
    pb = (st1["persistent_batches"] - st0["persistent_batches"]) / max(steps, 1)
    ms = replicas.slowest(statistics.mean(times), dist, dev)
    return {"times": times, "ms": ms, "launches": int(launches), "tp_batches": tp, "tuned": tuned,
            "enqueue_ms_median": 1e3 * statistics.median(timer.enqueue), "budget": budget, "out": out,
            "checkpointed_per_step": ck, "persistent_batches_per_step": pb}


def run_e2e(torch, align, autotune, replicas, batch, dev, budget, steps, dist, world):
    """End to end through the host-buffer path of align_submit_batch: the
    batch as a user holds it (one packed pinned host tensor of emissions,
    packed targets and outputs); copies in and results out inside the timed
    region. Two steps in flight (step k+1 submitted before step k's results are
    waited for, host outputs double-buffered), and one step at a time."""
    n = len(batch)
    host_lp = batch.lp.cpu().pin_memory()
    tg_packed, tg_off = packed_targets(batch)
    total_T = int(batch.offsets[-1])
    mk = lambda: (torch.empty(total_T, dtype=torch.int32).pin_memory(),
                  torch.empty(total_T, dtype=torch.float32).pin_memory(),
                  torch.empty(n, dtype=torch.float32).pin_memory(), None)
    host_out, host_out2 = mk(), mk()
    h2d = host_lp.numel() * 4 + tg_packed.size * 4
    d2h = total_T * 8 + n * 4
    ha = align.Aligner(device=dev, batched=True, bp_budget_bytes=2 * budget, max_inflight=max(8192, 4 * n),
                       staging_bytes=min(int(2.6 * (h2d + d2h)) + (64 << 20), 32 << 30))
    autotune.apply(ha)
    enq = []

    def e2e_step(out):
        h0 = time.perf_counter()
        pr = ha.submit_packed(host_lp, batch.offsets, tg_packed, tg_off, out, host=True)
        ha.flush()
        enq.append(time.perf_counter() - h0)
        return pr

    try:
        e_times = []
        for k in range(2 + max(3, steps // 4)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pr = e2e_step(host_out)
            ha.wait_packed(pr)
            assert (pr.status == 0).all(), pr.status[pr.status != 0][:4]
            if k >= 2:
                e_times.append(time.perf_counter() - t0)
        sync_ms = 1e3 * statistics.mean(e_times)
        n_pipe = max(8, steps)
        torch.cuda.synchronize()
        for _ in range(2):
            ha.wait_packed(e2e_step(host_out))
        enq.clear()
        t0 = time.perf_counter()
        prev = None
        for k in range(n_pipe):
            pr = e2e_step(host_out if k % 2 == 0 else host_out2)
            if prev is not None:
                ha.wait_packed(prev)
                assert (prev.status == 0).all()
            prev = pr
        ha.wait_packed(prev)
        assert (prev.status == 0).all()
        e_ms = replicas.slowest(1e3 * (time.perf_counter() - t0) / n_pipe, dist, dev)
        sync_ms = replicas.slowest(sync_ms, dist, dev)
    finally:
        ha.close()
    cells = batch.cells
    return {"value": replicas.job_rate(cells, world, e_ms), "unit": "cells/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "steps_in_flight": 2,
            "host_submit_ms_median": 1e3 * statistics.median(enq),
            "one_step_at_a_time": {"ms_per_step": sync_ms, "value": replicas.job_rate(cells, world, sync_ms)}}


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":  # the CPU oracle: rank 0 alone runs and prints it
        if rank == 0:
            reference_arm(args, wl)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_17864_gb300 import align, autotune, replicas, synth

    if args.profile_beam:  # only decoder calls (vocabulary 500, beam 10), for profilers
        nb = args.profile_beam
        probs, off = synth.decoder_batch(synth.config_seed(7) + nb, nb, 500, device="cpu")
        probs = probs.to(dev)
        for _ in range(args.warmup + args.steps):
            r = align.ctc_beam_decode(probs, off, beam=10, blank=0, threshold=0.95)
        torch.cuda.synchronize()
        print(json.dumps({"profile": f"beam_decode_batch{nb}_V500_B10_a0.95", "calls": args.warmup + args.steps,
                          "kept_frames": int(r.kept.sum().item()), "frames": int(off[-1])}))
        return

    batch = make_workload_batch(wl, f"cuda:{dev}", n=(args.profile_utts or None) if args.profile else None)
    n = len(batch)
    cells = batch.cells
    C = int(batch.lp.shape[1])
    T_of = [int(batch.offsets[i + 1] - batch.offsets[i]) for i in range(n)]
    L_of = [len(t) for t in batch.targets]
    T_max = max(T_of)
    utts = [batch.utt(i) for i in range(n)]
    stream = torch.cuda.Stream(dev)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    if args.profile:
        tg, tg_off = packed_targets(batch)
        TT = int(batch.offsets[-1])
        out = (torch.empty(TT, dtype=torch.int32, device=dev), torch.empty(TT, dtype=torch.float32, device=dev),
               torch.empty(n, dtype=torch.float32, device=dev), None)
        need = sum(align.align_plan(T_of[i], C, L_of[i], budget=1 << 40)["backpointer_bytes"] for i in range(n))
        al = align.Aligner(device=dev, batched=True, stream=stream, bp_budget_bytes=max(4 << 30, int(1.2 * need)),
                           max_inflight=max(8192, 2 * n))
        autotune.apply(al)
        for _ in range(args.warmup + args.steps):
            pr = al.submit_packed(batch.lp, batch.offsets, tg, tg_off, out)
            al.flush()
            al.wait_packed(pr)
        torch.cuda.synchronize()
        launches = al.stats()["kernel_launches"]
        al.close()
        print(json.dumps({"profile": wl["name"], "batches": args.warmup + args.steps, "kernel_launches": launches}))
        return

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    t_frame_ns = align.align_probe_frame_latency(dev, 1, 1, 200000)

    clk = Clocks(dev)
    head = run_batched(torch, align, autotune, replicas, batch, dev, stream, flush_buf, args.steps, args.warmup,
                       dist, clocks=clk)
    times, ms, launches = head["times"], head["ms"], head["launches"]
    value = replicas.job_rate(cells, world, ms)
    budget = head["budget"]
    outs = []
    for i in range(n):
        f0, f1 = int(batch.offsets[i]), int(batch.offsets[i + 1])
        outs.append((torch.empty(f1 - f0, dtype=torch.int32, device=dev),
                     torch.empty(f1 - f0, dtype=torch.float32, device=dev),
                     torch.empty(1, dtype=torch.float32, device=dev), None))
    al = align.Aligner(device=dev, batched=True, stream=stream, bp_budget_bytes=budget, max_inflight=max(8192, 2 * n))
    autotune.apply(al)
    timer = DeviceTimer(torch, stream, flush_buf)
    timer.cycles = max(timer.cycles, int(2 * head["enqueue_ms_median"] * 1e-3 * 2.0e9))

    # Token spans (per transcript token: start, end, mean score) of this batch's
    # alignments: one packed call, timed with events on its stream.
    spans_line = None
    if not args.no_spans:
        sp_out = [(o[0], o[1], o[2], torch.empty(T, dtype=torch.int32, device=dev)) for o, T in zip(outs, T_of)]
        rs = al.submit_batch([(utts[i], batch.targets[i], 0, sp_out[i]) for i in range(n)])
        al.flush()
        al.wait(rs)
        assert all(r.status == 0 for r in rs)
        st_all = torch.cat([o[3] for o in sp_out])
        sc_all = torch.cat([o[1] for o in sp_out])
        tg_off = np.concatenate([[0], np.cumsum(L_of)]).astype(np.int64)
        fo_d = torch.as_tensor(np.asarray(batch.offsets, dtype=np.int64), device=dev)
        to_d = torch.as_tensor(tg_off, device=dev)
        totals = (int(batch.offsets[-1]), int(tg_off[-1]))
        sp_times = []
        with torch.cuda.stream(stream):
            for k in range(3 + args.steps):
                flush_buf.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                align.token_spans(st_all, sc_all, fo_d, to_d, stream=stream, totals=totals)
                e1.record(stream)
                e1.synchronize()
                if k >= 3:
                    sp_times.append(e0.elapsed_time(e1))
        sp_ms = statistics.mean(sp_times)
        n_tok = int(tg_off[-1])
        sp_bytes = int(st_all.numel()) * 8 + n_tok * 12  # states + scores read, start/end/score written
        spans_line = {"ms": sp_ms, "tokens": n_tok, "frames": int(st_all.numel()),
                      "tokens_per_s": n_tok / (sp_ms / 1e3), "alg_bytes": sp_bytes,
                      "gbs": sp_bytes / (sp_ms / 1e3) / 1e9, "launches": 2,
                      "note": "two memsets and two kernels on device-resident offsets; L2 flushed before each"}

    # Logits inputs: log_softmax fused into the kernel's staging (one request
    # flag) against a separate log_softmax pass over the packed [sum T, C]
    # logits followed by the log-probability path; same batch, device time.
    logits_line = None
    if not args.no_logits:
        lb = synth.make_batch(synth.specs(wl["cfg"], C=wl["C"]), device=f"cuda:{dev}", logits=True)
        l_utts = [lb.utt(i) for i in range(n)]
        lp_buf = torch.empty_like(lb.lp)
        lp_utts = [lp_buf[int(lb.offsets[i]):int(lb.offsets[i + 1])] for i in range(n)]

        def timed(fn):
            ts = []
            for k in range(3 + args.steps):
                flush_buf.fill_(1)
                with torch.cuda.stream(stream):
                    torch.cuda._sleep(timer.cycles)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    rs = fn()
                    al.join(stream)
                    e1.record(stream)
                al.wait(rs)
                assert all(r.status == 0 for r in rs)
                e1.synchronize()
                if k >= 3:
                    ts.append(e0.elapsed_time(e1))
            return statistics.mean(ts)

        def fused():
            rs = al.submit_batch([(l_utts[i], lb.targets[i], 0, outs[i]) for i in range(n)], logits=True)
            al.flush()
            return rs

        def separate():
            torch.log_softmax(lb.lp, dim=-1, out=lp_buf)
            rs = al.submit_batch([(lp_utts[i], lb.targets[i], 0, outs[i]) for i in range(n)])
            al.flush()
            return rs

        f_ms = timed(fused)
        s_ms = timed(separate)
        logits_line = {"fused_ms": f_ms, "separate_ms": s_ms, "fused_cells_per_s": cells / (f_ms / 1e3),
                       "separate_cells_per_s": cells / (s_ms / 1e3),
                       "separate": "torch.log_softmax over the packed logits, then the log-probability path",
                       "logit_bytes": int(lb.lp.numel()) * 4}
        del lb, lp_buf

    # Sum-product (ALIGN_REQ_SUM): the CTC forward score of every utterance of
    # the same batch over the same trellis (log-add in place of the max, no
    # backpointers, no backtrack), as one packed submit; device time.
    sum_line = None
    if not args.no_sum:
        tg_pk = np.concatenate([np.asarray(t, np.int32) for t in batch.targets])
        tgo_pk = np.concatenate([[0], np.cumsum(L_of)]).astype(np.int64)
        tot_sum = torch.empty(n, dtype=torch.float32, device=dev)
        su_times = []
        for k in range(3 + args.steps):
            flush_buf.fill_(1)
            with torch.cuda.stream(stream):
                torch.cuda._sleep(timer.cycles)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pr = al.ctc_forward_packed(batch.lp, batch.offsets, tg_pk, tgo_pk, tot_sum)
                al.flush()
                al.join(stream)
                e1.record(stream)
            al.wait_packed(pr)
            assert (pr.status == 0).all()
            e1.synchronize()
            if k >= 3:
                su_times.append(e0.elapsed_time(e1))
        su_ms = statistics.mean(su_times)
        sum_line = {"ms": su_ms, "cells_per_s": cells / (su_ms / 1e3), "viterbi_ms": ms,
                    "note": "log-add in base 2 (max factored out, hardware ex2 / lg2) in place of the max; total only"}

    # CTC beam search with blank collapse (the paper's CUDA decoder setting:
    # vocabulary 500, beam 10, batch 4; and a batch of 2 utterances per SM),
    # thresholds a = 0.95 and a = 1.0 (no collapse); device time per call,
    # L2 flushed before each. Frames/s counts every input frame.
    beam_line = None
    if not args.no_beam:
        beam_line = {"V": 500, "beam": 10, "T": "U[250,1750] frames", "runs": []}
        for nb in (4, 2 * torch.cuda.get_device_properties(dev).multi_processor_count):
            probs, off = synth.decoder_batch(synth.config_seed(7) + nb, nb, 500, device="cpu")
            probs = probs.to(dev)
            frames = int(off[-1])
            ws = torch.empty(align.align_ctc_beam_workspace_bytes(nb, frames, 10), dtype=torch.uint8, device=dev)
            for a in (0.95, 1.0):
                bt = []
                for k in range(3 + args.steps):
                    flush_buf.fill_(1)
                    with torch.cuda.stream(stream):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        r = align.ctc_beam_decode(probs, off, beam=10, blank=0, threshold=a, stream=stream,
                                                  workspace=ws)
                        e1.record(stream)
                    e1.synchronize()
                    if k >= 3:
                        bt.append(e0.elapsed_time(e1))
                b_ms = statistics.mean(bt)
                kept = r.kept.cpu().numpy().astype(np.int64)
                Ts = np.diff(off)
                alg = int(kept.sum()) * 500 * 4 + frames * 32  # kept rows once + one sector per frame (blank column)
                beam_line["runs"].append({
                    "batch": nb, "a": a, "ms": b_ms, "frames": frames, "kept_frames": int(kept.sum()),
                    "frames_per_s": frames / (b_ms / 1e3),
                    "ns_per_kept_frame_longest": b_ms * 1e6 / int(kept.max()),
                    "longest_T": int(Ts.max()), "alg_bytes": alg, "gbs": alg / (b_ms / 1e3) / 1e9})
            del probs, ws

    # Plain: one synchronous submit + poll per utterance (at most 256 utterances).
    plain = None
    if not args.no_plain:
        pl = align.Aligner(device=dev, stream=stream, bp_budget_bytes=budget)
        autotune.apply(pl)
        m = min(n, 256)
        lat = []
        dt = 0.0
        for k in range(2):
            flush_buf.fill_(1)
            torch.cuda.synchronize()
            t_all = time.perf_counter()
            for i in range(m):
                t0 = time.perf_counter()
                r = pl.submit(utts[i], batch.targets[i], 0, out=outs[i])
                pl.poll(r)
                if k == 1:
                    lat.append(time.perf_counter() - t0)
            dt = time.perf_counter() - t_all
        pl.close()
        pcells = sum(T_of[i] * (2 * L_of[i] + 1) for i in range(m))
        lat_ms = np.array(lat) * 1e3
        plain = {"value": pcells / dt, "unit": "cells/s", "utterances": m,
                 "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                 "launch": "one synchronous launch per utterance"}


    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, align, autotune, replicas, batch, dev, budget, args.steps, dist, world)

    serving = None
    if not args.no_serving and args.workload == "batch64":
        from paper_2310_17864_gb300 import serve
        serving = serving_run(align, serve, synth, autotune, dev, args.serving_requests, args.serving_warmup)
        # The same streams with ALIGN_F_PERSISTENT: every tick's batch as one
        # persistent launch.
        serving["with_persistent_launch"] = serving_run(align, serve, synth, autotune, dev, args.serving_requests,
                                                        args.serving_warmup, persistent=True)
    al.close()

    # The other single-GPU workloads, each with its own roofline (legs).
    legs = None
    if not args.no_legs:
        legs = {}
        # (leg, workload, forced checkpointed recompute, persistent launch)
        for name, wname, ck, ps in (("plain1", "plain1", False, False),
                                    ("longform", "longform", False, False),
                                    ("longform_checkpointed", "longform", True, False),
                                    ("ragged32", "ragged32", False, False),
                                    ("ragged32_persistent", "ragged32", False, True),
                                    ("ragged500", "ragged500", False, False),
                                    ("batch64_persistent", "batch64", False, True)):
            if wname == args.workload and not ck and not ps:
                continue
            lw = WORKLOADS[wname]
            lb = make_workload_batch(lw, f"cuda:{dev}")
            lclk = Clocks(dev)
            r = run_batched(torch, align, autotune, replicas, lb, dev, stream, flush_buf,
                            max(3, args.leg_steps // 2) if ck else args.leg_steps, max(3, args.warmup // 2), dist,
                            clocks=lclk, force_checkpoint=ck, persistent=ps)
            leg = {"metric": METRIC, "value": replicas.job_rate(lb.cells, world, r["ms"]), "unit": "cells/s",
                   "ms_per_step": r["ms"], "steps": len(r["times"]),
                   "p50_ms": float(np.percentile(r["times"], 50)), "p99_ms": float(np.percentile(r["times"], 99)),
                   "gpu_launches": r["launches"],
                   "config": {"workload": lw["name"], "utterances": len(lb), "cells_per_step": lb.cells,
                              "T_max": int(np.max(np.diff(lb.offsets))),
                              "l2": "flushed (256 MiB write) before every timed step",
                              "host_enqueue_ms_median": round(r["enqueue_ms_median"], 3),
                              "throughput_batches_per_step": r["tp_batches"],
                              "checkpointed_requests_per_step": r["checkpointed_per_step"],
                              "persistent_batches_per_step": r["persistent_batches_per_step"],
                              "input_sha256": input_digest(lb.lp)},
                   "roofline": roofline_of(lb, r["ms"], t_frame_ns, peaks, sm_count),
                   "clocks": lclk.summary()}
            if name == "ragged32" and not args.no_e2e:
                leg["e2e"] = run_e2e(torch, align, autotune, replicas, lb, dev, r["budget"], args.leg_steps, dist,
                                     world)
            legs[name] = leg
            del lb, r
            torch.cuda.empty_cache()

    if not replicas.prints(rank):
        if dist:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_rate(batch, args.cpu_seconds)

    rl = roofline_of(batch, ms, t_frame_ns, peaks, sm_count)
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"], "utterances": n, "cells_per_step": cells, "T_max": T_max,
                   "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"replicas{world}",
                   "tuning": ({"latency": autotune.load(mode="latency"), "throughput": autotune.load(mode="throughput"),
                              "throughput_batches_per_step": head["tp_batches"]}
                             if head["tuned"] else "built-in default (K=4, 4 warps per CTA)"),
                   "host_enqueue_ms_median": round(head["enqueue_ms_median"], 3),
                   "input_sha256": input_digest(batch.lp)},
        "p50_ms": float(np.percentile(times, 50)), "p99_ms": float(np.percentile(times, 99)),
        "plain": plain,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": rl,
        "legs": legs,
        "serving": serving,
        "token_spans": spans_line,
        "logits": logits_line,
        "ctc_forward": sum_line,
        "beam_decode": beam_line,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
