"""Autotuner of the trellis kernel shape per range of transcript length.

For every range of trellis sizes S (upper edges in ``BUCKETS``) it times each
candidate shape -- states per lane K and warps per CTA before a transcript is
split over a thread-block cluster -- on seeded synthetic utterances of that
size, checks that every candidate returns bit-identical results, and keeps
the fastest. Two criteria:

  * ``latency``: one utterance alone (the per-frame chain of a single team);
  * ``throughput``: a batch of utterances of that size filling the GPU.

The two tables are installed with ``align_set_tuning_bucket_for`` (the
library plans a batch with the throughput table when it oversubscribes the
GPU, else with the latency table) and saved as JSON with the GPU name, one
key per mode, for later runs. A bucket keeps the shape of the table it
started from (``prior``) unless another shape is faster by more than
``margin``: shapes within the run-to-run spread of each other are a tie, and
a tie does not move the table. Usage:

    python -m paper_2310_17864_gb300.autotune --mode both --out tuning.json
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

from . import align, synth

BUCKETS = (128, 256, 512, 1024, 2048, 4096, 8192, 16384)
KS = (2, 4, 8, 16)
CTA_WARPS = (1, 2, 4, 8, 16)
DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def _device_ms(torch, al, st, items, reps: int) -> tuple[float, list]:
    """Device time of one batch between events on `st`, the stream the context
    forks its batches from (held by a sleep while the host enqueues)."""
    times, res = [], None
    for _ in range(reps):
        with torch.cuda.stream(st):
            torch.cuda._sleep(20_000_000)  # hold the stream while the host enqueues
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            res = al.submit_batch(items)
            al.flush()
            al.join(st)
            e1.record(st)
        for r in res:
            al.poll(r)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times), res


def choose(times: dict, prior=None, margin: float = 0.0):
    """The shape of one bucket from its measured times {(K, cta_warps): ms}:
    the fastest, unless ``prior`` was measured within ``margin`` (a fraction)
    of it, which then stays."""
    best = min(times, key=lambda k: (times[k], k))
    if prior is not None and prior in times and times[prior] <= times[best] * (1.0 + margin):
        return prior
    return best


def tune(device: int = 0, mode: str = "latency", buckets=BUCKETS, C: int = 32, reps: int = 3,
         verbose: bool = False, prior=None, margin: float = 0.0) -> dict:
    """Measure every candidate per bucket; returns {"table": [(s_max, K, cta_warps)], "trials": {...}}.
    ``prior``: a table [(s_max, K, cta_warps)] whose shape a bucket keeps on a tie (see ``choose``)."""
    import torch

    prior_of = {int(s): (int(k), int(w)) for s, k, w in (prior or [])}

    table, trials = [], {}
    for bi, s_hi in enumerate(buckets):
        L = (s_hi - 1) // 2
        T = 4 * L                      # 20 ms frames, about four frames per character (L = T/4)
        n = 1 if mode == "latency" else max(1, min(512, (1 << 28) // max(T * s_hi, 1)))
        specs = [synth.Spec(T, C, L, 0.0, synth.sub_seed(synth.BASE_SEED + 90 + bi, i)) for i in range(n)]
        b = synth.make_batch(specs, device=f"cuda:{device}")
        ref_paths = None
        times = {}
        for K in KS:
            for cw in CTA_WARPS:
                try:
                    align.align_plan(T, C, L, budget=64 << 30, states_per_lane=K, cta_warps=cw)
                except align.AlignError:
                    continue
                st = torch.cuda.Stream(device)
                al = align.Aligner(device=device, batched=True, bp_budget_bytes=8 << 30, graphs=False, stream=st)
                try:
                    al.set_tuning(K, cw, 0)
                    if mode == "throughput":
                        # Batches that oversubscribe the GPU run the throughput build of
                        # the kernel; let the library choose as it does in service.
                        al.set_tuning_table([(1 << 30, K, cw)], "throughput")
                    outs = [(torch.empty(s.T, dtype=torch.int32, device=f"cuda:{device}"),
                             torch.empty(s.T, device=f"cuda:{device}"),
                             torch.empty(1, device=f"cuda:{device}"), None) for s in specs]
                    items = [(b.utt(i), b.targets[i], 0, outs[i]) for i in range(n)]
                    ms, res = _device_ms(torch, al, st, items, reps)
                finally:
                    al.close()
                paths = torch.cat([o[0] for o in outs]).cpu()
                if ref_paths is None:
                    ref_paths = paths
                elif not torch.equal(paths, ref_paths):
                    raise RuntimeError(f"shape K={K} cta_warps={cw} changed the alignment (S={s_hi})")
                trials[f"S{s_hi}_K{K}_cw{cw}"] = ms
                if verbose:
                    print(f"S<={s_hi:6d} K={K:2d} cta_warps={cw:2d}: {ms:8.3f} ms", flush=True)
                times[(K, cw)] = ms
        K, cw = choose(times, prior_of.get(s_hi), margin)
        table.append((s_hi, K, cw))
    return {"mode": mode, "table": table, "trials": trials}


def save(result: dict, path: str, device: int = 0) -> None:
    """Store the table of ``result["mode"]`` (and its trials) in ``path``,
    keeping the other mode's table if the file has one."""
    import torch
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data["gpu"] = torch.cuda.get_device_name(device)
    data[result["mode"]] = result["table"]
    data.setdefault("trials", {})[result["mode"]] = result["trials"]
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load(path: str = DEFAULT_TABLE, mode: str = "latency") -> list | None:
    """The table of ``mode`` saved by ``save``, or None when absent."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    table = data.get(mode)
    return [tuple(x) for x in table] if table else None


def apply(aligner: align.Aligner, path: str = DEFAULT_TABLE) -> bool:
    """Install every table found in ``path``; True if there was one."""
    found = False
    for mode in ("latency", "throughput"):
        table = load(path, mode)
        if table:
            aligner.set_tuning_table(table, mode)
            found = True
    return found


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--mode", choices=["latency", "throughput", "both"], default="both")
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--prior", default=DEFAULT_TABLE,
                    help="table whose shapes a bucket keeps on a tie ('' for none)")
    ap.add_argument("--margin", type=float, default=0.03,
                    help="a new shape must be faster than the prior one by this fraction")
    args = ap.parse_args()
    for mode in (("latency", "throughput") if args.mode == "both" else (args.mode,)):
        prior = load(args.prior, mode) if args.prior else None
        res = tune(args.device, mode, reps=args.reps, verbose=True, prior=prior, margin=args.margin)
        save(res, args.out, args.device)
        print(mode, json.dumps(res["table"]))


if __name__ == "__main__":
    main()
