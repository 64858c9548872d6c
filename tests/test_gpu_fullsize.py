"""GPU parity at the full sizes of the long-form, ragged and serving workloads.

The recursion is one FP32 add after an exact max per cell, so every result
(frame tokens, trellis states, per-frame scores, total) must equal the FP32
oracle's bit for bit, for every utterance:

  * long-form: one hour of 20 ms frames, T = 180,000, L = 45,000 (S = 90,001),
    once with full backpointers (a grid team spanning the GPU) and once forced
    through checkpointed recompute, as in the paper's claim that the GPU
    aligner handles long audio (Sec. 4, "CTC-based forced alignment");
  * ragged: all 4,096 utterances of the lognormal-length batch, with C = 32
    and with C = 500, as one packed batched submit;
  * serving: the whole Poisson request stream (2,200 requests) through the
    continuous-batching loop, each result also equal to the request aligned
    alone.

The oracle runs on the host cores while the GPU works (ctypes releases the
GIL during the C call).
"""
import concurrent.futures as cf
import os
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2310_17864_gb300 import align, build, serve, synth

pytestmark = pytest.mark.gpu


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def same_bits(a: np.ndarray, b: np.ndarray) -> bool:
    return np.ascontiguousarray(a).tobytes() == np.ascontiguousarray(b).tobytes()


def check_one(o: dict, path, states, scores, total, label: str):
    assert o["status"] == 0, (label, o["status"])
    assert np.array_equal(path, o["path"]), (label, np.nonzero(path != o["path"])[0][:8])
    assert np.array_equal(states, o["states"]), (label, np.nonzero(states != o["states"])[0][:8])
    assert same_bits(scores, o["scores"]), label
    assert same_bits(np.float32(total), np.float32(o["total"])), (label, total, o["total"])


def test_config3_longform_grid_team_and_checkpointed():
    """T = 180,000, L = 45,000: the default plan (grid team, full 2-bit
    backpointers, about 4.6 GB) and the checkpointed plan both equal the
    oracle (which runs its own segment recompute in bounded host memory)."""
    build.build()
    (s,) = synth.specs(3)
    u = synth.make_utterance(s.seed, s.T, s.C, s.L, s.repeat_frac)
    lp_np = u.lp.numpy()
    ref = {}
    th = threading.Thread(target=lambda: ref.update(o=oracle.viterbi_f32(lp_np, u.targets, 0)))
    th.start()
    lp = u.lp.cuda()
    got = {}
    for name, kw in [("full", {}), ("checkpointed", {"force_checkpoint": True})]:
        a = align.Aligner(device=0, bp_budget_bytes=8 << 30, **kw)
        try:
            r = a.align(lp, u.targets, 0, want_states=True)
            st = a.stats()
            assert r.status == 0, (name, r.status)
            assert st["grid_teams"] == 1, (name, st)
            assert st["checkpointed"] == (1 if name == "checkpointed" else 0), (name, st)
            got[name] = (r.path.cpu().numpy(), r.states.cpu().numpy(), r.scores.cpu().numpy(),
                         r.total.cpu().numpy()[0])
        finally:
            a.close()
    th.join()
    for name, g in got.items():
        check_one(ref["o"], *g, label=f"longform {name}")


@pytest.mark.parametrize("C", [32, 500])
def test_config4_ragged_all_utterances(C):
    """All 4,096 utterances of the ragged workload in one packed batched
    submit; every utterance equals the oracle (run over the host cores in
    chunks, so host memory stays bounded at C = 500)."""
    build.build()
    b = synth.make_batch(synth.specs(4, C=C), device="cuda")
    n = len(b)
    assert n == 4096
    tg = np.concatenate([np.asarray(t, np.int32) for t in b.targets])
    tg_off = np.concatenate([[0], np.cumsum([len(t) for t in b.targets])]).astype(np.int64)
    TT = int(b.offsets[-1])
    out = (torch.empty(TT, dtype=torch.int32, device="cuda"), torch.empty(TT, dtype=torch.float32, device="cuda"),
           torch.empty(n, dtype=torch.float32, device="cuda"), torch.empty(TT, dtype=torch.int32, device="cuda"))
    need = sum(align.align_plan(int(b.offsets[i + 1] - b.offsets[i]), C, len(b.targets[i]), budget=1 << 40)
               ["backpointer_bytes"] for i in range(n))
    a = align.Aligner(device=0, batched=True, bp_budget_bytes=int(1.2 * need) + (1 << 30), max_inflight=2 * n)
    try:
        pr = a.submit_packed(b.lp, b.offsets, tg, tg_off, out)
        a.flush()
        a.wait_packed(pr)
        assert (pr.status == 0).all(), np.nonzero(pr.status)[0][:8]
    finally:
        a.close()
    path, scores, total, states = (x.cpu().numpy() for x in out)
    chunk = 256
    with cf.ThreadPoolExecutor(max_workers=host_cores()) as ex:
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            f0, f1 = int(b.offsets[c0]), int(b.offsets[c1])
            lp_host = b.lp[f0:f1].cpu().numpy()

            def one(i):
                s0, s1 = int(b.offsets[i]) - f0, int(b.offsets[i + 1]) - f0
                return i, oracle.viterbi_f32(lp_host[s0:s1], b.targets[i], 0, max_bp_bytes=256 << 20)

            for i, o in ex.map(one, range(c0, c1)):
                g0, g1 = int(b.offsets[i]), int(b.offsets[i + 1])
                check_one(o, path[g0:g1], states[g0:g1], scores[g0:g1], total[i], f"C{C} utterance {i}")


def test_config5_serving_stream_equals_oracle_and_alone():
    """The whole serving stream (2,200 requests, T lognormal around 1,500
    frames up to 60,000) through the continuous-batching loop with a 16 GiB
    backpointer budget: every result equals the oracle and the same request
    aligned alone."""
    build.build()
    specs = synth.specs(5)
    b = synth.make_batch(specs, device="cuda")
    n = len(b)
    lp_host = b.lp.cpu().numpy()
    ex = cf.ThreadPoolExecutor(max_workers=host_cores())
    futs = [ex.submit(oracle.viterbi_f32, lp_host[int(b.offsets[i]):int(b.offsets[i + 1])], b.targets[i], 0,
                      max_bp_bytes=256 << 20) for i in range(n)]
    alone = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    ref = []
    try:
        for i in range(n):
            r = alone.align(b.utt(i), b.targets[i], 0, want_states=True)
            assert r.status == 0, i
            ref.append((r.path.cpu().numpy(), r.states.cpu().numpy(), r.scores.cpu().numpy(),
                        r.total.cpu().numpy()[0]))
    finally:
        alone.close()
    srv = align.Aligner(device=0, batched=True, bp_budget_bytes=16 << 30)
    try:
        reqs = serve.poisson_requests(b, rate_per_s=40000.0, seed=5)
        for r in reqs:
            T = int(r.log_probs.shape[0])
            r.out = (torch.empty(T, dtype=torch.int32, device="cuda"), torch.empty(T, device="cuda"),
                     torch.empty(1, device="cuda"), torch.empty(T, dtype=torch.int32, device="cuda"))
        st = serve.serve(srv, reqs)
    finally:
        srv.close()
    assert st.n == n and st.max_inflight > 1
    for i, r in enumerate(reqs):
        assert r.result.status == 0, i
        got = (r.out[0].cpu().numpy(), r.out[3].cpu().numpy(), r.out[1].cpu().numpy(), r.out[2].cpu().numpy()[0])
        for x, y in zip(got, ref[i]):
            assert same_bits(np.asarray(x), np.asarray(y)), f"served request {i} differs from alone"
        check_one(futs[i].result(), *got, label=f"served request {i}")
    ex.shutdown()
