"""GPU parity of logits inputs (ALIGN_REQ_LOGITS) against the FP64
log_softmax oracle.

log_softmax subtracts one value per frame, lse_t, from every class of frame
t, so the best CTC path over the log-probabilities is the best path over the
raw logits (the sum over any path differs by the same sum of lse_t). The fast
kernel therefore runs the Viterbi recursion on the logits unchanged and, in
its score pass, computes lse_t = m + logf(sum_c expf(x - m)) for each frame
and scores[t] = x[t][path[t]] - lse_t; the total is the sum of the scores in a
fixed tree order. (Checkpointed requests run the generic kernel, whose lse
pre-pass subtracts __expf-based shifts from the emissions inside the
recursion.) Tolerances, derived from the FP32 operations:
  per frame |lp_gpu - lp64| <= (C + 6 + 2.4 d) * 2^-24 + 2^-22 (|lse64| + |lp64|),
  d = the largest |x - m| of the row: C * 2^-24 for the FP32 sum of C
  exponentials of non-positive numbers, (2 + 1.2 d) * 2^-23 for the
  exponentials (covering __expf's 2 + floor(1.173 |x|) ulps and expf's few
  ulps with the error of x - m), 4 * 2^-24 for logf on values in [1, C],
  2^-22 (|lse| + |lp|) for the roundings of m + log s and of x - lse;
  total: |total - sum(scores)| <= gamma_T * sum |scores| (any summation order);
  path: optimal for the FP64 log-probabilities up to twice the summed
  per-frame bound plus twice the FP32 fold error of a path sum of logits,
  gamma_T * sum_t max_c |x[t][c]| (the recursion's adds on raw logits).
Checked besides: the alignment is legal and collapses to the transcript."""
import numpy as np
import pytest
import torch

import oracle
from oracle import checks, normalize
from paper_2310_17864_gb300 import align, build, synth

pytestmark = pytest.mark.gpu


def check(res, logits, targets, label=""):
    x = np.asarray(logits, dtype=np.float32)
    T, C = x.shape
    targets = np.asarray(targets, np.int32)
    lp64, lse64 = normalize.log_softmax64(x)
    assert res.status == 0, (label, res.status)
    path = res.path.cpu().numpy()
    states = res.states.cpu().numpy()
    sc = res.scores.cpu().numpy()
    assert checks.legal_state_path(states, targets, 0), label
    assert checks.collapse(path, 0) == targets.tolist(), label
    ref = lp64[np.arange(T), path]
    xf = np.where(np.isfinite(x), x, np.nan)
    d = np.nan_to_num(np.nanmax(xf, axis=1) - np.nanmin(xf, axis=1))
    tol = (C + 6 + 2.4 * d) * 2.0 ** -24 + 2.0 ** -22 * (np.abs(lse64) + np.abs(ref))
    err = np.abs(sc.astype(np.float64) - ref)
    assert (err <= tol).all(), (label, float(err.max()), int(np.argmax(err - tol)))
    total = float(res.total.cpu().numpy()[0])
    sc64 = sc.astype(np.float64)
    assert abs(total - sc64.sum()) <= checks.gamma(T) * float(np.abs(sc64).sum()) + 1e-30, (label, total, sc64.sum())
    finite = np.where(np.isfinite(lp64), np.abs(lp64), 0.0)
    rowmax = finite.max(axis=1)
    E = float(((C + 6 + 2.4 * d) * 2.0 ** -24 + 2.0 ** -22 * (np.abs(lse64) + rowmax)).sum())
    E += checks.gamma(T) * float(rowmax.sum()) + float((2.0 ** -24 * rowmax).sum())
    E += checks.gamma(T) * float(np.nan_to_num(np.nanmax(np.abs(xf), axis=1)).sum())
    best = oracle.viterbi_f64(lp64.astype(np.float32), targets, 0)
    assert best["status"] == 0
    assert ref.sum() >= best["total"] - 2 * E, (label, ref.sum(), best["total"], E)


def run(al, u, label):
    r = al.align(u.lp.cuda(), u.targets, 0, want_states=True, logits=True)
    check(r, u.lp.numpy(), u.targets, label)


@pytest.fixture(scope="module")
def al():
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=8 << 30)
    yield a
    a.close()


@pytest.mark.parametrize("T,C,L", [(1, 4, 0), (1, 6, 1), (2, 5, 1), (200, 32, 40), (3000, 32, 700),
                                   (500, 500, 120), (333, 29, 90), (12000, 32, 3000), (64, 3, 20)])
def test_logits_shapes(al, T, C, L):
    u = synth.make_utterance(T * 7 + L, T, C, L, repeat_frac=0.1, logits=True)
    run(al, u, f"T{T}C{C}L{L}")


@pytest.mark.parametrize("K,cw", [(2, 1), (2, 15), (4, 4), (8, 2), (16, 1)])
def test_logits_launch_shapes(K, cw):
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        a.set_tuning(K, cw, 16)
        for (T, C, L, s) in [(700, 32, 300, 1), (400, 500, 100, 2)]:
            run(a, synth.make_utterance(s * 100 + K, T, C, L, repeat_frac=0.1, logits=True), f"K{K}cw{cw}C{C}")
    finally:
        a.close()


def test_logits_checkpointed_and_grid_team():
    build.build()
    ck = align.Aligner(device=0, force_checkpoint=True, bp_budget_bytes=4 << 30)
    try:
        run(ck, synth.make_utterance(91, 3000, 32, 700, repeat_frac=0.1, logits=True), "checkpointed")
    finally:
        ck.close()
    g = align.Aligner(device=0, bp_budget_bytes=8 << 30)
    try:
        run(g, synth.make_utterance(92, 34000, 32, 16500, logits=True), "grid team")
    finally:
        g.close()


def test_logits_and_log_probs_in_one_batch_and_host():
    """Logits and log-probability requests share a batch (separate launch
    groups); logits through host buffers too; and a logits request gives the
    same alignment as the log-probabilities computed from the kernel's own
    scores would, in FP32: the batched result equals the single one."""
    build.build()
    us = [synth.make_utterance(200 + i, 600 + 50 * i, 32, 150, logits=True) for i in range(4)]
    lps = [synth.make_utterance(300 + i, 500, 32, 100) for i in range(3)]
    al = align.Aligner(device=0, batched=True, bp_budget_bytes=4 << 30)
    one = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        mk = lambda T, host: tuple(torch.empty(n, dtype=dt, pin_memory=host) if host else
                                   torch.empty(n, dtype=dt, device="cuda")
                                   for n, dt in ((T, torch.int32), (T, torch.float32), (1, torch.float32),
                                                 (T, torch.int32)))
        rl = al.submit_batch([(u.lp.cuda(), u.targets, 0, mk(u.T, False)) for u in us], logits=True)
        rp = al.submit_batch([(u.lp.cuda(), u.targets, 0, mk(u.T, False)) for u in lps])
        rh = al.submit_batch([(u.lp.pin_memory(), u.targets, 0, mk(u.T, True)) for u in us], host=True, logits=True)
        al.flush()
        al.wait(rl + rp + rh)
        for u, r, h in zip(us, rl, rh):
            check(r, u.lp.numpy(), u.targets, "batched logits")
            ref = one.align(u.lp.cuda(), u.targets, 0, logits=True)
            assert torch.equal(r.path, ref.path) and torch.equal(h.path, ref.path.cpu())
            assert torch.equal(r.scores.view(torch.int32), ref.scores.view(torch.int32))
        for u, r in zip(lps, rp):
            o = oracle.viterbi_f32(u.lp.numpy(), np.asarray(u.targets, np.int32), 0)
            assert np.array_equal(r.path.cpu().numpy(), o["path"])
    finally:
        al.close()
        one.close()
