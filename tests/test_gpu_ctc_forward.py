"""GPU parity of the sum-product variant (ALIGN_REQ_SUM): the CTC forward
score over the same trellis, with log-add in place of the max.

Tolerance (tests/ctc_forward_bounds.py derives it): the kernel works in FP32
and in base 2 with the hardware 2^x and log2(x); per frame the two FP32 adds
round by at most 2^-23 |beta_t| (natural-log units), the emission's base
change by 1.5 * 2^-23 |e|, the log-add by 2^-20, and a log-sum-exp does not
amplify errors carried from earlier frames (a convex combination). The test
sums these over the frames with |beta_t| bounded by the binary64 oracle's
largest |beta_t(s)| over the states that can still reach the end. Closed
forms at large S (per-frame emissions equal across classes, so every path's
score is known and the paths are counted exactly) pin the cluster and grid
team paths with a bound small enough that dropping a final state or the last
frame's emission fails.
"""
import numpy as np
import pytest
import torch

import ctc_forward_bounds as cfb
import oracle
from paper_2310_17864_gb300 import align, build, synth

pytestmark = pytest.mark.gpu


def check(status, total, lp, targets, blank, label=""):
    o = oracle.ctc_forward_f64(lp, np.asarray(targets, np.int32), blank, live_abs_max=True)
    assert status == o["status"], (label, status, o["status"])
    if o["status"] != 0:
        assert total == -np.inf, (label, total)
        return o
    tol = cfb.tolerance(lp, o["amax"], o["total"])
    assert abs(total - o["total"]) <= tol, (label, total, o["total"], tol)
    return o


@pytest.fixture(scope="module")
def al():
    build.build()
    a = align.Aligner(device=0, batched=True, bp_budget_bytes=4 << 30)
    yield a
    a.close()


def packed(us, device="cuda"):
    lp = torch.cat([u.lp for u in us]).contiguous()
    offsets = np.concatenate([[0], np.cumsum([u.lp.shape[0] for u in us])])
    tg = np.concatenate([np.asarray(u.targets, np.int32) for u in us] + [np.zeros(0, np.int32)])
    tg_off = np.concatenate([[0], np.cumsum([len(u.targets) for u in us])])
    return lp.to(device), offsets, tg, tg_off


@pytest.mark.parametrize("T,C,L", [
    (1, 2, 0), (1, 4, 1), (2, 2, 1), (3, 3, 2), (7, 5, 3), (50, 2, 1), (64, 32, 0),
    (300, 32, 63), (300, 32, 64), (900, 32, 255), (900, 32, 256), (3000, 32, 1023),
    (3000, 32, 1024), (400, 29, 90), (333, 3, 100), (2000, 500, 400),
])
def test_shapes(al, T, C, L):
    u = synth.make_utterance(T * 37 + L, T, C, L, repeat_frac=0.1)
    st, tot = al.ctc_forward(u.lp.cuda(), u.targets, 0)
    check(st, tot, u.lp.numpy(), u.targets, 0, f"T{T}C{C}L{L}")


def test_packed_batch_device_and_host(al):
    """A ragged packed batch (device and pinned host buffers): every total
    within the bound of the oracle's, one request per utterance."""
    specs = synth.specs(4, C=32, n=24)
    us = [synth.make_utterance(s.seed, s.T, s.C, s.L, s.repeat_frac) for s in specs]
    for host in (False, True):
        lp, off, tg, tg_off = packed(us, "cpu" if host else "cuda")
        if host:
            lp = lp.pin_memory()
            total = torch.empty(len(us), dtype=torch.float32).pin_memory()
        else:
            total = torch.empty(len(us), dtype=torch.float32, device="cuda")
        pr = al.ctc_forward_packed(lp, off, tg, tg_off, total, host=host)
        al.flush()
        al.wait_packed(pr)
        tt = total.cpu().numpy()
        for i, u in enumerate(us):
            check(int(pr.status[i]), float(tt[i]), u.lp.numpy(), u.targets, 0, f"host{host}utt{i}")


@pytest.mark.parametrize("K,cw", [(2, 1), (2, 16), (4, 4), (8, 4), (16, 2)])
def test_launch_shapes(K, cw):
    """Every (states per lane, warps per CTA) shape, clusters of one-warp CTAs
    included, and wide rows (C = 500)."""
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        a.set_tuning(K, cw, 16)
        for (T, C, L, seed) in [(700, 32, 300, 11), (333, 500, 120, 12), (95, 29, 40, 13), (1200, 32, 500, 15)]:
            u = synth.make_utterance(seed * 1000 + K * 10 + cw, T, C, L, repeat_frac=0.1)
            st, tot = a.ctc_forward(u.lp.cuda(), u.targets, 0)
            check(st, tot, u.lp.numpy(), u.targets, 0, f"K{K}cw{cw}T{T}C{C}")
    finally:
        a.close()


def test_grid_team():
    """With clusters limited to one CTA, a transcript beyond one CTA runs as a
    grid team of one-warp CTAs linked through global memory."""
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        a.set_tuning(4, 1, 1)
        for (T, L, seed) in [(1500, 700, 3), (600, 290, 4)]:
            u = synth.make_utterance(seed, T, 32, L, repeat_frac=0.1)
            st, tot = a.ctc_forward(u.lp.cuda(), u.targets, 0)
            check(st, tot, u.lp.numpy(), u.targets, 0, f"grid T{T}")
        stt = a.stats()
        assert stt["grid_teams"] == 2 and stt["sum_requests"] == 2, stt
    finally:
        a.close()


def test_minus_inf_and_nopath(al):
    """-inf emissions prune paths; when none is left the status is no-path
    and the total -inf, as in the oracle."""
    rng = np.random.default_rng(9)
    lp = rng.standard_normal((40, 6)).astype(np.float32)
    lp[rng.random(lp.shape) < 0.3] = -np.inf
    tg = np.array([1, 2, 3], np.int32)
    st, tot = al.ctc_forward(torch.from_numpy(lp).cuda(), tg, 0)
    check(st, tot, lp, tg, 0, "pruned")
    lp2 = rng.standard_normal((10, 6)).astype(np.float32)
    lp2[4, :] = -np.inf
    st, tot = al.ctc_forward(torch.from_numpy(lp2).cuda(), tg, 0)
    assert st == align.ALIGN_E_NOPATH and tot == -np.inf


def test_sum_and_viterbi_in_one_batch(al):
    """Sum-product and Viterbi requests of one flush run as separate shape
    groups: each result equals the oracle's."""
    us = [synth.make_utterance(70 + i, 400 + 50 * i, 32, 100 + 20 * i) for i in range(6)]
    lp, off, tg, tg_off = packed(us)
    TT, n = int(off[-1]), len(us)
    tot_sum = torch.empty(n, dtype=torch.float32, device="cuda")
    out = (torch.empty(TT, dtype=torch.int32, device="cuda"), torch.empty(TT, device="cuda"),
           torch.empty(n, device="cuda"), torch.empty(TT, dtype=torch.int32, device="cuda"))
    p1 = al.ctc_forward_packed(lp, off, tg, tg_off, tot_sum)
    p2 = al.submit_packed(lp, off, tg, tg_off, out)
    al.flush()
    al.wait_packed(p1)
    al.wait_packed(p2)
    for i, u in enumerate(us):
        check(int(p1.status[i]), float(tot_sum[i].item()), u.lp.numpy(), u.targets, 0, f"sum{i}")
        o = oracle.viterbi_f32(u.lp.numpy(), np.asarray(u.targets, np.int32), 0)
        f0, f1 = int(off[i]), int(off[i + 1])
        assert np.array_equal(out[0][f0:f1].cpu().numpy(), o["path"])
        assert np.float32(out[2][i].item()).tobytes() == np.float32(o["total"]).tobytes()
        assert tot_sum[i].item() >= out[2][i].item()  # the sum is at least its largest term


def test_logits_flag_rejected(al):
    """The sum-product takes log-probabilities only."""
    u = synth.make_utterance(5, 50, 8, 5)
    reqs = np.zeros(1, dtype=align._REQ_DTYPE)
    tg = np.asarray(u.targets, np.int32)
    lp = u.lp.cuda()
    total = torch.empty(1, device="cuda")
    reqs["lp"], reqs["T"], reqs["C"], reqs["tg"], reqs["L"] = lp.data_ptr(), 50, 8, tg.ctypes.data, tg.size
    reqs["flags"] = align.ALIGN_REQ_SUM | align.ALIGN_REQ_LOGITS
    reqs["total"] = total.data_ptr()
    with pytest.raises(align.AlignError) as e:
        align.align_submit_batch(al.ctx, reqs)
    assert e.value.code == align.ALIGN_E_INVAL


@pytest.mark.parametrize("L,spare,team", [(2980, 20, "cluster"), (10000, 20, "grid")])
def test_closed_form_large_S(L, spare, team):
    """Exact totals from path counts at S = 5,961 (a thread-block cluster) and
    S = 20,001 (a grid team over the GPU's SMs), default plans."""
    build.build()
    lp, tg, exact, tol = cfb.closed_form_case(L, spare)
    T = lp.shape[0]
    plan = align.align_plan(T, 32, L, budget=4 << 30)
    a = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        st, tot = a.ctc_forward(torch.from_numpy(lp).cuda(), tg, 0)
        grid = a.stats()["grid_teams"]
    finally:
        a.close()
    assert st == 0
    if team == "grid":
        assert grid == 1
    else:
        assert grid == 0 and plan["cluster_ctas"] > 1
    assert abs(tot - exact) <= tol, (tot, exact, tol)
