"""GPU parity of the persistent launch (ALIGN_F_PERSISTENT).

A batch whose requests all qualify runs as one cooperative launch in which
resident CTAs take the requests' seats from a device counter, longest chain
first; a request of several CTAs links them through global memory. The
recursion is the same FP32 max-plus as every other launch, so paths, states,
per-frame scores and totals must equal the FP32 oracle bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import checks
from paper_2310_17864_gb300 import align, build, synth

pytestmark = pytest.mark.gpu


def compare(res, lp_np, targets, blank, label=""):
    o = oracle.viterbi_f32(lp_np, targets, blank)
    assert res.status == o["status"], (label, res.status, o["status"])
    if o["status"] != 0:
        return
    path = res.path.cpu().numpy()
    assert np.array_equal(path, o["path"]), (label, np.nonzero(path != o["path"])[0][:10])
    if res.states is not None:
        assert np.array_equal(res.states.cpu().numpy(), o["states"]), label
    assert res.scores.cpu().numpy().tobytes() == o["scores"].tobytes(), label
    assert np.float32(res.total.cpu().numpy()[0]).tobytes() == np.float32(o["total"]).tobytes(), label


def outs(T):
    return (torch.empty(T, dtype=torch.int32, device="cuda"), torch.empty(T, device="cuda"),
            torch.empty(1, device="cuda"), torch.empty(T, dtype=torch.int32, device="cuda"))


def run_batch(al, utts, label):
    """Submits [(lp (T, C) float32 numpy, targets)] as one batch, flushes,
    checks every result against the oracle."""
    lps = [torch.as_tensor(np.ascontiguousarray(lp, np.float32)).cuda() for lp, _ in utts]
    rs = al.submit_batch([(lps[i], utts[i][1], 0, outs(lps[i].shape[0])) for i in range(len(utts))])
    al.flush()
    for r in rs:
        al.poll(r)
    for i, r in enumerate(rs):
        compare(r, utts[i][0], np.asarray(utts[i][1], np.int32), 0, f"{label}[{i}]")
    return rs


def mixed_batch(seed, C, n_small, big):
    """n_small utterances of 50..1500 frames and 5..300 labels, the (T, L) of
    `big`, and the degenerate cases (one frame, no labels)."""
    rng = np.random.default_rng(seed)
    utts = []
    for k in range(n_small):
        L = int(rng.integers(5, 300))
        T = int(rng.integers(2 * L + 2, 2 * L + 1200))
        u = synth.make_utterance(seed * 1000 + k, T, C, L, repeat_frac=0.1)
        utts.append((u.lp.numpy(), u.targets))
    for k, (T, L) in enumerate(big):
        u = synth.make_utterance(seed * 1000 + 500 + k, T, C, L, repeat_frac=0.1)
        utts.append((u.lp.numpy(), u.targets))
    for k, (T, L) in enumerate([(1, 0), (2, 1), (100, 0), (37, 18)]):
        u = synth.make_utterance(seed * 1000 + 900 + k, T, C, L)
        utts.append((u.lp.numpy(), u.targets))
    return utts


@pytest.fixture(scope="module")
def pal():
    build.build()
    a = align.Aligner(device=0, batched=True, persistent=True, bp_budget_bytes=8 << 30)
    # One shape for every batch: K = 4, two compute warps (256 states per CTA),
    # so transcripts of more than 127 labels take teams of several CTAs.
    for mode in ("latency", "throughput"):
        a.set_tuning_table([(1 << 30, 4, 2)], mode=mode)
    yield a
    a.close()


def test_window_mode_teams_and_edges(pal):
    """C = 32 (whole 32-frame windows per hand-off): one-CTA requests, teams
    of 2..12 CTAs (S up to 3,001) and the degenerate cases in one launch."""
    before = pal.stats()["persistent_batches"]
    utts = mixed_batch(1, 32, 40, [(3000, 1500), (2400, 1000), (1800, 700), (900, 300)])
    run_batch(pal, utts, "win")
    assert pal.stats()["persistent_batches"] == before + 1


def test_block_mode_wide_vocabulary(pal):
    """C = 500 (packages of 4 frames per hand-off) with a multi-CTA team."""
    before = pal.stats()["persistent_batches"]
    utts = mixed_batch(2, 500, 10, [(1500, 600)])
    run_batch(pal, utts, "blk")
    assert pal.stats()["persistent_batches"] == before + 1


def test_every_last_window_length(pal):
    """T - 1 = 32 q + r for every r: the last (partial) window of every length,
    single- and multi-CTA, in one persistent launch."""
    utts = []
    for r in range(32):
        for L in (20, 200):
            T = 2 * L + 64 + r + 1
            u = synth.make_utterance(7000 + 100 * r + L, T, 32, L)
            utts.append((u.lp.numpy(), u.targets))
    run_batch(pal, utts, "tail")


def test_more_seats_than_resident_ctas():
    """3,000 utterances of the ragged C = 32 workload: more seats than resident
    CTAs, so CTAs run job after job (the emission ring's phases carry over).
    Every result satisfies the invariants, a sample matches the oracle."""
    build.build()
    specs = synth.specs(4, C=32, n=3000)
    b = synth.make_batch(specs, device="cuda")
    a = align.Aligner(device=0, batched=True, persistent=True, bp_budget_bytes=16 << 30)
    try:
        rs = a.submit_batch([(b.utt(i), b.targets[i], 0, outs(specs[i].T)) for i in range(len(b))])
        a.flush()
        for r in rs:
            a.poll(r)
        st = a.stats()
        assert st["persistent_batches"] >= 1
        lp_host = b.lp.cpu().numpy()
        for i, r in enumerate(rs):
            assert r.status == 0, (i, r.status)
            path = r.path.cpu().numpy()
            assert checks.collapse(path, 0) == b.targets[i].tolist()
            sl = lp_host[b.offsets[i]:b.offsets[i + 1]]
            assert (r.scores.cpu().numpy() == sl[np.arange(sl.shape[0]), path]).all()
            assert checks.fold_f32_fast(r.scores.cpu().numpy()) == r.total.cpu().numpy()[0]
            if i % 60 == 0:
                compare(r, sl, b.targets[i], 0, f"ragged[{i}]")
    finally:
        a.close()


def test_ineligible_batches_launch_per_shape_group(pal):
    """A batch over two vocabularies is not persistent; its results are the
    same."""
    before = pal.stats()["persistent_batches"]
    u = synth.make_utterance(11, 400, 32, 100)
    v = synth.make_utterance(12, 300, 40, 80)
    lu = torch.as_tensor(u.lp.numpy()).cuda()
    lv = torch.as_tensor(v.lp.numpy()).cuda()
    rs = pal.submit_batch([(lu, u.targets, 0, outs(400)), (lv, v.targets, 0, outs(300))])
    pal.flush()
    for r in rs:
        pal.poll(r)
    compare(rs[0], u.lp.numpy(), u.targets, 0, "C32")
    compare(rs[1], v.lp.numpy(), v.targets, 0, "C40")
    assert pal.stats()["persistent_batches"] == before


def test_watchdog_in_persistent_launch():
    """The stall hook (the first warp of a team never hands its values on):
    with two compute warps per CTA every request ends with ALIGN_E_TIMEOUT
    after the wait limit, and a later context runs normally."""
    build.build()
    st = align.Aligner(device=0, batched=True, persistent=True, wait_limit_ms=50, test_stall=True)
    for mode in ("latency", "throughput"):
        st.set_tuning_table([(1 << 30, 4, 2)], mode=mode)
    utts = [synth.make_utterance(20 + k, 300, 32, 100) for k in range(6)]   # S = 201: two warps
    one = synth.make_utterance(30, 100, 32, 20)                              # S = 41: still two warps
    try:
        lps = [torch.as_tensor(u.lp.numpy()).cuda() for u in utts] + [torch.as_tensor(one.lp.numpy()).cuda()]
        tgs = [u.targets for u in utts] + [one.targets]
        rs = st.submit_batch([(lps[i], tgs[i], 0, outs(lps[i].shape[0])) for i in range(len(lps))])
        st.flush()
        for r in rs:
            st.poll(r)
        assert st.stats()["persistent_batches"] == 1
        assert all(r.status == align.ALIGN_E_TIMEOUT for r in rs), [r.status for r in rs]
    finally:
        st.close()
    ok = align.Aligner(device=0, batched=True, persistent=True)
    try:
        run_batch(ok, [(u.lp.numpy(), u.targets) for u in utts] + [(one.lp.numpy(), one.targets)], "after")
        assert ok.stats()["persistent_batches"] == 1
    finally:
        ok.close()
