"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The recursion is one FP32 add after an exact max per cell, so paths, states,
per-frame scores and totals must match the FP32 oracle bit for bit (tolerance
zero), for every launch shape (warp, CTA, cluster), mode (full backpointers,
checkpointed recompute, plain, batched, host I/O) and input class.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import checks
from paper_2310_17864_gb300 import align, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def al():
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=8 << 30)
    yield a
    a.close()


def compare(res, lp_np, targets, blank, label=""):
    o = oracle.viterbi_f32(lp_np, targets, blank)
    assert res.status == o["status"], (label, res.status, o["status"])
    if o["status"] not in (0,):
        return o
    path = res.path.cpu().numpy()
    scores = res.scores.cpu().numpy()
    total = res.total.cpu().numpy()[0]
    assert np.array_equal(path, o["path"]), (label, np.nonzero(path != o["path"])[0][:10])
    if res.states is not None:
        assert np.array_equal(res.states.cpu().numpy(), o["states"]), label
    assert scores.tobytes() == o["scores"].tobytes(), label
    assert np.float32(total).tobytes() == np.float32(o["total"]).tobytes(), (label, total, o["total"])
    return o


def run(al, lp, targets, blank=0, label=""):
    lp_t = torch.as_tensor(np.ascontiguousarray(lp, dtype=np.float32))
    res = al.align(lp_t.cuda(), targets, blank, want_states=True)
    return compare(res, lp_t.numpy(), np.asarray(targets, np.int32), blank, label)


def test_config1_plain_utterance(al):
    (s,) = synth.specs(1)
    u = synth.make_utterance(s.seed, s.T, s.C, s.L, s.repeat_frac)
    run(al, u.lp.numpy(), u.targets, 0, "cfg1")


@pytest.mark.parametrize("T,C,L", [
    (1, 2, 0), (1, 4, 1), (2, 2, 1), (3, 3, 2), (7, 5, 3), (50, 2, 1), (64, 32, 0),
    (300, 32, 63), (300, 32, 64), (300, 32, 31), (300, 32, 32),          # warp boundary (K=4: 128 states)
    (900, 32, 127), (900, 32, 128), (900, 32, 255), (900, 32, 256),      # 1-2 / 2-3 warps
    (3000, 32, 1023), (3000, 32, 1024), (9000, 32, 2047), (9000, 32, 2048),  # 16..32 warps, cluster edge
    (5000, 500, 900), (400, 29, 90), (400, 31, 90), (333, 3, 100),
])
def test_shapes(al, T, C, L):
    u = synth.make_utterance(T * 31 + L, T, C, L, repeat_frac=0.1)
    run(al, u.lp.numpy(), u.targets, 0, f"T{T}C{C}L{L}")


def test_tight_and_repeats(al):
    rng = np.random.default_rng(5)
    for L in (1, 5, 40, 200, 700):
        tg = synth.make_targets(rng, L, 8, repeat_frac=0.5)
        T = L + synth.count_repeats(tg)                    # exactly one feasible path
        lp = rng.standard_normal((T, 8)).astype(np.float32)
        run(al, lp, tg, 0, f"tight{L}")
        allrep = np.full(L, 3, np.int32)                   # all-repeat targets
        lp = rng.standard_normal((2 * L - 1 + 5, 8)).astype(np.float32)
        run(al, lp, allrep, 0, f"allrep{L}")


def test_integer_ties_tie_rule(al):
    """Integer emissions: many exact ties; the tie rule decides the path."""
    rng = np.random.default_rng(6)
    for (T, C, L) in [(10, 3, 3), (100, 4, 30), (700, 5, 200), (2000, 4, 600), (6000, 4, 2100)]:
        tg = synth.make_targets(rng, L, C, repeat_frac=0.2)
        lp = -rng.integers(0, 3, size=(T, C)).astype(np.float32)
        run(al, lp, tg, 0, f"ties{T}")
        run(al, np.zeros((T, C), np.float32), tg, 0, f"zeros{T}")


def test_minus_inf_and_nopath(al):
    rng = np.random.default_rng(7)
    u = synth.make_utterance(77, 400, 16, 100)
    lp = u.lp.numpy().copy()
    lp[rng.random(lp.shape) < 0.3] = -np.inf
    ext = synth.expand_tokens(u.targets)
    lp[np.arange(400), ext[u.planted]] = -0.5    # keep the planted path finite
    run(al, lp, u.targets, 0, "neginf")
    lp2 = u.lp.numpy().copy()
    lp2[:, u.targets[3]] = -np.inf                # a target that can never be emitted
    run(al, lp2, u.targets, 0, "nopath")


def test_nonzero_blank(al):
    rng = np.random.default_rng(8)
    C, blank = 40, 39
    tg = rng.integers(0, 39, size=120).astype(np.int32)
    lp = torch.log_softmax(torch.randn(700, C) * 3, -1).numpy()
    run(al, lp, tg, blank, "blank39")


def test_validation_errors(al):
    lp = torch.zeros(5, 4, device="cuda")
    for tg, blank, code in [([1, 4], 0, align.ALIGN_E_TARGET), ([0], 0, align.ALIGN_E_TARGET),
                            ([1], 4, align.ALIGN_E_INVAL), ([1, 1, 1, 1], 0, align.ALIGN_E_INFEASIBLE)]:
        with pytest.raises(align.AlignError) as e:
            al.submit(lp, tg, blank)
        assert e.value.code == code


def test_debug_checks_reject_nan_and_plus_inf():
    """ALIGN_F_DEBUG_CHECKS: NaN or +inf anywhere in the emissions (device or
    host inputs, log-probabilities or logits) fails the submit with
    ALIGN_E_NONFINITE; -inf (log 0) still aligns, as the oracle does."""
    build.build()
    a = align.Aligner(device=0, debug_checks=True, bp_budget_bytes=1 << 30)
    try:
        u = synth.make_utterance(77, 300, 32, 60)
        for bad in (float("nan"), float("inf")):
            lp = u.lp.clone()
            lp[123, 7] = bad
            for where in ("cuda", "cpu"):
                with pytest.raises(align.AlignError) as e:
                    if where == "cuda":
                        a.submit(lp.cuda(), u.targets, 0)
                    else:
                        a.submit_host(lp.pin_memory(), u.targets, 0)
                assert e.value.code == align.ALIGN_E_NONFINITE, (bad, where)
            with pytest.raises(align.AlignError) as e:
                a.submit(lp.cuda(), u.targets, 0, logits=True)
            assert e.value.code == align.ALIGN_E_NONFINITE
        lp = u.lp.clone()
        lp[200:210, 5] = float("-inf")
        run(a, lp.numpy(), u.targets, 0, "debug -inf")
        run(a, u.lp.numpy(), u.targets, 0, "debug clean")
    finally:
        a.close()


@pytest.mark.parametrize("K,cw", [(2, 1), (2, 2), (2, 8), (2, 16), (4, 1), (4, 16), (8, 4), (16, 2)])
def test_launch_shapes_bit_identical(K, cw):
    """Every (states per lane, warps per CTA) shape, including one-warp CTAs in
    clusters and 8- / 16-warp CTAs (receive blocks of 16 / 8 frames), gives the
    oracle's alignment; wide rows (C = 500) stage 4 frames per chunk."""
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=8 << 30)
    try:
        a.set_tuning(K, cw, 16)
        for (T, C, L, seed) in [(700, 32, 300, 11), (333, 500, 120, 12), (95, 29, 40, 13), (33, 32, 5, 14),
                                (1200, 32, 500, 15), (700, 500, 300, 16)]:
            u = synth.make_utterance(seed * 1000 + K * 10 + cw, T, C, L, repeat_frac=0.1)
            run(a, u.lp.numpy(), u.targets, 0, f"K{K}cw{cw}T{T}C{C}")
    finally:
        a.close()


@pytest.mark.parametrize("K", [2, 4, 8, 16])
def test_nan_emissions_follow_the_definition(K):
    """NaN log-probs: every comparison with NaN is false, as in the oracle's
    strict '>' tests, so paths and states match it exactly for every lane
    width (the skip rule never turns a NaN into a winning value)."""
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=8 << 30)
    try:
        a.set_tuning(K, 4, 16)
        u = synth.make_utterance(777 + K, 300, 32, 60, repeat_frac=0.1)
        lp = u.lp.numpy().copy()
        rng = np.random.default_rng(5 + K)
        lp[rng.random(lp.shape) < 0.01] = np.nan
        res = a.align(torch.as_tensor(lp).cuda(), u.targets, 0, want_states=True)
        o = oracle.viterbi_f32(lp, np.asarray(u.targets, np.int32), 0)
        assert res.status == o["status"]
        if o["status"] != 0:  # -inf final score: no path to compare
            return
        assert np.array_equal(res.states.cpu().numpy(), o["states"])
        assert np.array_equal(res.path.cpu().numpy(), o["path"])
        t = float(res.total.cpu().numpy()[0])
        assert (np.isnan(t) and np.isnan(o["total"])) or np.float32(t).tobytes() == np.float32(o["total"]).tobytes()
    finally:
        a.close()


def test_checkpointed_equals_full():
    build.build()
    ck = align.Aligner(device=0, force_checkpoint=True)
    full = align.Aligner(device=0)
    try:
        for (T, C, L, seed) in [(1, 4, 1, 1), (2, 4, 1, 2), (17, 5, 4, 3), (400, 32, 100, 4), (401, 32, 100, 5),
                                (2500, 32, 600, 6), (9000, 32, 2100, 7)]:
            u = synth.make_utterance(seed, T, C, L, repeat_frac=0.1)
            a = ck.align(u.lp.cuda(), u.targets, 0, want_states=True)
            b = full.align(u.lp.cuda(), u.targets, 0, want_states=True)
            assert a.status == b.status == 0
            for x, y in [(a.path, b.path), (a.states, b.states), (a.scores, b.scores), (a.total, b.total)]:
                assert torch.equal(x.cpu().view(torch.int32), y.cpu().view(torch.int32))
            compare(a, u.lp.numpy(), u.targets, 0, f"ck{T}")
        assert ck.stats()["checkpointed"] >= 7
    finally:
        ck.close()
        full.close()


def test_budget_forces_checkpoint():
    """A request whose full backpointers exceed the budget runs checkpointed."""
    build.build()
    u = synth.make_utterance(9, 6000, 32, 1500)
    p = align.align_plan(6000, 32, 1500)
    a = align.Aligner(device=0, bp_budget_bytes=p["backpointer_bytes"] // 2)
    try:
        res = a.align(u.lp.cuda(), u.targets, 0)
        compare(res, u.lp.numpy(), u.targets, 0, "budget")
        assert a.stats()["checkpointed"] == 1
    finally:
        a.close()


def test_host_io(al):
    u = synth.make_utterance(10, 1500, 32, 375)
    lp = u.lp.pin_memory()
    res = al.submit_host(lp, u.targets, 0, want_states=True)
    al.flush()
    al.poll(res)
    compare(res, u.lp.numpy(), u.targets, 0, "host")


@pytest.mark.parametrize("pinned", [True, False])
def test_host_batch_copies(pinned):
    """Host-buffer requests of a batch (pinned, or pageable where the device
    reads host page tables; otherwise per-buffer copies) move in and out with
    batched copy kernels, including buffers larger than one copy chunk and
    unaligned row sizes; results equal the oracle."""
    build.build()
    shapes = [(300, 32, 70, 1), (9000, 32, 2000, 2), (257, 29, 60, 3), (40, 5, 9, 4), (2100, 500, 500, 5)]
    us = [synth.make_utterance(s, T, C, L, repeat_frac=0.1) for (T, C, L, s) in shapes]
    al = align.Aligner(device=0, batched=True, bp_budget_bytes=4 << 30)
    try:
        items, outs = [], []
        for u in us:
            T = u.lp.shape[0]
            lp = u.lp.pin_memory() if pinned else u.lp.clone()
            o = tuple(torch.empty(n, dtype=dt, pin_memory=pinned) for n, dt in
                      ((T, torch.int32), (T, torch.float32), (1, torch.float32), (T, torch.int32)))
            outs.append(o)
            items.append((lp, u.targets, 0, o))
        rs = al.submit_batch(items, host=True)
        al.flush()
        for r in rs:
            al.poll(r)
        for u, o, r in zip(us, outs, rs):
            ref = oracle.viterbi_f32(u.lp.numpy(), np.asarray(u.targets, np.int32), 0)
            assert r.status == ref["status"] == 0
            assert np.array_equal(o[0].numpy(), ref["path"]) and np.array_equal(o[3].numpy(), ref["states"])
            assert o[1].numpy().tobytes() == ref["scores"].tobytes()
            assert np.float32(o[2].numpy()[0]).tobytes() == np.float32(ref["total"]).tobytes()
    finally:
        al.close()


def test_config2_batched_equals_plain_and_oracle():
    build.build()
    b = synth.make_batch(synth.specs(2), device="cuda")
    plain = align.Aligner(device=0)
    batched = align.Aligner(device=0, batched=True)
    try:
        rp = [plain.submit(b.utt(i), b.targets[i], 0) for i in range(len(b))]
        rb = [batched.submit(b.utt(i), b.targets[i], 0) for i in range(len(b))]
        batched.flush()
        for x, y in zip(rp, rb):
            plain.poll(x)
            batched.poll(y)
        lp_host = b.lp.cpu().numpy()
        for i, (x, y) in enumerate(zip(rp, rb)):
            assert torch.equal(x.path, y.path) and torch.equal(x.scores.view(torch.int32), y.scores.view(torch.int32))
            sl = lp_host[b.offsets[i]:b.offsets[i + 1]]
            compare(y, sl, b.targets[i], 0, f"cfg2[{i}]")
    finally:
        plain.close()
        batched.close()


def test_cluster_long_transcript(al):
    """S beyond one CTA: the alpha vector spread over a thread-block cluster."""
    for (T, L) in [(12000, 3000), (40000, 17000)]:
        u = synth.make_utterance(T + L, T, 32, L)
        p = align.align_plan(T, 32, L, budget=8 << 30)
        assert p["cluster_ctas"] > 1
        run(al, u.lp.numpy(), u.targets, 0, f"cluster{L}")


def test_invariants_on_config4_sample():
    """Ragged batch (first 512 utterances of the C=32 workload) batched; every
    result satisfies the invariants and a sample matches the oracle."""
    build.build()
    specs = synth.specs(4, C=32, n=512)
    b = synth.make_batch(specs, device="cuda")
    a = align.Aligner(device=0, batched=True, bp_budget_bytes=8 << 30)
    try:
        rs = [a.submit(b.utt(i), b.targets[i], 0) for i in range(len(b))]
        a.flush()
        lp_host = b.lp.cpu().numpy()
        for i, r in enumerate(rs):
            a.poll(r)
            assert r.status == 0
            path = r.path.cpu().numpy()
            assert checks.collapse(path, 0) == b.targets[i].tolist()
            sl = lp_host[b.offsets[i]:b.offsets[i + 1]]
            assert (r.scores.cpu().numpy() == sl[np.arange(sl.shape[0]), path]).all()
            assert checks.fold_f32_fast(r.scores.cpu().numpy()) == r.total.cpu().numpy()[0]
            if i % 16 == 0:
                compare(r, sl, b.targets[i], 0, f"cfg4[{i}]")
    finally:
        a.close()


def test_submit_batch_equals_single_and_host_batch():
    build.build()
    specs = synth.specs(2)[:24]
    b = synth.make_batch(specs, device="cuda")
    a = align.Aligner(device=0)
    try:
        outs = [(torch.empty(s.T, dtype=torch.int32, device="cuda"), torch.empty(s.T, device="cuda"),
                 torch.empty(1, device="cuda"), torch.empty(s.T, dtype=torch.int32, device="cuda")) for s in specs]
        rb = a.submit_batch([(b.utt(i), b.targets[i], 0, outs[i]) for i in range(len(b))])
        for r in rb:
            a.poll(r)
        lp_host = b.lp.cpu()
        hout = [(torch.empty(s.T, dtype=torch.int32).pin_memory(), torch.empty(s.T).pin_memory(),
                 torch.empty(1).pin_memory(), torch.empty(s.T, dtype=torch.int32).pin_memory()) for s in specs]
        hl = [lp_host[b.offsets[i]:b.offsets[i + 1]].contiguous().pin_memory() for i in range(len(b))]
        rh = a.submit_batch([(hl[i], b.targets[i], 0, hout[i]) for i in range(len(b))], host=True)
        for r in rh:
            a.poll(r)
        for i in range(len(b)):
            compare(rb[i], lp_host[b.offsets[i]:b.offsets[i + 1]].numpy(), b.targets[i], 0, f"batch[{i}]")
            assert torch.equal(rb[i].path.cpu(), rh[i].path) and torch.equal(rb[i].states.cpu(), rh[i].states)
            assert rb[i].scores.cpu().numpy().tobytes() == rh[i].scores.numpy().tobytes()
        # A rejected request in a batch does not stop the others.
        bad = [(b.utt(0), b.targets[0], 0, outs[0]), (b.utt(1), np.array([0], np.int32), 0, outs[1])]
        with pytest.raises(align.AlignError):
            a.submit_batch(bad)
    finally:
        a.close()


def test_watchdog_timeout_keeps_context_usable():
    """A device-side wait that never completes ends with ALIGN_E_TIMEOUT after
    the configured limit; nothing faults and later work runs normally."""
    build.build()
    u = synth.make_utterance(3, 400, 32, 150)   # S = 301: several warps
    v = synth.make_utterance(4, 100, 32, 20)    # S = 41: a single warp
    st = align.Aligner(device=0, wait_limit_ms=50, test_stall=True)
    try:
        r = st.align(u.lp.cuda(), u.targets, 0)
        assert r.status == align.ALIGN_E_TIMEOUT
        r1 = st.align(v.lp.cuda(), v.targets, 0)   # one warp: no hand-off, unaffected
        compare(r1, v.lp.numpy(), v.targets, 0, "single-warp under stall flag")
    finally:
        st.close()
    ok = align.Aligner(device=0)
    try:
        r = ok.align(u.lp.cuda(), u.targets, 0)
        compare(r, u.lp.numpy(), u.targets, 0, "after timeout")
    finally:
        ok.close()


def test_grid_team_equals_cluster_and_checkpointed():
    """A transcript beyond one cluster of the default shape (S = 34,001) runs
    as a grid team (one 16-warp CTA per SM, links in global memory); the
    result is bit-identical to the cluster plan with more states per lane and
    to checkpointed recompute on the grid team."""
    build.build()
    T, L = 36000, 17000
    u = synth.make_utterance(31, T, 32, L)
    lp = u.lp.cuda()
    outs = {}
    for name, kw in [("grid", {}), ("cluster", {"grid_teams": False}), ("grid_ck", {"force_checkpoint": True})]:
        a = align.Aligner(device=0, bp_budget_bytes=8 << 30, **kw)
        try:
            r = a.align(lp, u.targets, 0, want_states=True)
            assert r.status == 0, (name, r.status)
            outs[name] = [x.cpu().view(torch.int32) for x in (r.path, r.states, r.scores, r.total)]
        finally:
            a.close()
    for name in ("cluster", "grid_ck"):
        for x, y in zip(outs["grid"], outs[name]):
            assert torch.equal(x, y), name
    # The oracle's frame states at sampled frames, from the forward/backward max-plus sums.
    o = oracle.viterbi_f32(u.lp.numpy(), np.asarray(u.targets, np.int32), 0)
    assert np.array_equal(outs["grid"][1].numpy(), o["states"])


def test_two_grid_teams_and_small_requests_in_one_batch():
    """Grid teams of one batch run one after the other on the context's grid
    stream (each needs its SMs at once) while small requests run beside them;
    every result equals the request aligned alone."""
    build.build()
    us = [synth.make_utterance(41, 36000, 32, 17000), synth.make_utterance(42, 34000, 32, 16500),
          synth.make_utterance(43, 500, 32, 120), synth.make_utterance(44, 800, 32, 200)]
    al = align.Aligner(device=0, batched=True, bp_budget_bytes=12 << 30)
    one = align.Aligner(device=0, bp_budget_bytes=8 << 30)
    try:
        items, outs = [], []
        for u in us:
            T = u.lp.shape[0]
            o = (torch.empty(T, dtype=torch.int32, device="cuda:0"), torch.empty(T, device="cuda:0"),
                 torch.empty(1, device="cuda:0"), None)
            outs.append(o)
            items.append((u.lp.cuda(), u.targets, 0, o))
        rs = al.submit_batch(items)
        al.flush()
        for r in rs:
            al.poll(r)
            assert r.status == 0
        for u, o in zip(us, outs):
            ref = one.align(u.lp.cuda(), u.targets, 0)
            assert torch.equal(o[0], ref.path) and torch.equal(o[1].view(torch.int32), ref.scores.view(torch.int32))
    finally:
        al.close()
        one.close()


def test_host_batch_large_moves_per_launch():
    """A host batch above 64 MB moves each launch's buffers on its own stream
    (copies overlapping other launches); results equal the device path."""
    build.build()
    specs = [synth.Spec(4000 + 37 * i, 300, 700 + 11 * i, 0.1, synth.sub_seed(777, i)) for i in range(16)]
    b = synth.make_batch(specs, device="cpu")
    assert b.lp.numel() * 4 > (64 << 20)
    n = len(b)
    tg = np.concatenate([np.asarray(t, np.int32) for t in b.targets])
    tg_off = np.concatenate([[0], np.cumsum([len(t) for t in b.targets])])
    TT = int(b.offsets[-1])
    out = (torch.empty(TT, dtype=torch.int32).pin_memory(), torch.empty(TT, dtype=torch.float32).pin_memory(),
           torch.empty(n, dtype=torch.float32).pin_memory(), None)
    al = align.Aligner(device=0, batched=True, bp_budget_bytes=4 << 30, staging_bytes=512 << 20)
    one = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        pr = al.submit_packed(b.lp.pin_memory(), b.offsets, tg, tg_off, out, host=True)
        al.flush()
        al.wait_packed(pr)
        assert (pr.status == 0).all()
        for i in range(n):
            f0, f1 = int(b.offsets[i]), int(b.offsets[i + 1])
            r = one.align(b.utt(i).cuda(), b.targets[i], 0)
            assert torch.equal(out[0][f0:f1], r.path.cpu())
            assert torch.equal(out[1][f0:f1].view(torch.int32), r.scores.cpu().view(torch.int32))
    finally:
        al.close()
        one.close()


@pytest.mark.parametrize("host", [False, True])
def test_submit_packed_equals_single_requests(host):
    """A packed ragged batch (one emission tensor, packed targets and outputs)
    gives the same results as submitting its utterances one by one."""
    build.build()
    specs = synth.specs(4, C=32, n=40)
    b = synth.make_batch(specs, device="cpu" if host else "cuda")
    n = len(b)
    tg = np.concatenate([np.asarray(t, np.int32) for t in b.targets])
    tg_off = np.concatenate([[0], np.cumsum([len(t) for t in b.targets])])
    TT = int(b.offsets[-1])
    kw = {"pin_memory": True} if host else {"device": "cuda"}
    out = (torch.empty(TT, dtype=torch.int32, **kw), torch.empty(TT, dtype=torch.float32, **kw),
           torch.empty(n, dtype=torch.float32, **kw), torch.empty(TT, dtype=torch.int32, **kw))
    lp = b.lp.pin_memory() if host else b.lp
    al = align.Aligner(device=0, batched=True, bp_budget_bytes=4 << 30)
    one = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        pr = al.submit_packed(lp, b.offsets, tg, tg_off, out, host=host)
        al.flush()
        al.wait_packed(pr)
        assert (pr.status == 0).all()
        for i in range(n):
            f0, f1 = int(b.offsets[i]), int(b.offsets[i + 1])
            r = one.align(b.utt(i).cuda(), b.targets[i], 0, want_states=True)
            assert torch.equal(out[0][f0:f1].cpu(), r.path.cpu())
            assert torch.equal(out[3][f0:f1].cpu(), r.states.cpu())
            assert torch.equal(out[1][f0:f1].cpu().view(torch.int32), r.scores.cpu().view(torch.int32))
            assert out[2][i].cpu().view(torch.int32).item() == r.total.cpu().view(torch.int32).item()
    finally:
        al.close()
        one.close()


def test_grid_team_watchdog():
    """The bounded waits of a grid team (ring, progress, team barrier) end a
    stalled request with ALIGN_E_TIMEOUT; the context stays usable."""
    build.build()
    u = synth.make_utterance(32, 36000, 32, 17000)
    st = align.Aligner(device=0, bp_budget_bytes=8 << 30, wait_limit_ms=100, test_stall=True)
    try:
        r = st.align(u.lp.cuda(), u.targets, 0)
        assert r.status == align.ALIGN_E_TIMEOUT
    finally:
        st.close()
    v = synth.make_utterance(4, 100, 32, 20)
    ok = align.Aligner(device=0)
    try:
        compare(ok.align(v.lp.cuda(), v.targets, 0), v.lp.numpy(), v.targets, 0, "after grid timeout")
    finally:
        ok.close()


def test_graph_replay_equals_direct_launch():
    """A batch with the same launch structure (descriptors uploaded to the
    device) is captured once and replayed; results equal direct launches of
    a batch whose kernels read the pinned descriptor image, bit for bit."""
    build.build()
    specs = synth.specs(2)[:20]
    b = synth.make_batch(specs, device="cuda")
    outs = lambda: [(torch.empty(s.T, dtype=torch.int32, device="cuda"), torch.empty(s.T, device="cuda"),
                     torch.empty(1, device="cuda"), torch.empty(s.T, dtype=torch.int32, device="cuda")) for s in specs]
    g = align.Aligner(device=0, batched=True, upload_descriptors=True)
    d = align.Aligner(device=0, batched=True, graphs=False)
    try:
        ref = d.submit_batch([(b.utt(i), b.targets[i], 0, o) for i, o in enumerate(outs())])
        d.flush()
        for r in ref:
            d.poll(r)
        for _ in range(3):
            rs = g.submit_batch([(b.utt(i), b.targets[i], 0, o) for i, o in enumerate(outs())])
            g.flush()
            for r, x in zip(rs, ref):
                g.poll(r)
                assert r.status == x.status == 0
                assert torch.equal(r.path, x.path) and torch.equal(r.states, x.states)
                assert r.scores.cpu().numpy().tobytes() == x.scores.cpu().numpy().tobytes()
        assert g.stats()["graph_launches"] == 2  # captured on the second batch, replayed on the third
        assert d.stats()["graph_launches"] == 0
    finally:
        g.close()
        d.close()


@pytest.mark.parametrize("K,cw", [(2, 2), (4, 1)])
def test_every_last_window_length(K, cw):
    """Frames in the last 32-frame window from 0 to 32 (so the last block of
    hand-off packages is full, partial, or a single frame), for a team of
    warps in one CTA and a cluster of one-warp CTAs."""
    build.build()
    a = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        a.set_tuning(K, cw, 16)
        for r in range(33):
            T = 32 * 5 + 1 + r                 # T - 1 frames after the first: 5 windows + r
            u = synth.make_utterance(1000 + 37 * r + K, T, 32, 70, repeat_frac=0.1)
            run(a, u.lp.numpy(), u.targets, 0, f"K{K}cw{cw}r{r}")
    finally:
        a.close()
