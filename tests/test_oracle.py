"""Pins of the CPU oracle against facts fixed by the definition and by mathematics.

The paper (TorchAudio 2.1, Sec. 4, "CTC-based forced alignment") prints no
worked example or alignment number, so each pin is one of: hand-derived tiny
cases, exhaustive enumeration, closed forms, invariants, the FP32 summation
error bound against a binary64 run, and an independent max-plus backward pass.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute, checks
from paper_2310_17864_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_case(rng, T, L, C, kind="float"):
    blank = int(rng.integers(0, C))
    labels = [c for c in range(C) if c != blank]
    targets = rng.choice(labels, size=L).astype(np.int32) if L else np.zeros(0, np.int32)
    if kind == "float":
        lp = rng.standard_normal((T, C)).astype(np.float32)
    elif kind == "int":
        lp = -rng.integers(0, 4, size=(T, C)).astype(np.float32)
    else:
        raise ValueError(kind)
    return lp, targets, blank


# ------------------------------------------------------------ golden cases --

def test_hand_examples():
    with open(os.path.join(HERE, "golden", "hand_examples.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        lp = np.asarray(c["lp"], np.float32)
        r = oracle.viterbi_f32(lp, np.asarray(c["targets"], np.int32), c["blank"])
        assert r["status"] == c["status"], c["name"]
        if c["status"] == 0:
            assert r["states"].tolist() == c["states"], c["name"]
            assert r["path"].tolist() == c["path"], c["name"]
            assert r["scores"].tolist() == c["scores"], c["name"]
            assert r["total"] == np.float32(c["total"]), c["name"]


# ------------------------------------------------------------- brute force --

def test_brute_force_random_floats():
    """Total equals the best FP32 left-fold path sum bit for bit; with a unique
    optimum the path is that optimum."""
    rng = np.random.default_rng(1)
    checked_unique = 0
    for _ in range(400):
        C = int(rng.integers(2, 5))
        L = int(rng.integers(0, 4))
        T = int(rng.integers(1, 8))
        lp, tg, blank = _rand_case(rng, T, L, C)
        rc, R = oracle.validate(tg, C, blank, T)
        r = oracle.viterbi_f32(lp, tg, blank)
        b = brute.brute_force(lp, tg, blank)
        if T < L + R:
            assert rc == oracle.E_INFEASIBLE and r["status"] == oracle.E_INFEASIBLE
            assert b["n_paths"] == 0
            continue
        assert b["n_paths"] > 0
        assert r["status"] == 0
        assert r["total"].tobytes() == np.float32(b["best"]).tobytes()
        if len(b["optimal"]) == 1:
            checked_unique += 1
            assert tuple(r["states"].tolist()) == b["optimal"][0]
    assert checked_unique > 200


def test_brute_force_integer_ties_pin_tie_rule():
    """Integer emissions make every sum exact and ties common. The oracle must
    return the optimal state path that is greatest read backwards from the last
    frame (stay > advance > skip inside the recursion, trailing blank on a final tie)."""
    rng = np.random.default_rng(2)
    multi = 0
    for _ in range(600):
        C = int(rng.integers(2, 5))
        L = int(rng.integers(0, 4))
        T = int(rng.integers(1, 9))
        lp, tg, blank = _rand_case(rng, T, L, C, kind="int")
        r = oracle.viterbi_f32(lp, tg, blank)
        b = brute.brute_force(lp, tg, blank)
        if b["n_paths"] == 0:
            assert r["status"] == oracle.E_INFEASIBLE
            continue
        assert r["total"] == b["best"]
        assert tuple(r["states"].tolist()) == b["chosen"]
        multi += len(b["optimal"]) > 1
    assert multi > 150


def test_brute_force_fp64_twin():
    rng = np.random.default_rng(3)
    for _ in range(200):
        C = int(rng.integers(2, 5))
        L = int(rng.integers(0, 4))
        T = int(rng.integers(1, 8))
        lp, tg, blank = _rand_case(rng, T, L, C)
        b = brute.brute_force(lp, tg, blank, dtype=np.float64)
        r = oracle.viterbi_f64(lp, tg, blank)
        if b["n_paths"] == 0:
            assert r["status"] == oracle.E_INFEASIBLE
            continue
        assert r["total"] == b["best"]


def test_brute_force_minus_inf_emissions():
    """log 0 entries: unreachable cells stay -inf, no NaN; all -inf -> no path."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        C = int(rng.integers(2, 5))
        L = int(rng.integers(0, 4))
        T = int(rng.integers(1, 7))
        lp, tg, blank = _rand_case(rng, T, L, C)
        lp[rng.random(lp.shape) < 0.4] = -np.inf
        r = oracle.viterbi_f32(lp, tg, blank)
        b = brute.brute_force(lp, tg, blank)
        if b["n_paths"] == 0:
            assert r["status"] == oracle.E_INFEASIBLE
            continue
        assert not np.isnan(r["total"])
        if b["best"] == -np.inf:
            assert r["status"] == oracle.E_NOPATH and r["total"] == -np.inf
        else:
            assert r["status"] == 0 and r["total"] == b["best"]
            if len(b["optimal"]) == 1:
                assert tuple(r["states"].tolist()) == b["optimal"][0]


# ------------------------------------------------------------ closed forms --

def test_closed_form_empty_transcript():
    rng = np.random.default_rng(5)
    lp = rng.standard_normal((57, 7)).astype(np.float32)
    r = oracle.viterbi_f32(lp, [], 3)
    assert r["status"] == 0
    assert (r["path"] == 3).all() and (r["states"] == 0).all()
    assert r["total"] == checks.fold_f32(lp[:, 3])


def test_closed_form_tight():
    """T = L + R: exactly one path, labels on consecutive frames, blanks only between repeats."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        L = int(rng.integers(1, 30))
        tg = synth.make_targets(rng, L, 6, repeat_frac=0.3)
        R = synth.count_repeats(tg)
        T = L + R
        lp = rng.standard_normal((T, 6)).astype(np.float32)
        r = oracle.viterbi_f32(lp, tg, 0)
        want = []
        for i, lab in enumerate(tg):
            if i and tg[i - 1] == lab:
                want.append(0)
            want.append(int(lab))
        assert r["path"].tolist() == want
    lp = rng.standard_normal((4, 6)).astype(np.float32)
    assert oracle.viterbi_f32(lp, [1, 1, 2, 2], 0)["status"] == oracle.E_INFEASIBLE


def test_closed_form_uniform_earliest_alignment():
    """Equal emissions everywhere: all paths tie bit for bit and the tie rule
    yields the earliest alignment (labels first, blanks to the end)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        C = 9
        L = int(rng.integers(1, 20))
        tg = synth.make_targets(rng, L, C, repeat_frac=0.3)
        R = synth.count_repeats(tg)
        T = L + R + int(rng.integers(0, 15))
        lp = np.full((T, C), -np.log(np.float32(C)), np.float32)
        r = oracle.viterbi_f32(lp, tg, 0)
        want = []
        for i, lab in enumerate(tg):
            if i and tg[i - 1] == lab:
                want.append(0)
            want.append(int(lab))
        want += [0] * (T - len(want))
        assert r["path"].tolist() == want


def test_closed_form_planted_path():
    rng = np.random.default_rng(8)
    for _ in range(20):
        C = 12
        L = int(rng.integers(1, 25))
        tg = synth.make_targets(rng, L, C, repeat_frac=0.2)
        T = L + synth.count_repeats(tg) + int(rng.integers(0, 40))
        planted = synth.plant_state_path(rng, T, tg)
        ext = synth.expand_tokens(tg)
        lp = np.full((T, C), -1e4, np.float32)
        lp[np.arange(T), ext[planted]] = 0.0
        r = oracle.viterbi_f32(lp, tg, 0)
        assert r["states"].tolist() == planted.tolist()
        assert r["total"] == 0.0


# -------------------------------------------------------------- invariants --

@pytest.mark.parametrize("cfg_like", [(200, 32, 40, 0.1), (700, 32, 175, 0.0), (300, 500, 100, 0.0)])
def test_invariants_synthetic(cfg_like):
    T, C, L, rf = cfg_like
    u = synth.make_utterance(synth.sub_seed(99, T), T, C, L, repeat_frac=rf)
    lp = u.lp.numpy()
    r = oracle.viterbi_f32(lp, u.targets, 0)
    assert r["status"] == 0
    assert checks.collapse(r["path"], 0) == u.targets.tolist()
    assert checks.legal_state_path(r["states"], u.targets, 0)
    ext = synth.expand_tokens(u.targets)
    assert (r["path"] == ext[r["states"]]).all()
    assert (r["scores"] == lp[np.arange(T), r["path"]]).all()
    assert checks.fold_f32(r["scores"]).tobytes() == np.float32(r["total"]).tobytes()
    # No randomly sampled valid path beats it (same sampler as the planted path).
    rng = np.random.default_rng(10)
    for _ in range(300):
        p = synth.plant_state_path(rng, T, u.targets)
        assert checks.legal_state_path(p, u.targets, 0)
        assert checks.fold_f32(lp[np.arange(T), ext[p]]) <= r["total"]


def test_fold_fast_matches_loop():
    rng = np.random.default_rng(11)
    v = (rng.standard_normal(5000) * 7).astype(np.float32)
    assert checks.fold_f32_fast(v).tobytes() == checks.fold_f32(v).tobytes()


def test_fp64_backward_pass_and_error_bound():
    """An independent max-plus backward pass reproduces the binary64 total; the
    forward/backward sum is the total at every frame; FP32 vs FP64 obeys the
    recursive-summation bound |d| <= gamma_{T-1} * sum|scores|."""
    for (T, C, L) in [(120, 32, 30), (257, 16, 64), (60, 500, 20)]:
        u = synth.make_utterance(synth.sub_seed(7, T), T, C, L)
        lp = u.lp.numpy()
        r32 = oracle.viterbi_f32(lp, u.targets, 0)
        r64 = oracle.viterbi_f64(lp, u.targets, 0)
        beta = checks.backward_maxplus_f64(lp, u.targets, 0)
        start = max(beta[0, 0], beta[0, 1] if beta.shape[1] > 1 else -np.inf)
        assert start == pytest.approx(r64["total"], rel=1e-12, abs=1e-12)
        alpha = checks.forward_maxplus_f64(lp, u.targets, 0)
        ext = checks.ext_array(u.targets, 0)
        through = np.max(alpha + beta - lp[:, ext].astype(np.float64), axis=1)
        np.testing.assert_allclose(through, r64["total"], rtol=1e-9)
        if (r32["states"] == r64["states"]).all():
            bound = checks.gamma(T - 1) * np.abs(r64["scores"]).sum()
            assert abs(float(r32["total"]) - r64["total"]) <= bound


def test_infeasible_and_invalid_inputs():
    lp = np.zeros((3, 4), np.float32)
    assert oracle.viterbi_f32(lp, [1, 4], 0)["status"] == oracle.E_TARGET      # out of range
    assert oracle.viterbi_f32(lp, [1, 0], 0)["status"] == oracle.E_TARGET      # blank as target
    assert oracle.viterbi_f32(lp, [-1], 0)["status"] == oracle.E_TARGET
    assert oracle.viterbi_f32(lp, [1], 4)["status"] == oracle.E_INVAL          # blank out of range
    assert oracle.viterbi_f32(np.zeros((3, 1), np.float32), [], 0)["status"] == oracle.E_INVAL  # C < 2
    assert oracle.viterbi_f32(lp, [1, 1, 1], 0)["status"] == oracle.E_INFEASIBLE  # needs 5 frames
    assert oracle.viterbi_f32(np.zeros((5, 4), np.float32), [1, 1, 1], 0)["status"] == 0
    assert oracle.viterbi_f32(np.zeros((1, 4), np.float32), [2], 0)["path"].tolist() == [2]


def test_segment_recompute_matches_dense():
    """The bounded-memory mode (alpha rows every ~sqrt(T) frames, segments
    recomputed last to first) gives identical outputs."""
    for (T, C, L) in [(1, 4, 0), (2, 4, 1), (17, 5, 4), (100, 8, 30), (401, 32, 100), (1000, 32, 250)]:
        u = synth.make_utterance(synth.sub_seed(3, T), T, C, L, repeat_frac=0.1)
        lp = u.lp.numpy()
        d = oracle.viterbi_f32(lp, u.targets, 0)
        s = oracle.viterbi_f32(lp, u.targets, 0, max_bp_bytes=1)
        for k in ("states", "path", "scores"):
            assert (d[k] == s[k]).all(), (T, k)
        assert d["total"].tobytes() == s["total"].tobytes()
        tot = oracle.viterbi_total_f32(lp, u.targets, 0)
        assert tot["total"].tobytes() == d["total"].tobytes()
        assert tot["final_state"] == d["states"][-1]
    # integer ties through the segmented walk
    rng = np.random.default_rng(12)
    for _ in range(30):
        T = int(rng.integers(1, 60))
        L = int(rng.integers(0, max(1, T // 3)))
        lp, tg, blank = _rand_case(rng, T, L, 4, kind="int")
        d = oracle.viterbi_f32(lp, tg, blank)
        s = oracle.viterbi_f32(lp, tg, blank, max_bp_bytes=1)
        assert d["status"] == s["status"]
        if d["status"] == 0:
            assert (d["states"] == s["states"]).all()
