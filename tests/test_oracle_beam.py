"""Pins of the CTC prefix beam search oracle (oracle/beam.py).

What fixes the oracle independently of itself: hand-worked dyadic cases
(tests/golden/beam_hand.json), brute-force enumeration of every frame path on
tiny inputs (the beam, when nothing is pruned, holds every label sequence with
its total probability), the sum-product forward score of the trellis oracle
(pinned on its own), probability mass conservation, one-hot inputs whose
answer is the collapse of the planted path, and the pruning bound.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import beam

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "beam_hand.json")


def collapse(path, blank):
    out = []
    prev = None
    for p in path:
        if p != blank and p != prev:
            out.append(p)
        prev = p
    return tuple(out)


def brute(P, blank):
    """Probability of every label sequence: sum over all frame paths (binary64)."""
    T, V = P.shape
    probs = {}
    for path in itertools.product(range(V), repeat=T):
        pr = 1.0
        for t, c in enumerate(path):
            pr *= float(P[t, c])
        key = collapse(path, blank)
        probs[key] = probs.get(key, 0.0) + pr
    return probs


def rows(rng, T, V, peak=0.0):
    x = rng.standard_normal((T, V)) * 1.5
    x[np.arange(T), rng.integers(0, V, T)] += peak
    e = np.exp(x - x.max(axis=1, keepdims=True))
    return (e / e.sum(axis=1, keepdims=True)).astype(np.float32)


def test_hand_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        P = np.asarray(c["P"], np.float32)
        r = beam.beam_search(P, c["blank"], c["beam"], c["a"])
        assert r["kept"].tolist() == c["kept"], c["name"]
        assert r["exp"] == c["exp"], (c["name"], r["exp"])
        assert len(r["hyps"]) == len(c["hyps"]), c["name"]
        for got, want in zip(r["hyps"], c["hyps"]):
            prefix, times, total, pb, pnb = got
            assert list(prefix) == want["prefix"] and list(times) == want["times"], c["name"]
            assert (float(total), float(pb), float(pnb)) == (want["total"], want["pb"], want["pnb"]), (c["name"], got)


def test_blank_collapse_runs():
    P = np.zeros((8, 3), np.float32)
    P[:, 0] = np.array([0.99, 0.97, 0.5, 0.96, 0.96, 0.96, 0.2, np.float32(0.95)], np.float32)
    P[:, 1] = 1 - P[:, 0]
    assert beam.blank_collapse(P, 0, 0.95).tolist() == [0, 2, 3, 6, 7]   # 0.95 is not above 0.95
    assert beam.blank_collapse(P, 0, 1.0).tolist() == list(range(8))
    assert beam.blank_collapse(P, 0, 0.0).tolist() == [0]                 # one run of blank frames
    assert beam.blank_collapse(P, 1, 0.95).tolist() == list(range(8))     # the blank index decides


@pytest.mark.parametrize("T,V,blank,seed", [(1, 3, 0, 1), (3, 3, 0, 2), (4, 3, 2, 3), (5, 3, 1, 4), (3, 4, 0, 5),
                                             (4, 4, 3, 6)])
def test_unpruned_beam_is_every_sequence(T, V, blank, seed):
    """A beam wider than the number of prefixes prunes nothing: it holds
    every label sequence with the summed probability of its frame paths, in
    descending order, and the probabilities add up to one."""
    rng = np.random.default_rng(seed)
    P = rows(rng, T, V)
    ref = brute(P, blank)
    B = sum((V - 1) ** k for k in range(T + 1))
    r = beam.beam_search(P, blank, B, 1.0)
    got = {h[0]: float(h[2]) * 2.0 ** r["exp"] for h in r["hyps"] if h[2] > 0}
    assert set(got) == set(ref)
    # the rest of the beam are prefixes no frame path yields (a repeat with no blank room)
    assert all(h[0] not in ref for h in r["hyps"] if h[2] == 0)
    for k, v in ref.items():
        assert abs(got[k] - v) <= 1e-5 * v + 1e-30, (k, got[k], v)
    tot = [float(h[2]) for h in r["hyps"]]
    assert tot == sorted(tot, reverse=True)
    assert abs(sum(got.values()) - 1.0) < 1e-5


def test_hypotheses_match_forward_score():
    """Unpruned, each hypothesis' probability is the CTC forward probability
    of its labels (the sum-product oracle, pinned on its own)."""
    rng = np.random.default_rng(11)
    T, V = 6, 4
    P = rows(rng, T, V, peak=2.0)
    B = sum((V - 1) ** k for k in range(T + 1))
    r = beam.beam_search(P, 0, B, 1.0)
    lp = np.log(P.astype(np.float64))
    for prefix, _, total, _, _ in r["hyps"][:12]:
        f = oracle.ctc_forward_f64(lp, np.asarray(prefix, np.int32), 0)
        assert f["status"] == 0
        assert abs(beam.log_score(total, r["exp"]) - f["total"]) < 1e-5, prefix


def test_pruning_only_loses_paths():
    """With a narrow beam every hypothesis keeps at most its forward
    probability, prefixes are distinct and totals descend; the best of a
    wide beam is at least the best of a narrow one."""
    rng = np.random.default_rng(12)
    for trial in range(6):
        T, V = 14, 5
        P = rows(rng, T, V, peak=1.0)
        lp = np.log(P.astype(np.float64))
        best = []
        for B in (2, 4, 16):
            r = beam.beam_search(P, 0, B, 1.0)
            prefixes = [h[0] for h in r["hyps"]]
            assert len(set(prefixes)) == len(prefixes) == B
            tot = [float(h[2]) for h in r["hyps"]]
            assert tot == sorted(tot, reverse=True)
            for prefix, _, total, _, _ in r["hyps"]:
                f = oracle.ctc_forward_f64(lp, np.asarray(prefix, np.int32), 0)
                assert beam.log_score(total, r["exp"]) <= f["total"] + 1e-5
            best.append(beam.log_score(r["hyps"][0][2], r["exp"]))
        assert best[2] >= best[0] - 1e-6


def test_one_hot_planted_path():
    """One-hot frames: the only sequence with probability is the collapse of
    the planted path; its label times are the first frames of its label runs
    (kept by the collapse), with and without blank collapse."""
    path = [0, 0, 0, 3, 3, 0, 3, 1, 1, 0, 0, 0, 0, 2, 0, 2, 2, 0, 0]
    V = 4
    P = np.zeros((len(path), V), np.float32)
    P[np.arange(len(path)), path] = 1.0
    want = collapse(path, 0)
    starts = [t for t in range(len(path)) if path[t] != 0 and (t == 0 or path[t - 1] != path[t])]
    for a in (1.0, 0.95):
        r = beam.beam_search(P, 0, 3, a)
        prefix, times, total, _, _ = r["hyps"][0]
        assert prefix == want and list(times) == starts
        assert float(total) * 2.0 ** r["exp"] == 1.0
        assert all(float(h[2]) == 0.0 for h in r["hyps"][1:])
    assert beam.blank_collapse(P, 0, 0.95).tolist() == [0, 3, 4, 5, 6, 7, 8, 9, 13, 14, 15, 16, 17]


def test_log_score():
    assert beam.log_score(np.float32(0.5), 3) == pytest.approx(math.log(4.0))
    assert beam.log_score(np.float32(0.0), 3) == -math.inf
