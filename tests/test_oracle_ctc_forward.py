"""Pins of the sum-product (CTC forward score) oracle: exhaustive enumeration
of every valid state path on tiny inputs, PyTorch's CTC loss (a library
routine for the same quantity), and closed forms."""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import brute
from paper_2310_17864_gb300 import synth


def brute_sum(lp, targets, blank=0):
    lp = np.asarray(lp, np.float64)
    ext = brute.expand(targets, blank)
    paths = brute.enumerate_paths(lp.shape[0], targets, blank)
    vals = [sum(lp[t, ext[s]] for t, s in enumerate(p)) for p in paths]
    m = max(vals)
    return m + math.log(sum(math.exp(v - m) for v in vals))


@pytest.mark.parametrize("seed", range(12))
def test_equals_enumeration(seed):
    rng = np.random.default_rng(seed)
    C = int(rng.integers(2, 5))
    L = int(rng.integers(0, 4))
    tg = rng.integers(1, C, size=L).astype(np.int32)
    R = int(np.sum(tg[1:] == tg[:-1])) if L > 1 else 0
    T = L + R + int(rng.integers(0, 4))
    if T < 1:
        T = 1
    lp = rng.normal(size=(T, C)).astype(np.float32)
    o = oracle.ctc_forward_f64(lp, tg, 0)
    assert o["status"] == 0
    assert abs(o["total"] - brute_sum(lp, tg)) <= 1e-12 * (1 + abs(o["total"]))


def test_equals_torch_ctc_loss():
    for seed, (T, C, L) in enumerate([(50, 6, 10), (200, 32, 40), (120, 29, 30)]):
        u = synth.make_utterance(500 + seed, T, C, L, repeat_frac=0.2)
        o = oracle.ctc_forward_f64(u.lp.numpy(), u.targets, 0)
        loss = torch.nn.functional.ctc_loss(u.lp.double().unsqueeze(1), torch.as_tensor(u.targets, dtype=torch.long)[None],
                                            torch.tensor([T]), torch.tensor([L]), blank=0, reduction="sum")
        assert abs(o["total"] + loss.item()) <= 1e-9 * (1 + abs(o["total"]))


def test_closed_forms():
    # L = T without repeats: one path (the labels, no blank) -> its score.
    lp = np.log(np.full((3, 4), 0.25, np.float64)).astype(np.float32)
    o = oracle.ctc_forward_f64(lp, [1, 2, 3], 0)
    assert abs(o["total"] - 3 * math.log(0.25)) < 1e-6
    # Uniform emissions: total = log(number of valid paths) + T log(1/C).
    T, C, tg = 5, 3, [1, 2]
    n = len(brute.enumerate_paths(T, tg, 0))
    lp = np.full((T, C), math.log(1.0 / C), np.float32)
    o = oracle.ctc_forward_f64(lp, tg, 0)
    assert abs(o["total"] - (math.log(n) + T * float(np.float32(math.log(1.0 / C))))) < 1e-9
    # Empty transcript: the all-blank path only.
    lp = np.log(np.array([[0.5, 0.5], [0.25, 0.75]])).astype(np.float32)
    o = oracle.ctc_forward_f64(lp, [], 0)
    assert abs(o["total"] - (float(lp[0, 0]) + float(lp[1, 0]))) < 1e-12
    # The sum is at least the Viterbi maximum and at most it plus log(#paths).
    u = synth.make_utterance(9, 12, 4, 4)
    tot = oracle.ctc_forward_f64(u.lp.numpy(), u.targets, 0)["total"]
    best = oracle.viterbi_f64(u.lp.numpy(), u.targets, 0)["total"]
    n = len(brute.enumerate_paths(12, u.targets, 0))
    assert best <= tot <= best + math.log(n) + 1e-9


def test_infeasible_and_nopath():
    assert oracle.ctc_forward_f64(np.zeros((1, 3), np.float32), [1, 1], 0)["status"] == oracle.E_INFEASIBLE
    lp = np.full((3, 3), -np.inf, np.float32)
    assert oracle.ctc_forward_f64(lp, [1], 0)["status"] == oracle.E_NOPATH
