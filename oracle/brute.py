"""Exhaustive search over CTC state paths for tiny problems -- TEST INFRASTRUCTURE ONLY.

This is the plain definition of the alignment problem (paper Sec. 4, "CTC-based
forced alignment"; trellis of the cited CTC work): among all monotone state
sequences s_0..s_{T-1} over the 2L+1 blank-interleaved states that start in
state 0 or 1, end in state 2L or 2L-1, move by 0, 1 or 2 per frame, and skip
(move by 2) only into a label state whose label differs from the label two
states back, pick the one with the largest emission sum. Every path is
enumerated; nothing here uses dynamic programming.

Sums are left folds in the given precision starting from the first frame's
emission, exactly as a Viterbi recursion accumulates them.
"""
from __future__ import annotations

import numpy as np


def expand(targets, blank: int) -> list[int]:
    ext = [blank]
    for lab in targets:
        ext += [int(lab), blank]
    return ext


def _skip_ok(ext, s: int) -> bool:
    return s % 2 == 1 and s >= 3 and ext[s] != ext[s - 2]


def enumerate_paths(T: int, targets, blank: int):
    """Yield every valid state sequence as a tuple of length T."""
    ext = expand(targets, blank)
    S = len(ext)
    finals = {S - 1, S - 2} if S > 1 else {0}
    starts = [0, 1] if S > 1 else [0]
    out = []

    def rec(seq):
        t = len(seq)
        if t == T:
            if seq[-1] in finals:
                out.append(tuple(seq))
            return
        s = seq[-1]
        # Remaining frames must be able to reach a final state: each frame moves by <= 2.
        for nxt in (s, s + 1, s + 2):
            if nxt >= S:
                continue
            if nxt == s + 2 and not _skip_ok(ext, nxt):
                continue
            seq.append(nxt)
            rec(seq)
            seq.pop()

    for s0 in starts:
        rec([s0])
    return out


def fold(values, dtype):
    acc = dtype(values[0])
    for v in values[1:]:
        acc = dtype(acc + dtype(v))
    return acc


def path_score(lp, states, ext, dtype=np.float32):
    return fold([lp[t][ext[s]] for t, s in enumerate(states)], dtype)


def brute_force(lp, targets, blank: int, dtype=np.float32) -> dict:
    """Best score, all optimal state paths and the reverse-lexicographically greatest one."""
    lp = np.asarray(lp, dtype=np.float32)
    T = lp.shape[0]
    ext = expand(targets, blank)
    paths = enumerate_paths(T, targets, blank)
    if not paths:
        return {"n_paths": 0, "best": None, "optimal": [], "chosen": None}
    scores = [path_score(lp, p, ext, dtype) for p in paths]
    best = max(scores)
    optimal = [p for p, sc in zip(paths, scores) if sc == best]
    chosen = max(optimal, key=lambda p: tuple(reversed(p)))
    return {"n_paths": len(paths), "best": best, "optimal": optimal, "chosen": chosen}
