"""Token spans of a forced alignment -- oracle, TEST INFRASTRUCTURE ONLY.

The paper (Sec. 4, "CTC-based forced alignment") presents forced alignment as
producing the alignment between audio frames and transcript tokens. Collapsing
the frame-level alignment into one span per transcript token is the form such
a consumer needs: transcript token i (0-based) occupies exactly the frames
whose trellis state is the label state 2i + 1, and on a valid CTC path those
frames are consecutive. This module writes that definition out with plain
Python loops:

  start[i] = first frame t with states[t] == 2i + 1
  end[i]   = one past the last such frame
  score[i] = (scores[start] + scores[start+1] + ... + scores[end-1]) / (end - start)

The sum is an FP32 left fold in frame order and the division one FP32 division
(the result a caller gets from the same float32 arithmetic). A token with no
frame (impossible for a valid alignment) gets start = end = -1, score = 0.

Only tests/ and the CPU legs of bench.py import this module.
"""
from __future__ import annotations

import numpy as np


def token_spans(states, scores, L: int):
    """states: int [T] trellis states of one alignment; scores: float32 [T];
    L: transcript length. Returns (start int32 [L], end int32 [L], score float32 [L])."""
    states = np.asarray(states)
    scores = np.asarray(scores, dtype=np.float32)
    start = np.full(L, -1, dtype=np.int32)
    end = np.full(L, -1, dtype=np.int32)
    score = np.zeros(L, dtype=np.float32)
    for t in range(states.size):
        s = int(states[t])
        if s % 2 == 1:
            i = (s - 1) // 2
            if start[i] < 0:
                start[i] = t
            end[i] = t + 1
    for i in range(L):
        if start[i] < 0:
            continue
        acc = np.float32(0.0)
        for t in range(start[i], end[i]):
            acc = np.float32(acc + scores[t])
        score[i] = np.float32(acc / np.float32(end[i] - start[i]))
    return start, end, score


def token_spans_packed(states, scores, frame_offsets, token_offsets):
    """A packed batch: utterance u owns frames frame_offsets[u]:frame_offsets[u+1]
    and tokens token_offsets[u]:token_offsets[u+1]; frames in the outputs are
    relative to the utterance's first frame."""
    n = len(frame_offsets) - 1
    parts = [token_spans(states[frame_offsets[u]:frame_offsets[u + 1]], scores[frame_offsets[u]:frame_offsets[u + 1]],
                         int(token_offsets[u + 1] - token_offsets[u])) for u in range(n)]
    if not parts:
        return (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(3))
