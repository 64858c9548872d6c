"""log_softmax over each frame -- oracle, TEST INFRASTRUCTURE ONLY.

The paper's aligner consumes the frame log-probabilities of a CTC model
(Sec. 4, "CTC-based forced alignment"); a model's last layer gives raw
per-frame scores, and log_softmax over the classes of each frame turns them
into log-probabilities: lp[t][c] = x[t][c] - log(sum_k exp(x[t][k])). Written
out in FP64 with the row maximum subtracted first (the identity
log sum exp(x) = m + log sum exp(x - m)); rows whose entries are all -inf give
NaN, as the formula does.

Only tests/ and the CPU legs of bench.py import this module.
"""
from __future__ import annotations

import numpy as np


def log_softmax64(logits):
    """logits: float [T, C] -> (lp float64 [T, C], lse float64 [T])."""
    x = np.asarray(logits, dtype=np.float64)
    m = x.max(axis=1, keepdims=True)
    with np.errstate(invalid="ignore"):
        lse = m + np.log(np.exp(x - m).sum(axis=1, keepdims=True))
        lp = x - lse
    return lp, lse[:, 0]


def path_score64(lp64, tokens):
    """FP64 sum of lp64[t][tokens[t]] over the frames."""
    lp64 = np.asarray(lp64)
    return float(lp64[np.arange(lp64.shape[0]), np.asarray(tokens)].sum())
