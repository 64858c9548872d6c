"""Error bounds and a closed form for the sum-product (CTC forward) score.

The kernel computes the forward score in FP32 and in base 2 (log2 of
probabilities): per cell beta = m + log2(1 + 2^(d1) + 2^(d2)) + e * log2(e),
m the largest allowed predecessor and d <= 0 the others' distances to it,
with the hardware 2^x and log2(x); the total is the log-add of the two final
states times ln 2. Error of one cell, in natural-log units, given exact
inputs: the two FP32 adds round by at most 2^-24 of |beta| each (2^-23 |beta|
together), the emission's conversion to base 2 by at most 1.5 * 2^-23 |e|
(product rounding plus the FP32 constant), the log-add by at most 2^-20 (the
approximate exponentials and logarithm on sums in [1, 3]). A log-sum-exp is a
convex combination of its inputs' errors (partial derivatives >= 0, summing
to 1), so an error carried from frame t-1 does not grow. Hence

    |total_fp32 - total| <= sum_t (2^-23 M_t + 1.5 * 2^-23 m_t + 2^-20)
                            + 2^-22 |total| + 2^-20,

M_t = the largest |beta_t(s)| over the finite states that can still reach a
final state (the only ones the total depends on), m_t = max_c |lp[t][c]|.

Closed form: with per-frame emissions equal across classes (0 here) except at
the last frame, every CTC path of a transcript without adjacent repeats has
score vb (ends on the trailing blank) or vl (ends on the last label), and the
paths are counted exactly by stars and bars: T - L spare frames spread over
the L + 1 blank runs (>= 0 frames) and the L label runs (>= 1 frame).
"""
from __future__ import annotations

import math

import numpy as np


def tolerance(lp: np.ndarray, amax: np.ndarray, total: float) -> float:
    """The bound above, with M_t from the binary64 oracle (live_abs_max)."""
    m = np.abs(np.where(np.isfinite(lp), lp, 0.0)).max(axis=1).astype(np.float64)
    body = float(np.sum(2.0 ** -23 * np.asarray(amax, np.float64) + 1.5 * 2.0 ** -23 * m + 2.0 ** -20))
    return (1.0 + 2.0 ** -10) * (body + 2.0 ** -22 * abs(total) + 2.0 ** -20)


def path_counts(L: int, T: int) -> tuple[int, int]:
    """(paths ending on the trailing blank, paths ending on the last label) for
    a transcript of L >= 1 labels without adjacent repeats and T >= L frames."""
    d = T - L
    n_blank = math.comb(d - 1 + 2 * L, 2 * L) if d >= 1 else 0
    n_label = math.comb(d + 2 * L - 1, 2 * L - 1)
    return n_blank, n_label


def closed_form_case(L: int, spare: int, C: int = 32):
    """Emissions, targets and the exact forward total of the closed form, with
    the two final states weighted about equally (so dropping either changes
    the total by about ln 2), and the error bound of the FP32 kernel on it.

    Every live state's partial paths extend to distinct complete paths, so
    0 <= beta_t(s) <= ln(N) for t < T-1 (emissions 0) and M_t <= ln(N) + |vl|."""
    T = L + spare
    tg = (1 + np.arange(L) % (C - 1)).astype(np.int32)   # 1, 2, ..., C-1, 1, 2, ...: no adjacent repeats
    n_b, n_l = path_counts(L, T)
    lp = np.zeros((T, C), np.float32)
    vb = np.float32(0.0)
    vl = np.float32(math.log(n_b) - math.log(n_l))      # balances the two final states
    lp[T - 1, 0] = vb
    lp[T - 1, tg[-1]] = vl
    xb = math.log(n_b) + float(vb)
    xl = math.log(n_l) + float(vl)
    mx = max(xb, xl)
    exact = mx + math.log(math.exp(xb - mx) + math.exp(xl - mx))
    B = math.log(n_b + n_l) + abs(float(vl))
    tol = (1.0 + 2.0 ** -10) * (T * (2.0 ** -23 * B + 2.0 ** -20) + 1.5 * 2.0 ** -23 * abs(float(vl))
                                + 2.0 ** -22 * abs(exact) + 2.0 ** -20)
    return lp, tg, exact, tol
