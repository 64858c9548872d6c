"""Invariants of a CTC forced alignment -- TEST INFRASTRUCTURE ONLY.

Each function restates a property that any correct alignment has (paper Sec. 4,
"CTC-based forced alignment"; CTC collapse map and trellis of the cited CTC
work), written independently of the oracle's recursion so that it can pin it.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24  # unit roundoff of binary32


def collapse(path, blank: int) -> list[int]:
    """CTC map B: merge runs of equal tokens, then drop blanks."""
    out = []
    prev = None
    for tok in path:
        tok = int(tok)
        if tok != prev and tok != blank:
            out.append(tok)
        prev = tok
    return out


def legal_state_path(states, targets, blank: int) -> bool:
    """Start in {0,1}, end in {S-1,S-2}, steps of 0/1/2 with the CTC skip rule."""
    ext = [blank]
    for lab in targets:
        ext += [int(lab), blank]
    S = len(ext)
    st = [int(s) for s in states]
    if not st or st[0] not in ((0, 1) if S > 1 else (0,)):
        return False
    if st[-1] not in ((S - 1, S - 2) if S > 1 else (0,)):
        return False
    for a, b in zip(st, st[1:]):
        d = b - a
        if d not in (0, 1, 2) or b >= S:
            return False
        if d == 2 and not (b % 2 == 1 and b >= 3 and ext[b] != ext[b - 2]):
            return False
    return True


def fold_f32(values) -> np.float32:
    """Left-to-right binary32 sum starting from the first element."""
    v = np.asarray(values, dtype=np.float32)
    acc = np.float32(v[0])
    for x in v[1:]:
        acc = np.float32(acc + x)
    return acc


def fold_f32_fast(values) -> np.float32:
    """Same left fold, vectorised through cumulative sums in binary32 (numpy
    accumulates sequentially for cumsum, so the result is the same fold)."""
    v = np.asarray(values, dtype=np.float32)
    return np.cumsum(v, dtype=np.float32)[-1]


def gamma(n: int, u: float = U32) -> float:
    """Recursive-summation error constant gamma_n = n u / (1 - n u)."""
    return n * u / (1.0 - n * u)


def ext_array(targets, blank: int) -> np.ndarray:
    L = len(targets)
    ext = np.full(2 * L + 1, blank, dtype=np.int64)
    ext[1::2] = np.asarray(targets, dtype=np.int64)
    return ext


def skip_mask(ext: np.ndarray) -> np.ndarray:
    S = ext.size
    m = np.zeros(S, dtype=bool)
    if S >= 4:
        idx = np.arange(3, S, 2)
        m[idx] = ext[idx] != ext[idx - 2]
    return m


def backward_maxplus_f64(lp, targets, blank: int) -> np.ndarray:
    """beta_t(s): best binary64 sum of emissions over frames t..T-1 for paths in
    state s at frame t that end in a final state. Vectorised over s; runs
    backwards in time, so it shares no step with a forward recursion."""
    lp = np.asarray(lp, dtype=np.float64)
    T = lp.shape[0]
    ext = ext_array(targets, blank)
    S = ext.size
    skip = skip_mask(ext)
    beta = np.full((T, S), -np.inf)
    beta[T - 1, S - 1] = lp[T - 1, ext[S - 1]]
    if S > 1:
        beta[T - 1, S - 2] = lp[T - 1, ext[S - 2]]
    for t in range(T - 2, -1, -1):
        nxt = beta[t + 1]
        best = nxt.copy()                       # stay: s -> s
        best[:-1] = np.maximum(best[:-1], nxt[1:])   # advance: s -> s+1
        if S > 2:
            cand = np.where(skip[2:], nxt[2:], -np.inf)  # skip: s -> s+2 when allowed
            best[:-2] = np.maximum(best[:-2], cand)
        beta[t] = best + lp[t, ext]
    return beta


def forward_maxplus_f64(lp, targets, blank: int) -> np.ndarray:
    """alpha_t(s) in binary64, vectorised over s (a second restatement of the
    forward recursion, used only together with the backward pass)."""
    lp = np.asarray(lp, dtype=np.float64)
    T = lp.shape[0]
    ext = ext_array(targets, blank)
    S = ext.size
    skip = skip_mask(ext)
    alpha = np.full((T, S), -np.inf)
    alpha[0, 0] = lp[0, ext[0]]
    if S > 1:
        alpha[0, 1] = lp[0, ext[1]]
    for t in range(1, T):
        prv = alpha[t - 1]
        best = prv.copy()
        best[1:] = np.maximum(best[1:], prv[:-1])
        if S > 2:
            cand = np.where(skip[2:], prv[:-2], -np.inf)
            best[2:] = np.maximum(best[2:], cand)
        alpha[t] = best + lp[t, ext]
    return alpha
