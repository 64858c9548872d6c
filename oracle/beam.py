"""CTC prefix beam search with blank collapse -- TEST INFRASTRUCTURE ONLY.

The CUDA CTC decoder of the paper (Sec. 5, "CUDA CTC decoder"): beam search
over CTC outputs, parallel over batch, hypotheses and vocabulary, after the
blank-collapse step it cites (frames whose blank probability exceeds a
threshold a are blank frames; a = 0.95 in its experiment, a = 1.0 disables
it). Written here as the textbook CTC prefix beam search, plainly:

* blank collapse: frame t is a blank frame when P[t, blank] > a; a frame is
  dropped when it and the frame before it are both blank frames, so every run
  of blank frames shrinks to its first frame (a single blank still separates
  two equal labels, so no prefix changes meaning);
* each hypothesis is a label prefix with two probabilities: pb (paths that end
  in blank) and pnb (paths that end in the prefix's last label);
* per kept frame with probabilities y, a hypothesis h with last label z can
  stay (blank: pb' = (pb + pnb) * y[blank]; repeat of z: pnb' = pnb * y[z]) or
  grow by a label c (pnb(h + c) = (pb + pnb) * y[c], or pb * y[c] when c = z,
  since a repeated label needs a blank in between);
* a grown prefix that equals a hypothesis already in the beam adds into that
  hypothesis' pnb instead of becoming a new one;
* the beam keeps the B largest totals pb + pnb.

Arithmetic: binary32, one rounding per operation in the order written below
(numpy float32 operations), so that the CUDA decoder can match it bit for
bit. Probabilities are rescaled after every frame by a power of two (exact)
so that the largest total lies in [0.5, 1); the exponents are summed in an
integer. Ties in the selection go to the candidate with the smaller index:
staying hypotheses first (index = beam slot i), then growths (index =
B + i * V + c).
"""
from __future__ import annotations

import math

import numpy as np

F = np.float32


def blank_collapse(P: np.ndarray, blank: int, a: float) -> np.ndarray:
    """Indices of the frames kept by blank collapse (threshold a)."""
    P = np.asarray(P, dtype=np.float32)
    is_blank = P[:, blank] > F(a)
    keep = np.ones(P.shape[0], dtype=bool)
    keep[1:] = ~(is_blank[1:] & is_blank[:-1])
    return np.nonzero(keep)[0]


class Hyp:
    __slots__ = ("prefix", "times", "pb", "pnb")

    def __init__(self, prefix, times, pb, pnb):
        self.prefix = prefix
        self.times = times
        self.pb = F(pb)
        self.pnb = F(pnb)


def beam_search(P: np.ndarray, blank: int, beam: int, a: float = 1.0) -> dict:
    """Prefix beam search over the kept frames of P ([T, V] probabilities).

    Returns {"kept": frame indices, "hyps": [(prefix, times, total, pb, pnb)]
    in beam order (largest total first), "exp": E} where the probability of a
    hypothesis is total * 2**E and times[k] is the frame at which label k of
    the prefix was first emitted.
    """
    P = np.asarray(P, dtype=np.float32)
    T, V = P.shape
    B = int(beam)
    kept = blank_collapse(P, blank, a)
    hyps = [Hyp((), (), 1.0, 0.0)]
    E = 0
    labels = np.arange(V)
    for t in kept:
        y = P[t]
        n = len(hyps)
        s = [F(h.pb + h.pnb) for h in hyps]
        stay_b = [F(s[i] * y[blank]) for i in range(n)]
        stay_nb = [F(h.pnb * y[h.prefix[-1]]) if h.prefix else F(0.0) for h in hyps]
        # A growth of hypothesis i by c that equals hypothesis j joins j.
        merged = set()
        for j, hj in enumerate(hyps):
            if not hj.prefix:
                continue
            for i, hi in enumerate(hyps):
                if hi.prefix == hj.prefix[:-1]:
                    c = hj.prefix[-1]
                    base = hi.pb if (hi.prefix and hi.prefix[-1] == c) else s[i]
                    stay_nb[j] = F(stay_nb[j] + F(base * y[c]))
                    merged.add((i, c))
                    break
        vals, idxs, srcs = [], [], []
        for i in range(n):
            vals.append(F(stay_b[i] + stay_nb[i]))
            idxs.append(i)
            srcs.append(("stay", i, -1))
        for i, h in enumerate(hyps):
            z = h.prefix[-1] if h.prefix else -1
            base = np.full(V, s[i], dtype=np.float32)
            if z >= 0:
                base[z] = h.pb
            ext = (base * y).astype(np.float32)
            for c in labels:
                if c == blank or (i, int(c)) in merged:
                    continue
                vals.append(ext[c])
                idxs.append(B + i * V + int(c))
                srcs.append(("grow", i, int(c)))
        vals_a = np.asarray(vals, dtype=np.float32)
        order = np.lexsort((np.asarray(idxs, dtype=np.int64), -vals_a.astype(np.float64)))[:B]
        new = []
        for o in order:
            kind, i, c = srcs[o]
            h = hyps[i]
            if kind == "stay":
                new.append(Hyp(h.prefix, h.times, stay_b[i], stay_nb[i]))
            else:
                new.append(Hyp(h.prefix + (c,), h.times + (int(t),), 0.0, vals_a[o]))
        hyps = new
        m = max(F(h.pb + h.pnb) for h in hyps)
        if m > 0:
            e = math.frexp(float(m))[1]  # m = f * 2**e, f in [0.5, 1)
            for h in hyps:
                h.pb = F(np.ldexp(h.pb, -e))
                h.pnb = F(np.ldexp(h.pnb, -e))
            E += e
    out = [(h.prefix, h.times, F(h.pb + h.pnb), h.pb, h.pnb) for h in hyps]
    return {"kept": kept, "hyps": out, "exp": E}


def log_score(total, E: int) -> float:
    """log of total * 2**E (binary64)."""
    return math.log(float(total)) + E * math.log(2.0) if total > 0 else -math.inf
