"""Seeded synthetic CTC emissions and transcripts.

The paper's forced-alignment feature (Sec. 4, "CTC-based forced alignment")
consumes the frame log-probabilities of a CTC acoustic model (20 ms frames,
wav2vec2-style character vocabularies) and a transcript. No model, dataset or
transcript is used here: these generators stand in for them with the same
shapes and structure.

Recipe, per utterance:
  * targets: uniform in 1..C-1 (blank = 0), optionally with a fraction of
    adjacent labels forced equal to the previous one;
  * a random feasible state path is planted: every label state gets >= 1
    frame, a blank gets >= 1 frame between two equal labels, and the remaining
    frames are spread over the 2L+1 states by a uniform multinomial;
  * logits = 3 * N(0, 1) with +4 added at the planted (frame, token) cells;
  * log_probs = log_softmax(logits) in FP32.

This module holds input generation only. It computes nothing of the alignment
method and is shared by the tests, the benchmark and the oracle checks.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

BASE_SEED = 2310178640
BLANK = 0


def config_seed(cfg: int) -> int:
    return BASE_SEED + int(cfg)


def sub_seed(seed: int, i: int) -> int:
    return (seed * 1000003 + i) % (2 ** 63)


def make_targets(rng: np.random.Generator, L: int, C: int, repeat_frac: float = 0.0,
                 blank: int = BLANK) -> np.ndarray:
    """Uniform labels in [0, C) minus the blank; a fraction forced equal to the previous label."""
    labels = rng.integers(0, C - 1, size=L).astype(np.int64)
    labels = labels + (labels >= blank)  # skip the blank id
    if repeat_frac > 0 and L > 1:
        rep = rng.random(L) < repeat_frac
        rep[0] = False
        for i in np.nonzero(rep)[0]:
            labels[i] = labels[i - 1]
    return labels.astype(np.int32)


def count_repeats(targets) -> int:
    t = np.asarray(targets)
    return int(np.sum(t[1:] == t[:-1])) if t.size > 1 else 0


def plant_state_path(rng: np.random.Generator, T: int, targets) -> np.ndarray:
    """A uniformly spread feasible state path over the 2L+1 CTC states (int32[T])."""
    t = np.asarray(targets)
    L = t.size
    S = 2 * L + 1
    need = np.zeros(S, dtype=np.int64)
    need[1::2] = 1
    if L > 1:
        eq = np.nonzero(t[1:] == t[:-1])[0]  # label i+1 equals label i
        need[2 * (eq + 1)] = 1               # the blank state between them
    extra = T - int(need.sum())
    if extra < 0:
        raise ValueError(f"infeasible: T={T} < L+R={int(need.sum())}")
    counts = need + rng.multinomial(extra, np.full(S, 1.0 / S))
    return np.repeat(np.arange(S, dtype=np.int32), counts)


def expand_tokens(targets, blank: int = BLANK) -> np.ndarray:
    t = np.asarray(targets, dtype=np.int64)
    ext = np.full(2 * t.size + 1, blank, dtype=np.int64)
    ext[1::2] = t
    return ext


def raw_logits(seed: int, T: int, C: int, planted_tokens: np.ndarray, device="cpu") -> torch.Tensor:
    """3*N(0,1) + 4*onehot(planted) as FP32 [T, C] (the scores before log_softmax)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    logits = torch.randn((T, C), generator=g, device=device, dtype=torch.float32)
    logits.mul_(3.0)
    idx = torch.as_tensor(planted_tokens, device=device, dtype=torch.int64)
    logits[torch.arange(T, device=device), idx] += 4.0
    return logits


def emissions(seed: int, T: int, C: int, planted_tokens: np.ndarray, device="cpu",
              out: torch.Tensor | None = None) -> torch.Tensor:
    """log_softmax(3*N(0,1) + 4*onehot(planted)) as FP32 [T, C]."""
    lp = torch.log_softmax(raw_logits(seed, T, C, planted_tokens, device), dim=-1)
    if out is not None:
        out.copy_(lp)
        return out
    return lp


@dataclasses.dataclass
class Utterance:
    lp: torch.Tensor          # [T, C] FP32
    targets: np.ndarray       # int32 [L]
    planted: np.ndarray       # int32 [T] planted state path
    seed: int

    @property
    def T(self) -> int:
        return int(self.lp.shape[0])

    @property
    def C(self) -> int:
        return int(self.lp.shape[1])

    @property
    def L(self) -> int:
        return int(self.targets.size)

    @property
    def cells(self) -> int:
        return self.T * (2 * self.L + 1)


def make_utterance(seed: int, T: int, C: int, L: int, repeat_frac: float = 0.0,
                   device="cpu", blank: int = BLANK, logits: bool = False) -> Utterance:
    """A seeded utterance; with logits=True, `lp` holds the raw scores before
    log_softmax (same seed: log_softmax of them is the logits=False lp)."""
    rng = np.random.default_rng(seed)
    targets = make_targets(rng, L, C, repeat_frac, blank)
    planted = plant_state_path(rng, T, targets)
    tokens = expand_tokens(targets, blank)[planted]
    if logits:
        lp = raw_logits(seed, T, C, tokens, device=device)
    else:
        lp = emissions(seed, T, C, tokens, device=device)
    return Utterance(lp=lp, targets=targets, planted=planted, seed=seed)


# ---------------------------------------------------------------- configs --

@dataclasses.dataclass
class Spec:
    T: int
    C: int
    L: int
    repeat_frac: float
    seed: int


def specs(cfg: int, *, C: int | None = None, n: int | None = None) -> list[Spec]:
    """Utterance shapes of the five workloads (sizes in frames of 20 ms).

    1: one utterance, T=200, C=32, L=40, ~10% forced adjacent repeats.
    2: 64 utterances, T uniform in 500..3000, L=round(T/4), C=32.
    3: one utterance, T=180000 (1 h), L=45000, C=32.
    4: 4096 utterances, T=clip(round(lognormal(ln 800, 0.8)), 50, 30000),
       L uniform in [round(T/5), round(T/3)], C in {32, 500} (C argument).
    5: serving stream, T=clip(round(lognormal(ln 1500, 0.8)), 100, 60000),
       L=T//4, C=32 (arrivals are drawn separately by ``arrivals``).
    ``n`` truncates the list (the first n utterances of the same stream).
    """
    seed = config_seed(cfg)
    rng = np.random.default_rng(seed)
    out: list[Spec] = []
    if cfg == 1:
        out = [Spec(200, 32, 40, 0.1, sub_seed(seed, 0))]
    elif cfg == 2:
        Ts = rng.integers(500, 3001, size=64)
        out = [Spec(int(T), 32, int(round(T / 4)), 0.0, sub_seed(seed, i)) for i, T in enumerate(Ts)]
    elif cfg == 3:
        out = [Spec(180000, 32, 45000, 0.0, sub_seed(seed, 0))]
    elif cfg == 4:
        cc = 32 if C is None else int(C)
        Ts = np.clip(np.round(rng.lognormal(math.log(800), 0.8, size=4096)), 50, 30000).astype(int)
        Ls = [int(rng.integers(int(round(T / 5)), int(round(T / 3)) + 1)) for T in Ts]
        out = [Spec(int(T), cc, L, 0.0, sub_seed(seed, i) ^ (cc << 40)) for i, (T, L) in enumerate(zip(Ts, Ls))]
    elif cfg == 5:
        count = 2200 if n is None else n
        Ts = np.clip(np.round(rng.lognormal(math.log(1500), 0.8, size=count)), 100, 60000).astype(int)
        out = [Spec(int(T), 32, int(T) // 4, 0.0, sub_seed(seed, i)) for i, T in enumerate(Ts)]
    else:
        raise ValueError(f"unknown workload {cfg}")
    if n is not None:
        out = out[:n]
    return out


def arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Poisson arrival times (seconds from 0) for a serving run."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


@dataclasses.dataclass
class Batch:
    lp: torch.Tensor              # packed [sum T, C] FP32 (all utterances share C)
    offsets: np.ndarray           # int64 [n+1] frame offsets into lp
    targets: list                 # list of int32 arrays
    planted: list                 # list of int32 arrays
    specs: list

    def __len__(self) -> int:
        return len(self.targets)

    def utt(self, i: int) -> torch.Tensor:
        return self.lp[int(self.offsets[i]):int(self.offsets[i + 1])]

    @property
    def cells(self) -> int:
        return int(sum((self.offsets[i + 1] - self.offsets[i]) * (2 * len(self.targets[i]) + 1)
                       for i in range(len(self))))


def make_batch(spec_list: list[Spec], device="cpu", logits: bool = False) -> Batch:
    """Generate every utterance into one packed [sum T, C] buffer (the raw
    scores before log_softmax when logits=True)."""
    Cs = {s.C for s in spec_list}
    if len(Cs) != 1:
        raise ValueError("a packed batch needs one vocabulary size")
    C = Cs.pop()
    offs = np.zeros(len(spec_list) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([s.T for s in spec_list])
    lp = torch.empty((int(offs[-1]), C), dtype=torch.float32, device=device)
    targets, planted = [], []
    for i, s in enumerate(spec_list):
        rng = np.random.default_rng(s.seed)
        tg = make_targets(rng, s.L, s.C, s.repeat_frac)
        pl = plant_state_path(rng, s.T, tg)
        if logits:
            lp[int(offs[i]):int(offs[i + 1])].copy_(raw_logits(s.seed, s.T, s.C, expand_tokens(tg)[pl], device=device))
        else:
            emissions(s.seed, s.T, s.C, expand_tokens(tg)[pl], device=device,
                      out=lp[int(offs[i]):int(offs[i + 1])])
        targets.append(tg)
        planted.append(pl)
    return Batch(lp=lp, offsets=offs, targets=targets, planted=planted, specs=spec_list)


# ---- decoder inputs (CTC beam search with blank collapse) ----
#
# Probabilities of a peaky CTC model over a V-token vocabulary (the paper's
# CUDA decoder experiment uses a 500-token vocabulary): a transcript of about
# T/10 tokens, each label on 1-2 frames, the other frames spread over the
# blanks around them; logits N(0,1) with a per-frame peak U[8, 16] added on
# the planted token, softmax in FP32. With V = 500 about 80 % of the planted
# frames get a probability above 0.95.

def decoder_probs(seed: int, T: int, V: int, device="cpu") -> torch.Tensor:
    rng = np.random.default_rng(seed)
    L = T // 10
    tg = make_targets(rng, L, V)
    lab = 1 + rng.integers(0, 2, size=L)
    blank_frames = T - int(lab.sum()) - int(np.sum(tg[1:] == tg[:-1]))
    if blank_frames < 0:
        raise ValueError("T too small for the planted transcript")
    eq = np.zeros(L + 1, dtype=np.int64)
    if L > 1:
        eq[1:L][tg[1:] == tg[:-1]] = 1      # a blank between equal labels
    bl = eq + rng.multinomial(blank_frames, np.full(L + 1, 1.0 / (L + 1)))
    tokens = []
    for i in range(L):
        tokens += [BLANK] * int(bl[i]) + [int(tg[i])] * int(lab[i])
    tokens += [BLANK] * int(bl[L])
    planted = np.asarray(tokens, dtype=np.int64)
    assert planted.size == T
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    logits = torch.randn((T, V), generator=g, dtype=torch.float32)
    peak = torch.from_numpy(rng.uniform(8.0, 16.0, size=T).astype(np.float32))
    logits[torch.arange(T), torch.from_numpy(planted)] += peak
    return torch.softmax(logits, dim=-1).to(device)


def decoder_batch(seed: int, n: int, V: int, t_lo: int = 250, t_hi: int = 1750, device="cpu"):
    """n utterances with T ~ U[t_lo, t_hi] packed: (probs [sum T, V], offsets int64 [n+1])."""
    rng = np.random.default_rng(seed)
    Ts = rng.integers(t_lo, t_hi + 1, size=n)
    parts = [decoder_probs(sub_seed(seed, i), int(T), V) for i, T in enumerate(Ts)]
    offsets = np.concatenate([[0], np.cumsum(Ts)]).astype(np.int64)
    return torch.cat(parts).to(device), offsets
