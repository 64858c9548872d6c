"""GPU parity of the CTC prefix beam search with blank collapse
(align_ctc_beam_decode) against the binary32 oracle (oracle/beam.py).

Both sides evaluate the same binary32 operations in the same order (the
rescale is by powers of two, exact), so the kept frames, every hypothesis'
labels and label frames, its total (bits) and the scale exponent must be
equal; only the reported log score, logf(total) + E ln 2 in FP32, is
compared with a tolerance: logf within 1 ulp (2^-23 relative), the FP32
constant ln 2 and product E ln 2 within 2^-23 relative each, and the final
add within 2^-24 of the result: 2^-21 (|log total| + |E| ln 2) covers them.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import beam
from paper_2310_17864_gb300 import align, build, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "beam_hand.json")


@pytest.fixture(scope="module", autouse=True)
def _build():
    build.build()


def decode(parts, B, blank, a):
    P = torch.cat([torch.as_tensor(p, dtype=torch.float32) for p in parts]).contiguous()
    off = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])]).astype(np.int64)
    res = align.ctc_beam_decode(P.cuda(), off, beam=B, blank=blank, threshold=a)
    torch.cuda.synchronize()
    return res


def compare(res, u, P, B, blank, a, label=""):
    o = beam.beam_search(np.asarray(P, np.float32), blank, B, a)
    assert int(res.kept[u]) == len(o["kept"]), label
    assert int(res.scale_exp[u]) == o["exp"], (label, int(res.scale_exp[u]), o["exp"])
    hyps = res.hypotheses(u)
    assert len(hyps) == len(o["hyps"]), (label, len(hyps), len(o["hyps"]))
    lens = res.lengths[u].cpu().numpy()
    assert (lens[len(o["hyps"]):] == -1).all(), label
    tot = res.totals[u].cpu().numpy()
    for b, ((tk, tm, sc), (prefix, times, total, _, _)) in enumerate(zip(hyps, o["hyps"])):
        assert tk == list(prefix), (label, b, tk[:10], list(prefix)[:10])
        assert tm == list(times), (label, b)
        assert np.float32(tot[b]).tobytes() == np.float32(total).tobytes(), (label, b, tot[b], total)
        want = beam.log_score(total, o["exp"])
        if want == -math.inf:
            assert sc == -math.inf
        else:
            tol = 2.0 ** -21 * (abs(math.log(float(total))) + abs(o["exp"]) * math.log(2.0)) + 1e-30
            assert abs(sc - want) <= tol, (label, b, sc, want, tol)
    return o


def test_hand_examples():
    for c in json.load(open(GOLDEN))["cases"]:
        P = np.asarray(c["P"], np.float32)
        res = decode([P], c["beam"], c["blank"], c["a"])
        compare(res, 0, P, c["beam"], c["blank"], c["a"], c["name"])


@pytest.mark.parametrize("T,V,B,blank,a", [
    (1, 2, 1, 0, 1.0), (5, 3, 4, 0, 1.0), (12, 5, 16, 2, 1.0), (60, 20, 8, 0, 0.95), (200, 29, 10, 0, 0.95),
    (150, 31, 3, 5, 0.9), (120, 64, 16, 0, 1.0), (300, 500, 10, 0, 0.95), (250, 500, 16, 0, 1.0),
    (90, 7, 1, 0, 0.5),
])
def test_shapes(T, V, B, blank, a):
    """Vocabularies with and without 16-byte rows, beams 1..16, blanks other
    than 0, thresholds from none to aggressive."""
    P = synth.decoder_probs(T * 7 + V + B, T, V)
    if blank:
        P = P[:, torch.roll(torch.arange(V), blank)]  # move the planted blank column to `blank`
    res = decode([P], B, blank, a)
    compare(res, 0, P.numpy(), B, blank, a, f"T{T}V{V}B{B}a{a}")


def test_packed_batch():
    """A packed ragged batch: each utterance equals the oracle on its own."""
    parts = [synth.decoder_probs(100 + i, T, 40) for i, T in enumerate([33, 150, 1, 77, 260, 12])]
    res = decode(parts, 6, 0, 0.95)
    for u, P in enumerate(parts):
        compare(res, u, P.numpy(), 6, 0, 0.95, f"utt{u}")


def test_flat_rows_overflow_the_survivor_list():
    """Uniform rows with a vocabulary of 1,500: every growth ties with every
    other, so the first frame's candidates (beyond the survivor list) go
    through the exact fallback; ties go to the smaller index."""
    T, V = 6, 1500
    P = np.full((T, V), 1.0 / V, np.float32)
    res = decode([P], 16, 0, 1.0)
    compare(res, 0, P, 16, 0, 1.0, "flat")
    rng = np.random.default_rng(3)
    Q = rng.integers(1, 3, size=(8, 3000)).astype(np.float32) / 4096.0  # many exact ties
    res = decode([Q], 12, 0, 1.0)
    compare(res, 0, Q, 12, 0, 1.0, "ties")


def test_one_hot_and_zero_rows():
    """One-hot frames (zeros everywhere else, many zero-valued candidates)
    and a row of zeros (every total zero: no rescale)."""
    path = [0, 0, 3, 3, 0, 3, 1, 1, 0, 0, 2, 0, 2, 2, 0]
    P = np.zeros((len(path), 5), np.float32)
    P[np.arange(len(path)), path] = 1.0
    for a in (1.0, 0.95):
        res = decode([P], 4, 0, a)
        compare(res, 0, P, 4, 0, a, f"onehot{a}")
    Z = np.zeros((4, 6), np.float32)
    Z[0] = 1.0 / 6
    res = decode([Z], 3, 0, 1.0)
    compare(res, 0, Z, 3, 0, 1.0, "zeros")


def test_validation():
    P = torch.rand(10, 5, device="cuda")
    for kw in ({"beam": 0}, {"beam": 17}, {"blank": 5}, {"threshold": -1.0}):
        args = {"beam": 4, "blank": 0, "threshold": 1.0}
        args.update(kw)
        with pytest.raises(align.AlignError) as e:
            align.ctc_beam_decode(P, [0, 10], **args)
        assert e.value.code == align.ALIGN_E_INVAL
