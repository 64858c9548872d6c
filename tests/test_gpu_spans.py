"""GPU parity of the token-span kernels (align_token_spans) against the
token-span oracle, on alignments produced by the library (bit-exact: spans
equal, scores equal bit for bit)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import spans
from paper_2310_17864_gb300 import align, build, synth

pytestmark = pytest.mark.gpu


def _packed_alignments(utts):
    """Align each utterance (device path, states kept); pack states/scores."""
    al = align.Aligner(device=0, bp_budget_bytes=4 << 30)
    try:
        st, sc, foff, toff = [], [], [0], [0]
        for u in utts:
            r = al.align(u.lp.cuda(), u.targets, 0, want_states=True)
            assert r.status == 0
            st.append(r.states)
            sc.append(r.scores)
            foff.append(foff[-1] + u.lp.shape[0])
            toff.append(toff[-1] + len(u.targets))
        return torch.cat(st), torch.cat(sc), np.array(foff), np.array(toff)
    finally:
        al.close()


def _check(states, scores, foff, toff):
    start, end, score = align.token_spans(states, scores, foff, toff)
    torch.cuda.synchronize()
    rs, re, rsc = spans.token_spans_packed(states.cpu().numpy(), scores.cpu().numpy(), foff, toff)
    assert np.array_equal(start.cpu().numpy(), rs)
    assert np.array_equal(end.cpu().numpy(), re)
    assert score.cpu().numpy().tobytes() == rsc.tobytes()


def test_spans_of_batch_alignments():
    build.build()
    utts = [synth.make_utterance(s.seed, s.T, s.C, s.L, s.repeat_frac) for s in synth.specs(2, n=12)]
    _check(*_packed_alignments(utts))


def test_spans_edge_cases():
    build.build()
    utts = [synth.make_utterance(1, 1, 4, 0),            # T = 1, empty transcript
            synth.make_utterance(2, 7, 5, 3, repeat_frac=1.0),   # tight, repeats
            synth.make_utterance(3, 300, 32, 0),         # long, empty transcript
            synth.make_utterance(4, 50, 3, 24, repeat_frac=0.0),  # near tight
            synth.make_utterance(5, 2000, 32, 600, repeat_frac=0.3)]
    _check(*_packed_alignments(utts))


def test_spans_without_frames():
    """States that visit no label state: every token gets -1, -1, 0."""
    build.build()
    states = torch.zeros(10, dtype=torch.int32, device="cuda")
    scores = torch.full((10,), -1.0, device="cuda")
    start, end, score = align.token_spans(states, scores, [0, 4, 10], [0, 2, 3])
    assert start.tolist() == [-1, -1, -1] and end.tolist() == [-1, -1, -1] and score.tolist() == [0.0, 0.0, 0.0]
