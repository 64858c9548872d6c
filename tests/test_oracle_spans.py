"""Pins of the token-span oracle (oracle/spans.py) against hand-derived cases,
invariants and the Viterbi oracle's own outputs."""
import numpy as np

import oracle
from oracle import spans
from paper_2310_17864_gb300 import synth


def test_hand_cases():
    # blank, a, a, blank, b, b, b, blank  (targets a, b): states 0,1,1,2,3,3,3,4
    st = np.array([0, 1, 1, 2, 3, 3, 3, 4])
    sc = np.array([-1.0, -0.5, -0.25, -2.0, -1.0, -2.0, -3.0, -0.5], np.float32)
    start, end, score = spans.token_spans(st, sc, 2)
    assert start.tolist() == [1, 4] and end.tolist() == [3, 7]
    assert score.tolist() == [np.float32(-0.375), np.float32(-2.0)]
    # Repeated label a, a with the mandatory blank between: states 1, 2, 3
    start, end, score = spans.token_spans(np.array([1, 2, 3]), np.array([-1, -2, -4], np.float32), 2)
    assert start.tolist() == [0, 2] and end.tolist() == [1, 3] and score.tolist() == [-1.0, -4.0]
    # Skip from label to label (no blank between different labels): states 1, 3, 3
    start, end, score = spans.token_spans(np.array([1, 3, 3]), np.array([-1, -1, -2], np.float32), 2)
    assert start.tolist() == [0, 1] and end.tolist() == [1, 3] and score.tolist() == [-1.0, -1.5]
    # Empty transcript: no spans.
    start, end, score = spans.token_spans(np.array([0, 0]), np.array([-1, -1], np.float32), 0)
    assert start.size == end.size == score.size == 0


def test_fp32_left_fold_and_division():
    # 1e8 + 1 + 1 - 1e8 in FP32 left to right is 0 (each +1 is rounded away); the mean is 0/4.
    st = np.array([1, 1, 1, 1])
    sc = np.array([1e8, 1.0, 1.0, -1e8], np.float32)
    _, _, score = spans.token_spans(st, sc, 1)
    assert score[0] == np.float32(0.0)
    # 1/3 in FP32 division of an FP32 sum
    _, _, score = spans.token_spans(np.array([1, 1, 1]), np.array([0.0, 0.0, 1.0], np.float32), 1)
    assert score[0] == np.float32(1.0) / np.float32(3.0)


def test_invariants_on_oracle_alignments():
    for seed, (T, C, L) in enumerate([(200, 32, 40), (500, 29, 150), (64, 5, 30), (1000, 32, 10)]):
        u = synth.make_utterance(100 + seed, T, C, L, repeat_frac=0.2)
        o = oracle.viterbi_f32(u.lp.numpy(), np.asarray(u.targets, np.int32), 0)
        start, end, score = spans.token_spans(o["states"], o["scores"], L)
        assert (start >= 0).all() and (end > start).all()
        assert (start[1:] >= end[:-1]).all()                         # ordered, disjoint
        odd = (o["states"] % 2 == 1)
        assert int((end - start).sum()) == int(odd.sum())             # cover the label frames exactly
        for i in range(L):                                            # every frame of span i is token i
            assert (o["path"][start[i]:end[i]] == u.targets[i]).all()
        # Blank frames between spans of equal labels
        for i in range(1, L):
            if u.targets[i] == u.targets[i - 1]:
                assert start[i] > end[i - 1]


def test_packed_equals_per_utterance():
    specs = synth.specs(2, n=6)
    outs, st_all, sc_all, foff, toff = [], [], [], [0], [0]
    for s in specs:
        u = synth.make_utterance(s.seed, s.T, s.C, s.L, s.repeat_frac)
        o = oracle.viterbi_f32(u.lp.numpy(), np.asarray(u.targets, np.int32), 0)
        outs.append(spans.token_spans(o["states"], o["scores"], s.L))
        st_all.append(o["states"]); sc_all.append(o["scores"])
        foff.append(foff[-1] + s.T); toff.append(toff[-1] + s.L)
    packed = spans.token_spans_packed(np.concatenate(st_all), np.concatenate(sc_all), foff, toff)
    for k in range(3):
        assert np.array_equal(packed[k], np.concatenate([x[k] for x in outs]))
