"""Pins of the FP64 log_softmax oracle (oracle/normalize.py)."""
import math

import numpy as np

from oracle import normalize


def test_closed_forms():
    lp, lse = normalize.log_softmax64([[0.0, 0.0]])
    assert np.allclose(lp, -math.log(2.0), rtol=0, atol=1e-15) and abs(lse[0] - math.log(2.0)) < 1e-15
    lp, lse = normalize.log_softmax64([[math.log(1.0), math.log(3.0)]])  # probabilities 1/4, 3/4
    assert abs(lp[0, 0] - math.log(0.25)) < 1e-15 and abs(lp[0, 1] - math.log(0.75)) < 1e-15
    lp, _ = normalize.log_softmax64([[0.0, -np.inf, 0.0]])           # a -inf class has probability 0
    assert lp[0, 1] == -np.inf and abs(lp[0, 0] - math.log(0.5)) < 1e-15


def test_rows_sum_to_one_and_shift_invariance():
    rng = np.random.default_rng(3)
    x = rng.normal(0.0, 3.0, size=(50, 37)).astype(np.float32)
    lp, _ = normalize.log_softmax64(x)
    assert np.allclose(np.exp(lp).sum(axis=1), 1.0, rtol=0, atol=1e-12)
    lp2, _ = normalize.log_softmax64(x.astype(np.float64) + 1000.0)   # huge shift: no overflow
    assert np.allclose(lp, lp2, rtol=0, atol=1e-9)
    assert (np.argmax(lp, axis=1) == np.argmax(x, axis=1)).all()       # order preserving


def test_path_score():
    lp = np.log(np.array([[0.5, 0.5], [0.25, 0.75]]))
    assert abs(normalize.path_score64(lp, [0, 1]) - math.log(0.375)) < 1e-15
