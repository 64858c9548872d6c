"""The beam-search oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/beam.py (loaded as a
separate module on the CPU) and runs the pins of tests/test_oracle_beam.py
against it: at least one must fail.
"""
import importlib.util
import os
import sys
import types

import pytest

import oracle
from oracle import beam as beam_ok

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_beam as pins  # noqa: E402

SRC = beam_ok.__file__

MUTANTS = {
    "repeat_without_blank": ("base[z] = h.pb", "base[z] = s[i]"),
    "no_merge": ("stay_nb[j] = F(stay_nb[j] + F(base * y[c]))\n                    merged.add((i, c))",
                 "pass"),
    "ties_to_larger_index": ("np.lexsort((np.asarray(idxs, dtype=np.int64),", "np.lexsort((-np.asarray(idxs, dtype=np.int64),"),
    "collapse_keeps_last_of_run": ("keep[1:] = ~(is_blank[1:] & is_blank[:-1])", "keep[:-1] = ~(is_blank[:-1] & is_blank[1:])"),
    "threshold_inclusive": ("is_blank = P[:, blank] > F(a)", "is_blank = P[:, blank] >= F(a)"),
    "repeat_from_pb": ("F(h.pnb * y[h.prefix[-1]])", "F(h.pb * y[h.prefix[-1]])"),
    "blank_from_pb_only": ("stay_b = [F(s[i] * y[blank])", "stay_b = [F(hyps[i].pb * y[blank])"),
    "rescale_wrong_way": ("h.pb = F(np.ldexp(h.pb, -e))\n                h.pnb = F(np.ldexp(h.pnb, -e))",
                          "h.pb = F(np.ldexp(h.pb, e))\n                h.pnb = F(np.ldexp(h.pnb, e))"),
    "times_of_previous_frame": ("h.times + (int(t),)", "h.times + (int(t) - 1,)"),
}


def load_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"beam_mutant_{name}")
    exec(compile(src.replace(old, new), f"<{name}>", "exec"), mod.__dict__)
    return mod


def battery(mod) -> list[str]:
    failed = []
    saved = pins.beam
    pins.beam = mod
    try:
        for fn in (pins.test_hand_examples, pins.test_blank_collapse_runs, pins.test_hypotheses_match_forward_score,
                   pins.test_pruning_only_loses_paths, pins.test_one_hot_planted_path):
            try:
                fn()
            except AssertionError:
                failed.append(fn.__name__)
        for args in [(3, 3, 0, 2), (4, 3, 2, 3), (3, 4, 0, 5)]:
            try:
                pins.test_unpruned_beam_is_every_sequence(*args)
            except AssertionError:
                failed.append("unpruned")
    finally:
        pins.beam = saved
    return failed


def test_unmodified_oracle_passes():
    assert battery(beam_ok) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    assert battery(load_mutant(name)), name
