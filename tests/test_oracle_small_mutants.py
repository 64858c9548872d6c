"""The pins of the token-span and log_softmax oracles must catch plausible
mistakes: each case plants one in a copy of the module (loaded on the CPU)
and runs the pins of tests/test_oracle_spans.py / test_oracle_normalize.py
against it; at least one must fail."""
import os
import sys
import types

import pytest

from oracle import normalize as normalize_ok
from oracle import spans as spans_ok

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_normalize as npins  # noqa: E402
import test_oracle_spans as spins  # noqa: E402

SPAN_MUTANTS = {
    "end_is_last_frame": ("end[i] = t + 1", "end[i] = t"),
    "token_of_state": ("i = (s - 1) // 2", "i = s // 2 - 1 if s > 1 else 0"),
    "mean_over_one_more": ("np.float32(end[i] - start[i])", "np.float32(end[i] - start[i] + 1)"),
    "fold_in_float64": ("acc = np.float32(acc + scores[t])", "acc = acc + np.float64(scores[t])"),
    "last_span_start": ("if start[i] < 0:\n                start[i] = t", "start[i] = t"),
}
NORM_MUTANTS = {
    "no_log": ("m + np.log(np.exp(x - m).sum(axis=1, keepdims=True))", "m + np.exp(x - m).sum(axis=1, keepdims=True)"),
    "shift_not_added_back": ("lse = m + np.log(", "lse = np.log("),
    "sign": ("lp = x - lse", "lp = lse - x"),
    "max_over_columns": ("m = x.max(axis=1, keepdims=True)", "m = x.max(axis=0, keepdims=True)"),
}


def _mutant(module, old, new, name):
    src = open(module.__file__).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"mutant_{name}")
    exec(compile(src.replace(old, new), f"<{name}>", "exec"), mod.__dict__)
    return mod


def _run(pinmod, attr, mod, names):
    saved = getattr(pinmod, attr)
    setattr(pinmod, attr, mod)
    failed = []
    try:
        for n in names:
            try:
                getattr(pinmod, n)()
            except (AssertionError, IndexError, ValueError):
                failed.append(n)
    finally:
        setattr(pinmod, attr, saved)
    return failed


SPAN_PINS = ["test_hand_cases", "test_fp32_left_fold_and_division", "test_invariants_on_oracle_alignments"]
NORM_PINS = ["test_closed_forms", "test_rows_sum_to_one_and_shift_invariance"]


def test_unmodified_oracles_pass():
    assert _run(spins, "spans", spans_ok, SPAN_PINS) == []
    assert _run(npins, "normalize", normalize_ok, NORM_PINS) == []


@pytest.mark.parametrize("name", sorted(SPAN_MUTANTS))
def test_span_mutant_is_caught(name):
    mod = _mutant(spans_ok, *SPAN_MUTANTS[name], name)
    assert _run(spins, "spans", mod, SPAN_PINS), name


@pytest.mark.parametrize("name", sorted(NORM_MUTANTS))
def test_normalize_mutant_is_caught(name):
    mod = _mutant(normalize_ok, *NORM_MUTANTS[name], name)
    assert _run(npins, "normalize", mod, NORM_PINS), name
