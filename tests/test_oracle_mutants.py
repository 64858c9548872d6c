"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU, in a
temporary directory), builds it, and runs the pin battery against it: at
least one pin must fail. This shows the pins are strong enough to trust the
unmodified oracle.
"""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle
from oracle import brute, checks
from paper_2310_17864_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "viterbi.c")

MUTANTS = {
    "advance_wins_ties": ("prev[s - 1] > best", "prev[s - 1] >= best"),
    "skip_wins_ties": ("prev[s - 2] > best", "prev[s - 2] >= best"),
    "skip_ignores_labels": ("return ext_of(targets, blank, s) != ext_of(targets, blank, s - 2);", "return 1;"),
    "final_tie_to_label": ("(alpha[S - 2] > alpha[S - 1]) ? S - 2 : S - 1", "(alpha[S - 2] >= alpha[S - 1]) ? S - 2 : S - 1"),
    "no_label_start": ("if (S > 1) alpha[1] = lp_row0[ext_of(targets, blank, 1)];", ""),
    "feasibility_ignores_repeats": ("if (T < L + R) return OR_E_INFEASIBLE;", "if (T < L) return OR_E_INFEASIBLE;"),
    "emission_of_previous_state": ("cur[s] = best + lp_row[ext_of(targets, blank, s)];",
                                   "cur[s] = best + lp_row[ext_of(targets, blank, s > 0 ? s - 1 : s)];"),
    "score_of_blank": ("scores[t] = lp[t * C + tok];", "scores[t] = lp[t * C + blank];"),
    "backpointer_row_off_by_one": ("if (t > 0) s_cur -= bp[t * S + s_cur];", "if (t > 0) s_cur -= bp[(t - 1) * S + s_cur];"),
    "no_stay": ("float best = prev[s];\n        uint8_t code = 0;", "float best = -INFINITY;\n        uint8_t code = 0;"),
}


def _battery(clib) -> list[str]:
    """Run the pins against a given build; return the names of failed pins."""
    failed = []
    rng = np.random.default_rng(21)
    # brute force, random floats and integer ties
    for kind in ("float", "int"):
        for _ in range(150):
            C = int(rng.integers(2, 5))
            L = int(rng.integers(0, 4))
            T = int(rng.integers(1, 8))
            blank = int(rng.integers(0, C))
            labels = [c for c in range(C) if c != blank]
            tg = rng.choice(labels, size=L).astype(np.int32) if L else np.zeros(0, np.int32)
            lp = (rng.standard_normal((T, C)) if kind == "float" else -rng.integers(0, 4, (T, C))).astype(np.float32)
            r = oracle.viterbi_f32(lp, tg, blank, clib=clib)
            b = brute.brute_force(lp, tg, blank)
            if b["n_paths"] == 0:
                if r["status"] != oracle.E_INFEASIBLE:
                    failed.append("brute_infeasible")
                continue
            if r["status"] != 0 or r["total"] != b["best"]:
                failed.append("brute_total")
                continue
            ok_path = tuple(r["states"].tolist()) == b["chosen"] if kind == "int" else \
                (len(b["optimal"]) > 1 or tuple(r["states"].tolist()) == b["optimal"][0])
            if not ok_path:
                failed.append("brute_path")
            if not (r["scores"] == lp[np.arange(T), r["path"]]).all():
                failed.append("scores_gather")
    # invariants on a synthetic utterance
    u = synth.make_utterance(5, 150, 16, 40, repeat_frac=0.2)
    lp = u.lp.numpy()
    r = oracle.viterbi_f32(lp, u.targets, 0, clib=clib)
    if r["status"] != 0 or checks.collapse(r["path"], 0) != u.targets.tolist() \
            or not checks.legal_state_path(r["states"], u.targets, 0) \
            or checks.fold_f32(r["scores"]) != r["total"]:
        failed.append("invariants")
    return failed


def test_unmodified_oracle_passes_battery():
    assert _battery(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    with open(SRC) as f:
        src = f.read()
    assert old in src, f"mutation anchor missing: {old!r}"
    src = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "libmutant.so")
        with open(c, "w") as f:
            f.write(src)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", c, "-o", so, "-lm"])
        # A child process runs the battery, so a mutant that walks out of
        # bounds and crashes counts as caught instead of ending the test run.
        proc = subprocess.run([sys.executable, os.path.abspath(__file__), so],
                              capture_output=True, text=True, timeout=300)
    assert proc.returncode != 0, f"planted mistake {name} was not caught by any pin"


if __name__ == "__main__":
    failed_pins = _battery(oracle.load_variant(sys.argv[1]))
    print("failed pins:", sorted(set(failed_pins)))
    sys.exit(1 if failed_pins else 0)
