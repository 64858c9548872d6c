"""The sum-product oracle's pins (tests/test_oracle_ctc_forward.py) must catch
plausible mistakes: each case plants one in a copy of oracle/viterbi.c's
forward function, builds it with gcc in a temporary directory and runs the
pins against it in a child process (a crash counts as caught)."""
import os
import subprocess
import sys
import tempfile

import pytest

if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "viterbi.c")

MUTANTS = {
    "no_skip": ("double a2 = skip_allowed(targets, blank, s) ? prev[s - 2] : -INFINITY;",
                "double a2 = -INFINITY;"),
    "skip_into_any_state": ("double a2 = skip_allowed(targets, blank, s) ? prev[s - 2] : -INFINITY;",
                            "double a2 = (s >= 2) ? prev[s - 2] : -INFINITY;"),
    "no_advance": ("double a1 = (s >= 1) ? prev[s - 1] : -INFINITY;", "double a1 = -INFINITY;"),
    "final_blank_only": ("*total = log_add3(prev[S - 1], (S > 1) ? prev[S - 2] : -INFINITY, -INFINITY);",
                         "*total = log_add3(prev[S - 1], -INFINITY, -INFINITY);"),
    "max_instead_of_sum": ("return m + log(exp(x - m) + exp(y - m) + exp(z - m));", "return m;"),
    "no_label_start": ("    if (S > 1) prev[1] = (double)lp[ext_of(targets, blank, 1)];\n    if (amax) amax[0]",
                       "    if (amax) amax[0]"),
}


def _battery() -> list[str]:
    import test_oracle_ctc_forward as pins
    failed = []
    for name, fn, args in [("enumeration", pins.test_equals_enumeration, [(s,) for s in range(12)]),
                           ("torch_ctc_loss", pins.test_equals_torch_ctc_loss, [()]),
                           ("closed_forms", pins.test_closed_forms, [()])]:
        for a in args:
            try:
                fn(*a)
            except AssertionError:
                failed.append(name)
                break
    return failed


def test_unmodified_oracle_passes():
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor: {name}"
    src = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "libmutant.so")
        with open(c, "w") as f:
            f.write(src)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", c, "-o", so, "-lm"])
        proc = subprocess.run([sys.executable, os.path.abspath(__file__), so],
                              capture_output=True, text=True, timeout=300)
    assert proc.returncode != 0, f"planted mistake {name} was not caught: {proc.stdout} {proc.stderr[-500:]}"


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    oracle._lib = oracle.load_variant(sys.argv[1])  # every oracle call of the pins uses the mutant
    failed_pins = _battery()
    print("failed pins:", sorted(set(failed_pins)))
    sys.exit(1 if failed_pins else 0)
