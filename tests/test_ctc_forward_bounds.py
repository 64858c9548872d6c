"""Host checks of the sum-product error bound and closed form used by the GPU
parity tests (tests/test_gpu_ctc_forward.py): the closed form is pinned to
exhaustive enumeration and to the binary64 oracle, and the bound is shown to
be tight enough to catch the plausible kernel mistakes named below."""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2310_17864_gb300 import synth

import ctc_forward_bounds as cfb


@pytest.mark.parametrize("L,T", [(1, 1), (1, 3), (2, 2), (2, 5), (3, 6), (4, 7)])
def test_path_counts_equal_enumeration(L, T):
    tg = list(1 + np.arange(L) % 3)
    S = 2 * L + 1
    paths = brute.enumerate_paths(T, tg, 0)
    n_b = sum(1 for p in paths if p[-1] == S - 1)
    n_l = sum(1 for p in paths if p[-1] == S - 2)
    assert cfb.path_counts(L, T) == (n_b, n_l)


def test_closed_form_equals_oracle():
    lp, tg, exact, _ = cfb.closed_form_case(300, 12)
    o = oracle.ctc_forward_f64(lp, tg, 0)
    assert o["status"] == 0
    assert abs(o["total"] - exact) <= 1e-9 * (1.0 + abs(exact)), (o["total"], exact)


@pytest.mark.parametrize("L,spare", [(2980, 20), (10000, 20)])
def test_closed_form_bound_catches_final_state_and_last_emission_mistakes(L, spare):
    """On the closed forms the GPU tests run (a cluster team and a grid team),
    a kernel that drops either final state from the last log-add, or the last
    frame's emission, is off by more than the bound."""
    lp, tg, exact, tol = cfb.closed_form_case(L, spare)
    n_b, n_l = cfb.path_counts(L, L + spare)
    vl = float(lp[-1, tg[-1]])
    only_blank = math.log(n_b)                 # vb = 0
    only_label = math.log(n_l) + vl
    no_last_emission = math.log(n_b + n_l)
    for wrong in (only_blank, only_label, no_last_emission):
        assert abs(wrong - exact) > 2 * tol, (wrong, exact, tol)
    assert tol < 0.25


def test_realistic_bound_catches_dropped_last_emission():
    """The GPU test's T = 3000, C = 32, L = 1023 case: dropping the last
    frame's emission moves the total by more than the bound. (Dropping one
    final state moves it by 0.5-1 nat here, below what any rigorous FP32 bound
    allows at |total| ~ 8000; the closed forms above catch that mistake.)"""
    T, C, L = 3000, 32, 1023
    u = synth.make_utterance(T * 37 + L, T, C, L, repeat_frac=0.1)
    lp = u.lp.numpy()
    o = oracle.ctc_forward_f64(lp, u.targets, 0, live_abs_max=True)
    tol = cfb.tolerance(lp, o["amax"], o["total"])
    lp2 = lp.copy()
    lp2[-1, :] = 0.0
    wrong = oracle.ctc_forward_f64(lp2, u.targets, 0)["total"]
    assert abs(wrong - o["total"]) > tol, (wrong, o["total"], tol)
    assert tol < 3.0
