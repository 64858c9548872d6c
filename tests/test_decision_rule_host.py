"""The paired blank / label decision of the fast kernel, checked exhaustively
against the definition on the host.

The Viterbi recursion over the CTC trellis (paper Sec. 4, "CTC-based forced
alignment"; trellis of the cited CTC work) takes, for a label state s, the
best of stay (alpha(s)), advance (alpha(s-1)) and skip (alpha(s-2), when the
label differs from the one two states back), with strict '>' in that order;
the blank state s-1 below it takes the better of stay (alpha(s-1)) and
advance (alpha(s-2)). The kernel decides both with one comparison
p > alpha(s-1), p = alpha(s-2), and records per frame one bit per state:
"advance won" for the blank state, "stay lost" for the label state; the
backtrack reads a label state's move as a skip when skipping is allowed and
the blank state below advanced at the same frame. This test enumerates every
ordering of the three values (ties and -inf included) and both skip
permissions, and checks moves, bits and values against the definition.
"""
import itertools
import math

VALUES = (-math.inf, -3.0, -2.0, -1.0, 0.0)
STAY, ADVANCE, SKIP = 0, 1, 2


def definition(p, a_blank, a_label, skip_ok):
    """Moves and pre-emission values of the blank and the label state."""
    blank_move = ADVANCE if p > a_blank else STAY
    blank_val = p if blank_move == ADVANCE else a_blank
    m, label_move = a_label, STAY
    if a_blank > m:
        m, label_move = a_blank, ADVANCE
    if skip_ok and p > m:
        m, label_move = p, SKIP
    return blank_move, blank_val, label_move, m


def paired(p, a_blank, a_label, skip_ok):
    """The kernel's rule: one comparison for the pair, one bit per state."""
    adv = p > a_blank
    mb = p if adv else a_blank
    mv = mb if skip_ok else a_blank
    moved = mv > a_label
    return adv, mb, moved, (mv if moved else a_label)


def decode_label(moved_bit, blank_adv_bit, skip_ok):
    """The backtrack's reading of a label state's bit."""
    if not moved_bit:
        return STAY
    return SKIP if (skip_ok and blank_adv_bit) else ADVANCE


def test_paired_rule_equals_definition_on_every_ordering():
    n = 0
    for p, ab, al in itertools.product(VALUES, repeat=3):
        for skip_ok in (False, True):
            bm, bv, lm, lv = definition(p, ab, al, skip_ok)
            adv, mb, moved, mv = paired(p, ab, al, skip_ok)
            assert (ADVANCE if adv else STAY) == bm, (p, ab, al, skip_ok)
            assert mb == bv, (p, ab, al, skip_ok)
            assert decode_label(moved, adv, skip_ok) == lm, (p, ab, al, skip_ok)
            assert mv == lv, (p, ab, al, skip_ok)
            n += 1
    assert n == 2 * len(VALUES) ** 3


def test_a_planted_mistake_in_the_rule_is_caught():
    """Reading the label's move as a skip without the permission check, or
    comparing with '>=', must disagree with the definition somewhere."""
    bad_perm = bad_tie = False
    for p, ab, al in itertools.product(VALUES, repeat=3):
        for skip_ok in (False, True):
            _, _, lm, _ = definition(p, ab, al, skip_ok)
            adv, _, moved, _ = paired(p, ab, al, skip_ok)
            if moved and (SKIP if adv else ADVANCE) != lm:
                bad_perm = True
            mv = (p if p >= ab else ab) if skip_ok else ab
            if (mv >= al) != (lm != STAY):
                bad_tie = True
    assert bad_perm and bad_tie
