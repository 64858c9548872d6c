"""The seeded input generators and the tuning-table file, on the CPU: shapes,
determinism and the structure each recipe states (planted paths, peaky
decoder rows, workload sizes), and the tuning-table round trip."""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2310_17864_gb300 import autotune, synth


def test_workload_specs_follow_their_recipes():
    (s1,) = synth.specs(1)
    assert (s1.T, s1.C, s1.L) == (200, 32, 40)
    s2 = synth.specs(2)
    assert len(s2) == 64 and all(500 <= s.T <= 3000 and s.L == round(s.T / 4) for s in s2)
    (s3,) = synth.specs(3)
    assert (s3.T, s3.L) == (180000, 45000)
    s4 = synth.specs(4, C=500)
    assert len(s4) == 4096 and all(50 <= s.T <= 30000 and s.C == 500 for s in s4)
    assert all(round(s.T / 5) <= s.L <= round(s.T / 3) for s in s4)
    med = float(np.median([s.T for s in s4]))
    assert 650 < med < 950  # lognormal with median 800
    assert [s.seed for s in synth.specs(4, C=32)] != [s.seed for s in s4]  # one stream per vocabulary
    assert synth.specs(2) == s2  # seeded


def test_planted_path_is_feasible_and_emissions_normalised():
    u = synth.make_utterance(123, 300, 32, 60, repeat_frac=0.3)
    lp = u.lp.numpy().astype(np.float64)
    assert np.allclose(np.exp(lp).sum(axis=1), 1.0, atol=1e-5)
    rng = np.random.default_rng(4)
    tg = synth.make_targets(rng, 50, 8, repeat_frac=0.5)
    path = synth.plant_state_path(rng, 50 + synth.count_repeats(tg) + 20, tg)
    assert path[0] in (0, 1) and path[-1] >= 2 * len(tg) - 1
    steps = np.diff(path)
    assert steps.min() >= 0 and steps.max() <= 2
    ext = synth.expand_tokens(tg)
    for t in np.nonzero(steps == 2)[0]:  # a skip only between different labels
        s = path[t + 1]
        assert s % 2 == 1 and ext[s] != ext[s - 2]


def test_decoder_probs_are_peaky_rows_of_a_planted_transcript():
    p = synth.decoder_probs(7, 600, 500)
    assert p.shape == (600, 500) and p.dtype == torch.float32
    assert torch.allclose(p.sum(dim=1), torch.ones(600), atol=1e-4)
    top = p.max(dim=1).values
    assert float((top > 0.5).float().mean()) > 0.9            # one token dominates nearly every frame
    assert float((p[:, 0] > 0.95).float().mean()) > 0.5       # mostly confident blanks
    assert torch.equal(p, synth.decoder_probs(7, 600, 500))   # seeded
    probs, off = synth.decoder_batch(3, 5, 40, t_lo=20, t_hi=60)
    assert off[0] == 0 and off[-1] == probs.shape[0] and len(off) == 6
    assert np.all(np.diff(off) >= 20) and np.all(np.diff(off) <= 60)


def test_arrivals_are_poisson():
    a = synth.arrivals(20000, 500.0, 9)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 500.0) < 0.05 / 500.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05     # exponential: cv = 1


def test_tuning_table_file_round_trip(tmp_path):
    path = os.path.join(tmp_path, "t.json")
    assert autotune.load(path) is None
    with open(path, "w") as f:
        json.dump({"gpu": "x", "latency": [[128, 2, 4], [1 << 30, 2, 2]]}, f)
    assert autotune.load(path, "latency") == [(128, 2, 4), (1 << 30, 2, 2)]
    assert autotune.load(path, "throughput") is None
    shipped = autotune.load(autotune.DEFAULT_TABLE, "latency")
    assert shipped and all(len(r) == 3 and r[1] in (2, 4, 8, 16) for r in shipped)
    assert [r[0] for r in shipped] == sorted(r[0] for r in shipped)


def test_autotune_choice_keeps_the_prior_shape_on_a_tie():
    """A bucket keeps its prior shape unless another is faster by more than the margin."""
    from paper_2310_17864_gb300 import autotune

    times = {(4, 2): 0.2638, (4, 4): 0.2659, (2, 4): 0.3171}
    assert autotune.choose(times) == (4, 2)
    assert autotune.choose(times, prior=(4, 4), margin=0.03) == (4, 4)
    assert autotune.choose(times, prior=(4, 4), margin=0.0) == (4, 2)
    assert autotune.choose(times, prior=(2, 4), margin=0.03) == (4, 2)   # 20 % slower: replaced
    assert autotune.choose(times, prior=(8, 1), margin=0.03) == (4, 2)   # prior not measured
    assert autotune.choose({(4, 4): 1.0, (2, 2): 1.0}) == (2, 2)        # exact tie: smaller shape
