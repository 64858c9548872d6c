"""The autotuner times every candidate shape for a range of S, checks that all
candidates give the same alignment, and its table is applied by the planner."""
import pytest

from paper_2310_17864_gb300 import align, autotune, build

pytestmark = pytest.mark.gpu


def test_autotune_one_bucket_and_apply(tmp_path):
    build.build()
    res = autotune.tune(device=0, mode="latency", buckets=(600,), reps=1)
    (s_max, K, cw), = res["table"]
    assert s_max == 600 and K in autotune.KS and cw in autotune.CTA_WARPS
    assert len(res["trials"]) >= 10
    path = str(tmp_path / "t.json")
    autotune.save(res, path)
    assert autotune.load(path) == [(600, K, cw)]
    a = align.Aligner(device=0)
    try:
        assert autotune.apply(a, path)
    finally:
        a.close()
