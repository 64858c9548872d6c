"""The autotuner times every candidate shape for a range of S, checks that all
candidates give the same alignment, and its table is applied by the planner."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_17864_gb300 import align, autotune, build, synth

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
    assert autotune.load(path, "throughput") is None
    a = align.Aligner(device=0)
    try:
        assert autotune.apply(a, path)
    finally:
        a.close()


def _batch_outputs(al, b, n):
    outs = [(torch.empty(b.utt(i).shape[0], dtype=torch.int32, device="cuda:0"),
             torch.empty(b.utt(i).shape[0], device="cuda:0"), torch.empty(1, device="cuda:0"), None)
            for i in range(n)]
    rs = al.submit_batch([(b.utt(i), b.targets[i], 0, outs[i]) for i in range(n)])
    al.flush()
    for r in rs:
        al.poll(r)
        assert r.status == 0
    return outs


@pytest.mark.parametrize("K,cw", [(4, 4), (2, 1)])
def test_throughput_table_for_oversubscribed_batches(K, cw):
    """A batch whose work exceeds what the GPU runs at once is planned with
    the throughput table, a small one with the latency table; both give the
    oracle's alignment."""
    build.build()
    specs = [synth.Spec(300, 32, 200, 0.1, synth.sub_seed(4242, i)) for i in range(400)]
    b = synth.make_batch(specs, device="cuda:0")
    both = align.Aligner(device=0, batched=True, bp_budget_bytes=4 << 30)
    lat = align.Aligner(device=0, batched=True, bp_budget_bytes=4 << 30)
    try:
        for a in (both, lat):
            a.set_tuning_table([(1 << 20, 2, 1)], "latency")
        both.set_tuning_table([(1 << 20, K, cw)], "throughput")
        small = _batch_outputs(both, b, 2)
        assert both.stats()["throughput_batches"] == 0
        big = _batch_outputs(both, b, 400)
        assert both.stats()["throughput_batches"] == 1
        ref = _batch_outputs(lat, b, 400)
        assert lat.stats()["throughput_batches"] == 0
        for x, y in zip(big, ref):
            assert torch.equal(x[0], y[0]) and torch.equal(x[1].view(torch.int32), y[1].view(torch.int32))
        for i in (0, 1, 399):
            o = oracle.viterbi_f32(b.utt(i).cpu().numpy(), np.asarray(b.targets[i], np.int32), 0)
            assert np.array_equal(big[i][0].cpu().numpy(), o["path"])
            if i < 2:
                assert np.array_equal(small[i][0].cpu().numpy(), o["path"])
    finally:
        both.close()
        lat.close()
