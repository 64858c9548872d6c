"""Continuous batching: requests arriving while others run are admitted as
backpointer memory frees up, overlap on the GPU, and every result is the same
alone and in the mix (bit for bit)."""
import numpy as np
import pytest
import torch

from paper_2310_17864_gb300 import align, build, serve, synth

pytestmark = pytest.mark.gpu


def test_serving_mix_equals_alone():
    build.build()
    specs = synth.specs(5, n=160)
    b = synth.make_batch(specs, device="cuda")
    alone = align.Aligner(device=0)
    ref = []
    try:
        for i in range(len(b)):
            r = alone.align(b.utt(i), b.targets[i], 0, want_states=True)
            ref.append((r.path.clone(), r.scores.clone(), r.total.clone(), r.states.clone(), r.status))
    finally:
        alone.close()
    # A budget that holds only a few of the largest requests at once, so
    # admission has to wait for memory released by finished batches.
    big = max(align.align_plan(s.T, s.C, s.L)["backpointer_bytes"] for s in specs)
    srv = align.Aligner(device=0, batched=True, bp_budget_bytes=4 * big)
    try:
        reqs = serve.poisson_requests(b, rate_per_s=20000.0, seed=11)
        for r in reqs:
            T = int(r.log_probs.shape[0])
            r.out = (torch.empty(T, dtype=torch.int32, device="cuda"), torch.empty(T, device="cuda"),
                     torch.empty(1, device="cuda"), torch.empty(T, dtype=torch.int32, device="cuda"))
        st = serve.serve(srv, reqs)
        stats = srv.stats()
    finally:
        srv.close()
    assert st.n == len(b)
    for i, r in enumerate(reqs):
        p, s, t, states, status = ref[i]
        assert r.result.status == status == 0
        assert torch.equal(r.out[0], p) and torch.equal(r.out[3], states), i
        assert r.out[1].cpu().numpy().tobytes() == s.cpu().numpy().tobytes(), i
        assert r.out[2].cpu().numpy().tobytes() == t.cpu().numpy().tobytes(), i
    # Work overlapped: several requests in flight at once, several batches launched.
    assert st.max_inflight > 1
    assert stats["kernel_launches"] > 1
    assert np.all(st.latency_ms > 0)
