"""The allocation-free entry point (align_forced_noalloc) against the normal one.

align_forced_noalloc serves callers that cannot allocate device memory when
they need an alignment (for example a real-time thread, or a host with a fixed
device-memory budget): all its scratch lives in a fixed array inside the
library. This file is collected last so that, if it fails, a run that stops at
the first failure has already run every other test; it also passes alone.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_17864_gb300 import align, build, synth

pytestmark = pytest.mark.gpu


def _outs(T):
    return (torch.empty(T, dtype=torch.int32, device="cuda"), torch.empty(T, dtype=torch.float32, device="cuda"),
            torch.empty(1, dtype=torch.float32, device="cuda"), torch.empty(T, dtype=torch.int32, device="cuda"))


def _noalloc(u, stream):
    path, scores, total, states = _outs(u.T)
    lp = u.lp.cuda()
    torch.cuda.synchronize()
    o = align.AlignOut(path.data_ptr(), scores.data_ptr(), total.data_ptr(), states.data_ptr())
    rc, st = align.align_forced_noalloc(lp.data_ptr(), u.T, u.C, u.targets, 0, o, stream.cuda_stream)
    assert rc == align.ALIGN_OK, align.align_noalloc_last_error()
    return st, path, scores, total, states


def test_noalloc_matches_submit_two_calls_in_a_row():
    build.build()
    (s1,) = synth.specs(1)
    u1 = synth.make_utterance(s1.seed, s1.T, s1.C, s1.L, s1.repeat_frac)   # one warp
    u2 = synth.make_utterance(77, 2400, 32, 600)                           # a 3-CTA cluster team
    ref = align.Aligner(device=0)
    stream = torch.cuda.Stream()
    try:
        for u in (u1, u2, u1):   # consecutive calls share and reuse the scratch array
            r = ref.align(u.lp.cuda(), u.targets, 0, want_states=True)
            st, path, scores, total, states = _noalloc(u, stream)
            assert st == r.status == align.ALIGN_OK
            # Same kernel arithmetic: tolerance zero.
            assert torch.equal(path, r.path) and torch.equal(states, r.states)
            assert scores.cpu().numpy().tobytes() == r.scores.cpu().numpy().tobytes()
            assert total.cpu().numpy().tobytes() == r.total.cpu().numpy().tobytes()
            # And the CPU oracle's alignment, bit for bit.
            o = oracle.viterbi_f32(u.lp.numpy(), u.targets, 0)
            assert o["status"] == 0
            assert np.array_equal(path.cpu().numpy(), o["path"]) and np.array_equal(states.cpu().numpy(), o["states"])
            assert scores.cpu().numpy().tobytes() == o["scores"].tobytes()
            assert total.cpu().numpy().tobytes() == np.float32(o["total"]).tobytes()
    finally:
        ref.close()


def test_noalloc_rejects_host_buffers():
    """Emissions or outputs in host memory are refused with ALIGN_E_INVAL and a
    message before anything runs on the GPU."""
    build.build()
    u = synth.make_utterance(6, 100, 32, 20)
    path, scores, total, states = _outs(u.T)
    o = align.AlignOut(path.data_ptr(), scores.data_ptr(), total.data_ptr(), states.data_ptr())
    lp_host = u.lp.contiguous()
    rc, _ = align.align_forced_noalloc(lp_host.data_ptr(), u.T, u.C, u.targets, 0, o, None)
    assert rc == align.ALIGN_E_INVAL
    assert "device memory" in align.align_noalloc_last_error()
    host_path = torch.empty(u.T, dtype=torch.int32)
    o2 = align.AlignOut(host_path.data_ptr(), scores.data_ptr(), total.data_ptr(), states.data_ptr())
    rc, _ = align.align_forced_noalloc(u.lp.cuda().data_ptr(), u.T, u.C, u.targets, 0, o2, None)
    assert rc == align.ALIGN_E_INVAL


def test_noalloc_rejects_requests_beyond_its_scratch():
    build.build()
    u = synth.make_utterance(5, 60000, 32, 15000)
    path, scores, total, states = _outs(u.T)
    o = align.AlignOut(path.data_ptr(), scores.data_ptr(), total.data_ptr(), states.data_ptr())
    lp = u.lp.cuda()
    rc, _ = align.align_forced_noalloc(lp.data_ptr(), u.T, u.C, u.targets, 0, o, None)
    assert rc == align.ALIGN_E_TOO_LARGE
    assert "scratch" in align.align_noalloc_last_error()


def test_noalloc_refuses_a_capturing_stream():
    """The call copies from host memory and synchronises its stream, so on a
    stream under capture it returns ALIGN_E_INVAL with a message and records
    nothing."""
    build.build()
    u = synth.make_utterance(7, 100, 32, 20)
    path, scores, total, states = _outs(u.T)
    lp = u.lp.cuda()
    o = align.AlignOut(path.data_ptr(), scores.data_ptr(), total.data_ptr(), states.data_ptr())
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        rc, _ = align.align_forced_noalloc(lp.data_ptr(), u.T, u.C, u.targets, 0, o, s.cuda_stream)
    assert rc == align.ALIGN_E_INVAL
    assert "captured" in align.align_noalloc_last_error()
