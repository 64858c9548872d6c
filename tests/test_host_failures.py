"""Failure paths that need no GPU fault: NULL handles and arguments are
rejected before any CUDA call, and a CUDA runtime failure (here: no usable
GPU in this process) comes back as ALIGN_E_CUDA with its text, without a
crash."""
import ctypes

import pytest
import torch

from paper_2310_17864_gb300 import align, build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    align.lib()


def test_null_handles_are_rejected():
    L = align.lib()
    out = align.AlignOut(None, None, None, None)
    rid = ctypes.c_uint64(0)
    assert L.align_destroy(None) == align.ALIGN_OK                       # destroy(NULL) is a no-op
    assert L.align_flush(None) == align.ALIGN_E_INVAL
    assert L.align_join(None, None) == align.ALIGN_E_INVAL
    assert L.align_get_stats(None, None, 0) == align.ALIGN_E_INVAL
    assert L.align_set_tuning(None, 2, 2, 2) == align.ALIGN_E_INVAL
    assert L.align_poll(None, 1, 0, None) == align.ALIGN_E_INVAL
    assert L.align_poll_done(None, None, None, 0, None) == align.ALIGN_E_INVAL
    assert L.align_submit(None, None, 10, 4, None, 0, 0, out, ctypes.byref(rid)) == align.ALIGN_E_INVAL
    assert L.align_submit_host(None, None, 10, 4, None, 0, 0, out, ctypes.byref(rid)) == align.ALIGN_E_INVAL
    assert L.align_forced_noalloc(None, 10, 4, None, 0, 0, out, None, None) == align.ALIGN_E_INVAL
    assert L.align_create(None, None) == align.ALIGN_E_INVAL


@pytest.mark.skipif(torch.cuda.is_available(), reason="needs a process without a usable GPU")
def test_cuda_failure_is_reported_not_fatal():
    with pytest.raises(align.AlignError) as e:
        align.align_create(align.AlignConfig(device=0))
    assert e.value.code == align.ALIGN_E_CUDA
    assert align.last_error()  # the CUDA runtime's own message
    with pytest.raises(align.AlignError) as e:  # and again: the library state is unharmed
        align.align_create(align.AlignConfig(device=0))
    assert e.value.code == align.ALIGN_E_CUDA
