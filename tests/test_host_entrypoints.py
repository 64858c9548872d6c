"""Host-side argument checks of the row entry points (no GPU needed: every
case below is rejected, or finishes, before any CUDA call)."""
import pytest

from paper_2310_17864_gb300 import align, build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    align.lib()


def test_beam_workspace_bytes():
    f = align.align_ctc_beam_workspace_bytes
    assert f(-1, 10, 4) == 0 and f(1, -1, 4) == 0 and f(1, 10, 0) == 0
    a, b = f(4, 1000, 10), f(4, 2000, 10)
    assert a > 0 and b > a
    # kept list (4 B / frame), three node arrays (4 B per node, beam nodes per frame + a
    # root per utterance) and the ranked labels (4 B per frame and beam slot), each
    # rounded up to 256 B
    r = lambda x: (x + 255) // 256 * 256
    assert a == r(4 * 1000) + 3 * r(4 * (1000 * 10 + 4)) + r(4 * 1000 * 10)
    assert f(4, 1000, 16) > a


@pytest.mark.parametrize("kw", [
    {"n": -1}, {"total_frames": -1}, {"V": 1}, {"blank": -1}, {"blank": 7}, {"beam": 0}, {"beam": 17},
    {"threshold": float("nan")}, {"threshold": -0.5},
])
def test_beam_decode_rejects_bad_arguments(kw):
    args = dict(probs=1, frame_offsets=1, n=1, total_frames=4, V=7, blank=0, beam=4, threshold=0.95,
                workspace=1, workspace_bytes=1 << 20, tokens=1, timesteps=1, lengths=1, totals=1,
                scale_exp=1, scores=1, kept=1, stream_ptr=None)
    args.update(kw)
    with pytest.raises(align.AlignError) as e:
        align.align_ctc_beam_decode(*args.values())
    assert e.value.code == align.ALIGN_E_INVAL


def test_beam_decode_checks_pointers_and_workspace():
    base = dict(probs=1, frame_offsets=1, n=2, total_frames=8, V=5, blank=0, beam=3, threshold=1.0,
                workspace=1, workspace_bytes=1 << 20, tokens=1, timesteps=1, lengths=1, totals=1,
                scale_exp=1, scores=1, kept=1, stream_ptr=None)
    for name in ("probs", "frame_offsets", "workspace", "tokens", "timesteps", "lengths", "totals", "scale_exp",
                 "scores", "kept"):
        a = dict(base, **{name: None})
        with pytest.raises(align.AlignError) as e:
            align.align_ctc_beam_decode(*a.values())
        assert e.value.code == align.ALIGN_E_INVAL, name
    a = dict(base, workspace_bytes=align.align_ctc_beam_workspace_bytes(2, 8, 3) - 1)
    with pytest.raises(align.AlignError) as e:
        align.align_ctc_beam_decode(*a.values())
    assert e.value.code == align.ALIGN_E_INVAL
    # an empty batch is done without touching the device
    align.align_ctc_beam_decode(*dict(base, n=0, total_frames=0).values())


def test_token_spans_argument_checks():
    with pytest.raises(align.AlignError) as e:
        align.align_token_spans(1, 1, 1, 1, -1, 0, 0, 1, 1, 1)
    assert e.value.code == align.ALIGN_E_INVAL
    with pytest.raises(align.AlignError) as e:
        align.align_token_spans(None, 1, 1, 1, 2, 10, 3, 1, 1, 1)
    assert e.value.code == align.ALIGN_E_INVAL
    align.align_token_spans(None, None, None, None, 0, 0, 0, None, None, None)  # nothing to do
