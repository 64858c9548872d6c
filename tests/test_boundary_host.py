"""Host-side tests of the C ABI (no GPU): the library loads, exports every entry
point declared in include/align.h, and its validation and planning logic
behave as documented."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2310_17864_gb300 import align, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "align.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(align_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol():
    names = declared_entry_points()
    assert len(names) >= 12
    L = align.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(align.EXPORTS)


def test_status_strings():
    for code in range(-11, 2):
        s = align.status_string(code)
        assert s.startswith("ALIGN_") and s != "ALIGN_E_UNKNOWN", code
    assert align.status_string(-6) == "ALIGN_E_NOPATH"
    assert align.status_string(align.ALIGN_E_NONFINITE) == "ALIGN_E_NONFINITE"


def test_header_constants_match_binding():
    """Every ALIGN_E_* / ALIGN_F_* / ALIGN_REQ_* value in include/align.h has
    the same value in the binding."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "align.h")).read()
    found = 0
    for name, val in re.findall(r"#define (ALIGN_(?:E|F|REQ)_[A-Z_]+) \(?(-?0x[0-9a-fA-F]+|-?\d+)u?\)?", hdr):
        v = int(val, 16) if "0x" in val.lower() else int(val)
        assert getattr(align, name) == v, name
        found += 1
    assert found >= 18


def test_validate_agrees_with_oracle():
    """Two independent implementations of step A1 agree on random inputs."""
    rng = np.random.default_rng(0)
    for _ in range(3000):
        C = int(rng.integers(1, 6))
        L = int(rng.integers(0, 6))
        T = int(rng.integers(0, 10))
        blank = int(rng.integers(-1, 6))
        tg = rng.integers(-1, 6, size=L).astype(np.int32)
        a = align.align_validate(tg, C, blank, T)
        o = oracle.validate(tg, C, blank, T)
        assert a[0] == o[0], (tg, C, blank, T)
        if a[0] == 0:
            assert a[1] == o[1]


def test_plan_shapes_and_footprints():
    # Config-1 sized: S = 81 fits one warp of K=4 lanes.
    p = align.align_plan(200, 32, 40)
    assert (p["states_per_lane"], p["warps_per_cta"], p["cluster_ctas"]) == (4, 1, 1)
    # 199 frames = 7 windows of 32 frames x 6 words (5376 B), plus 7 anchor rows of 96 B
    # (S=81 -> 96) padded to 256 B.
    assert p["backpointer_bytes"] == 5376 + 768
    assert p["checkpointed"] == 0
    # S = 1501: 12 warps of 128 states; by default 4 warps per CTA, a cluster of 3.
    p = align.align_plan(3000, 32, 750)
    assert p["warps_per_cta"] == 4 and p["cluster_ctas"] == 3
    p = align.align_plan(3000, 32, 750, cta_warps=16)
    assert p["warps_per_cta"] == 12 and p["cluster_ctas"] == 1
    # Hour-long: S = 90001 needs a cluster.
    p = align.align_plan(180000, 32, 45000, budget=8 << 30)
    assert p["cluster_ctas"] > 1
    assert p["states_per_lane"] * 32 * p["warps_per_cta"] * p["cluster_ctas"] >= 90001
    assert p["checkpointed"] == 0
    # Small budget: checkpointed, footprint ~ sqrt(T) rows.
    q = align.align_plan(180000, 32, 45000, budget=1 << 30)
    assert q["checkpointed"] == 1
    # Segments of whole 32-frame anchor windows, at least sqrt(T) frames and about
    # twice the team's pipeline fill (a 32-frame window per warp boundary):
    # 11 CTAs x 16 warps -> 175 boundaries -> 2 x 5600 frames.
    warps = q["warps_per_cta"] * q["cluster_ctas"]
    assert q["checkpoint_every"] % 32 == 0 and q["checkpoint_every"] >= np.sqrt(180000)
    assert q["checkpoint_every"] == 2 * 32 * (warps - 1)
    assert q["checkpoints"] == (180000 - 1) // q["checkpoint_every"] + 1
    assert q["checkpoint_bytes"] < (1 << 30) < q["backpointer_bytes"]
    # Forced checkpointing.
    assert align.align_plan(500, 32, 100, flags=align.ALIGN_F_FORCE_CHECKPOINT)["checkpointed"] == 1
    # A budget too small for such segments gets shorter ones (down to sqrt(T)).
    small = align.align_plan(180000, 32, 45000, budget=q["checkpoint_bytes"] // 2)
    assert small["checkpointed"] == 1 and small["checkpoint_every"] < q["checkpoint_every"]
    assert small["checkpoint_every"] >= np.sqrt(180000)
    # Nothing fits.
    with pytest.raises(align.AlignError) as e:
        align.align_plan(180000, 32, 45000, budget=1 << 20)
    assert e.value.code == align.ALIGN_E_TOO_LARGE
    # Stage depth: 32 rows of C=32, fewer rows of C=500 (8 KB stages for the fast
    # kernel's shapes, K = 2 or 4 and C <= 512; else 4 KB for one-warp CTAs).
    assert align.align_plan(100, 32, 10)["frames_per_stage"] == 32       # 4 KB of rows
    assert align.align_plan(3000, 32, 750)["frames_per_stage"] == 32     # 12 warps
    assert align.align_plan(3000, 500, 750)["frames_per_stage"] == 4     # 8 KB cap
    assert align.align_plan(100, 500, 10)["frames_per_stage"] == 4       # 8 KB stages of 2 KB rows
    assert align.align_plan(100, 600, 10)["frames_per_stage"] == 1       # generic kernel: 4 KB of 2.4 KB rows
    # Rows per stage are a power of two dividing the 32-frame anchor window.
    assert align.align_plan(3000, 96, 750)["frames_per_stage"] == 16     # 8 KB / 384 B = 21 -> 16
    assert align.align_plan(100, 96, 10)["frames_per_stage"] == 16       # 8 KB / 384 B = 21 -> 16


@pytest.mark.parametrize("K", [2, 4, 8, 16])
def test_plan_capacity_covers_states(K):
    rng = np.random.default_rng(K)
    for _ in range(200):
        L = int(rng.integers(0, 60000))
        try:
            p = align.align_plan(2 * L + 10, 32, L, budget=64 << 30, states_per_lane=K)
        except align.AlignError as e:
            assert e.code == align.ALIGN_E_TOO_LARGE
            continue
        cap = p["states_per_lane"] * 32 * p["warps_per_cta"] * p["cluster_ctas"]
        assert cap >= 2 * L + 1
        assert p["cluster_ctas"] <= 16 and p["warps_per_cta"] <= 16
        # No empty warp group: the last warp holds at least one state.
        assert cap - 2 * L - 1 < p["states_per_lane"] * 32 * p["cluster_ctas"]


def test_product_has_no_cpu_fallback(monkeypatch):
    """The binding refuses to run without the CUDA library."""
    monkeypatch.setattr(align, "_lib", None)
    monkeypatch.setattr(align, "LIB_PATH", "/nonexistent/libalign.so")
    with pytest.raises(ImportError):
        align.lib()


def test_request_row_layout_matches_abi():
    """The numpy row layout used to build whole batches equals align_request."""
    import ctypes
    assert align._REQ_DTYPE.itemsize == ctypes.sizeof(align.AlignRequest)
    out_off = align.AlignRequest.out.offset
    want = {"lp": align.AlignRequest.log_probs.offset, "T": align.AlignRequest.T.offset,
            "C": align.AlignRequest.C.offset, "tg": align.AlignRequest.targets.offset,
            "L": align.AlignRequest.L.offset, "blank": align.AlignRequest.blank.offset,
            "flags": align.AlignRequest.flags.offset, "path": out_off + align.AlignOut.path.offset,
            "scores": out_off + align.AlignOut.scores.offset, "total": out_off + align.AlignOut.total.offset,
            "states": out_off + align.AlignOut.states.offset}
    assert {k: align._REQ_DTYPE.fields[k][1] for k in want} == want
