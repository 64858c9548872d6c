"""CPU oracle for CTC forced alignment -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package. The product path (the CUDA
library and its binding) never imports, links or calls it, and it imports
nothing from the product package.

Contents:
  * ``viterbi.c``  -- plain C Viterbi over the CTC trellis, FP32 and FP64
    (paper Sec. 4, "CTC-based forced alignment"; trellis of the cited CTC work),
    and the sum-product forward score over the same trellis in FP64.
  * ``spans.py``   -- token spans of an alignment (start, end, mean score).
  * ``normalize.py`` -- per-frame log_softmax in FP64.
  * ``beam.py``    -- CTC prefix beam search with blank collapse (paper Sec. 5,
    CUDA CTC decoder), binary32 in a fixed operation order.
  * ``brute.py``   -- exhaustive enumeration of state paths for tiny inputs.
  * ``checks.py``  -- invariants: collapse, legal moves, fold sums, a max-plus
    backward pass, the FP32 summation error bound.

This module compiles ``viterbi.c`` with gcc into ``liboracle.so`` on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "viterbi.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Status codes of the oracle (same meaning as the library's public codes, but
# defined here independently).
OK = 0
E_INVAL = -1
E_TARGET = -2
E_INFEASIBLE = -3
E_NOPATH = -6
E_NOMEM = -10

# Default dense-backpointer limit: 2 GiB of host memory.
DEFAULT_MAX_BP_BYTES = 2 << 30


def build(force: bool = False, extra_flags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile viterbi.c into a shared library (plain IEEE arithmetic)."""
    out = out or _SO
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-fno-strict-aliasing", *extra_flags, _SRC, "-o", out + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    i32 = ctypes.c_int32
    lib.oracle_validate.argtypes = [p, i64, i64, i32, i64, p]
    lib.oracle_validate.restype = ctypes.c_int
    lib.oracle_viterbi_f32.argtypes = [p, i64, i64, p, i64, i32, i64, p, p, p, p]
    lib.oracle_viterbi_f32.restype = ctypes.c_int
    lib.oracle_viterbi_total_f32.argtypes = [p, i64, i64, p, i64, i32, p, p]
    lib.oracle_viterbi_total_f32.restype = ctypes.c_int
    lib.oracle_viterbi_f64.argtypes = [p, i64, i64, p, i64, i32, p, p, p, p]
    lib.oracle_viterbi_f64.restype = ctypes.c_int
    lib.oracle_ctc_forward_f64.argtypes = [p, i64, i64, p, i64, i32, p, p]
    lib.oracle_ctc_forward_f64.restype = ctypes.c_int
    return lib


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def load_variant(path: str) -> ctypes.CDLL:
    """Load an alternative build of the oracle (used to plant mistakes in tests)."""
    return _bind(ctypes.CDLL(path))


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(lp, targets):
    lp = np.ascontiguousarray(np.asarray(lp, dtype=np.float32))
    if lp.ndim != 2:
        raise ValueError("lp must be [T, C]")
    tg = np.ascontiguousarray(np.asarray(targets, dtype=np.int32).reshape(-1))
    return lp, tg


def validate(targets, C: int, blank: int, T: int, *, L=None) -> tuple[int, int]:
    tg = np.ascontiguousarray(np.asarray(targets, dtype=np.int32).reshape(-1))
    rep = ctypes.c_int64(0)
    rc = lib().oracle_validate(_ptr(tg), int(tg.size if L is None else L), int(C), int(blank), int(T),
                               ctypes.byref(rep))
    return rc, rep.value


def viterbi_f32(lp, targets, blank: int = 0, *, max_bp_bytes: int = DEFAULT_MAX_BP_BYTES,
                clib: ctypes.CDLL | None = None) -> dict:
    """FP32 Viterbi alignment. Returns status, path, states, scores, total."""
    lp, tg = _prep(lp, targets)
    T, C = lp.shape
    path = np.zeros(T, np.int32)
    states = np.zeros(T, np.int32)
    scores = np.zeros(T, np.float32)
    total = np.zeros(1, np.float32)
    rc = (clib or lib()).oracle_viterbi_f32(_ptr(lp), T, C, _ptr(tg), tg.size, int(blank),
                                            int(max_bp_bytes), _ptr(path), _ptr(states),
                                            _ptr(scores), _ptr(total))
    return {"status": rc, "path": path, "states": states, "scores": scores, "total": total[0]}


def viterbi_total_f32(lp, targets, blank: int = 0) -> dict:
    """Forward pass only (O(S) memory): best total and final state."""
    lp, tg = _prep(lp, targets)
    T, C = lp.shape
    total = np.zeros(1, np.float32)
    fin = np.zeros(1, np.int32)
    rc = lib().oracle_viterbi_total_f32(_ptr(lp), T, C, _ptr(tg), tg.size, int(blank),
                                        _ptr(total), _ptr(fin))
    return {"status": rc, "total": total[0], "final_state": int(fin[0])}


def viterbi_f64(lp, targets, blank: int = 0) -> dict:
    """The same recursion in binary64 on the FP32 emissions."""
    lp, tg = _prep(lp, targets)
    T, C = lp.shape
    path = np.zeros(T, np.int32)
    states = np.zeros(T, np.int32)
    scores = np.zeros(T, np.float64)
    total = np.zeros(1, np.float64)
    rc = lib().oracle_viterbi_f64(_ptr(lp), T, C, _ptr(tg), tg.size, int(blank), _ptr(path),
                                  _ptr(states), _ptr(scores), _ptr(total))
    return {"status": rc, "path": path, "states": states, "scores": scores, "total": total[0]}


def ctc_forward_f64(lp, targets, blank: int = 0, *, live_abs_max: bool = False) -> dict:
    """Sum-product over the same trellis (log-add in place of max), binary64:
    the log of the total probability of the transcript's CTC paths. With
    live_abs_max, also "amax": per frame the largest |beta_t(s)| over the
    finite states that can still reach a final state (for error bounds)."""
    lp, tg = _prep(lp, targets)
    T, C = lp.shape
    total = np.zeros(1, np.float64)
    amax = np.zeros(T, np.float64) if live_abs_max else None
    rc = lib().oracle_ctc_forward_f64(_ptr(lp), T, C, _ptr(tg), tg.size, int(blank), _ptr(total), _ptr(amax))
    out = {"status": rc, "total": float(total[0])}
    if live_abs_max:
        out["amax"] = amax
    return out
