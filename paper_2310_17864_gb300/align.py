"""Thin ctypes binding of libalign.so (C ABI in include/align.h).

The functions named like the C entry points (``align_create``, ``align_submit``,
``align_poll`` ...) only marshal arguments; every step of the alignment runs in
the CUDA library. There is no CPU fallback: if libalign.so is missing or cannot
be loaded, ``lib()`` raises.

``Aligner`` is a convenience wrapper that owns a context and output tensors
(PyTorch is used only for device memory and streams).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libalign.so")

ALIGN_OK = 0
ALIGN_PENDING = 1
ALIGN_E_INVAL = -1
ALIGN_E_TARGET = -2
ALIGN_E_INFEASIBLE = -3
ALIGN_E_TOO_LARGE = -4
ALIGN_E_AGAIN = -5
ALIGN_E_NOPATH = -6
ALIGN_E_TIMEOUT = -7
ALIGN_E_CUDA = -8
ALIGN_E_NOTFOUND = -9
ALIGN_E_NOMEM = -10
ALIGN_E_NONFINITE = -11

ALIGN_F_BATCHED = 0x1
ALIGN_F_FORCE_CHECKPOINT = 0x2
ALIGN_F_NO_GRAPHS = 0x4
ALIGN_F_NO_GRID_TEAMS = 0x8
ALIGN_F_DEBUG_CHECKS = 0x10
ALIGN_F_GENERIC_KERNEL = 0x20
ALIGN_F_PERSISTENT = 0x40
ALIGN_F_UPLOAD_DESCRIPTORS = 0x80
ALIGN_F_TEST_STALL = 0x80000000

# Every entry point declared in include/align.h.
EXPORTS = ("align_create", "align_destroy", "align_submit", "align_submit_host", "align_submit_batch", "align_flush",
           "align_poll", "align_poll_done", "align_join", "align_get_stats", "align_status_string", "align_last_error",
           "align_set_tuning", "align_set_tuning_bucket", "align_set_tuning_bucket_for", "align_validate", "align_plan", "align_probe_frame_latency",
           "align_forced_noalloc", "align_noalloc_last_error", "align_token_spans",
           "align_ctc_beam_workspace_bytes", "align_ctc_beam_decode")


class AlignConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("bp_budget_bytes", ctypes.c_uint64), ("staging_bytes", ctypes.c_uint64),
                ("cuda_stream", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("wait_limit_ms", ctypes.c_uint32)]


class AlignOut(ctypes.Structure):
    _fields_ = [("path", ctypes.c_void_p), ("scores", ctypes.c_void_p), ("total", ctypes.c_void_p),
                ("states", ctypes.c_void_p)]


ALIGN_REQ_HOST = 0x1
ALIGN_REQ_LOGITS = 0x2   # log_probs holds raw logits: log_softmax is applied inside the kernel
ALIGN_REQ_SUM = 0x4      # sum-product forward score (total only) instead of the Viterbi alignment


class AlignRequest(ctypes.Structure):
    _fields_ = [("log_probs", ctypes.c_void_p), ("T", ctypes.c_int64), ("C", ctypes.c_int64),
                ("targets", ctypes.c_void_p), ("L", ctypes.c_int64), ("blank", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("out", AlignOut)]


class AlignStats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("requests_done", ctypes.c_uint64), ("cells", ctypes.c_uint64),
                ("checkpointed", ctypes.c_uint64), ("bp_bytes_peak", ctypes.c_uint64),
                ("throughput_batches", ctypes.c_uint64), ("grid_teams", ctypes.c_uint64),
                ("sum_requests", ctypes.c_uint64), ("persistent_batches", ctypes.c_uint64)]


class AlignPlanInfo(ctypes.Structure):
    _fields_ = [("states_per_lane", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("cluster_ctas", ctypes.c_int32), ("frames_per_stage", ctypes.c_int32),
                ("checkpointed", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("checkpoints", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("backpointer_bytes", ctypes.c_uint64), ("checkpoint_bytes", ctypes.c_uint64)]


class AlignError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = status_string(code)
        if code == ALIGN_E_CUDA:
            msg += ": " + last_error()
        super().__init__(f"{what}: {msg}" if what else msg)


_lib = None


def lib() -> ctypes.CDLL:
    """Load libalign.so (built by paper_2310_17864_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libalign.so not built at {LIB_PATH}; run paper_2310_17864_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        L.align_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(AlignConfig)]
        L.align_destroy.argtypes = [vp]
        L.align_submit.argtypes = [vp, vp, i64, i64, vp, i64, i32, AlignOut, ctypes.POINTER(u64)]
        L.align_submit_host.argtypes = [vp, vp, i64, i64, vp, i64, i32, AlignOut, ctypes.POINTER(u64)]
        L.align_submit_batch.argtypes = [vp, i32, ctypes.POINTER(AlignRequest), ctypes.POINTER(u64),
                                         ctypes.POINTER(i32)]
        L.align_flush.argtypes = [vp]
        L.align_poll.argtypes = [vp, u64, i32, ctypes.POINTER(i32)]
        L.align_join.argtypes = [vp, vp]
        L.align_poll_done.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(i32), i32, ctypes.POINTER(i32)]
        L.align_get_stats.argtypes = [vp, ctypes.POINTER(AlignStats), i32]
        L.align_status_string.argtypes = [i32]
        L.align_status_string.restype = ctypes.c_char_p
        L.align_last_error.argtypes = []
        L.align_last_error.restype = ctypes.c_char_p
        L.align_set_tuning.argtypes = [vp, i32, i32, i32]
        L.align_set_tuning_bucket.argtypes = [vp, i32, i32, i32]
        L.align_set_tuning_bucket_for.argtypes = [vp, i32, i32, i32, i32]
        L.align_token_spans.argtypes = [vp, vp, vp, vp, i32, i64, i64, vp, vp, vp, vp]
        L.align_ctc_beam_workspace_bytes.argtypes = [i32, i64, i32]
        L.align_ctc_beam_workspace_bytes.restype = u64
        L.align_ctc_beam_decode.argtypes = [vp, vp, i32, i64, i32, i32, i32, ctypes.c_float, vp, u64,
                                            vp, vp, vp, vp, vp, vp, vp, vp]
        L.align_probe_frame_latency.argtypes = [i32, i32, i32, i32, ctypes.POINTER(ctypes.c_double)]
        L.align_forced_noalloc.argtypes = [vp, i64, i64, vp, i64, i32, AlignOut, vp, ctypes.POINTER(i32)]
        L.align_noalloc_last_error.argtypes = []
        L.align_noalloc_last_error.restype = ctypes.c_char_p
        L.align_validate.argtypes = [vp, i64, i64, i32, i64, ctypes.POINTER(i64)]
        L.align_plan.argtypes = [i64, i64, i64, u64, u32, i32, i32, i32, ctypes.POINTER(AlignPlanInfo)]
        for name in EXPORTS:
            fn = getattr(L, name)
            if fn.restype is ctypes.c_int or fn.restype is None:
                fn.restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().align_status_string(int(code)).decode()


def last_error() -> str:
    return lib().align_last_error().decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise AlignError(rc, what)
    return rc


def _i32(targets) -> np.ndarray:
    if isinstance(targets, np.ndarray) and targets.dtype == np.int32 and targets.ndim == 1 and \
            targets.flags.c_contiguous:
        return targets
    return np.ascontiguousarray(np.asarray(targets, dtype=np.int32).reshape(-1))


# Row layout of AlignRequest (with its AlignOut) for building whole batches at once.
_REQ_DTYPE = np.dtype([("lp", np.uint64), ("T", np.int64), ("C", np.int64), ("tg", np.uint64), ("L", np.int64),
                       ("blank", np.int32), ("flags", np.uint32), ("path", np.uint64), ("scores", np.uint64),
                       ("total", np.uint64), ("states", np.uint64)])


# --------------------------------------------------------- same-named calls --

def align_create(cfg: AlignConfig | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().align_create(ctypes.byref(h), ctypes.byref(cfg) if cfg is not None else None), "align_create")
    return h


def align_destroy(ctx) -> None:
    _check(lib().align_destroy(ctx), "align_destroy")


def align_submit(ctx, log_probs_ptr: int, T: int, C: int, targets, blank: int, out: AlignOut) -> int:
    tg = _i32(targets)
    rid = ctypes.c_uint64()
    _check(lib().align_submit(ctx, ctypes.c_void_p(log_probs_ptr), T, C, tg.ctypes.data_as(ctypes.c_void_p),
                              tg.size, blank, out, ctypes.byref(rid)), "align_submit")
    return rid.value


def align_submit_host(ctx, log_probs_ptr: int, T: int, C: int, targets, blank: int, out: AlignOut) -> int:
    tg = _i32(targets)
    rid = ctypes.c_uint64()
    _check(lib().align_submit_host(ctx, ctypes.c_void_p(log_probs_ptr), T, C, tg.ctypes.data_as(ctypes.c_void_p),
                                   tg.size, blank, out, ctypes.byref(rid)), "align_submit_host")
    return rid.value


def align_submit_batch(ctx, reqs) -> tuple[list[int], list[int]]:
    """reqs: sequence of AlignRequest, or a numpy array of _REQ_DTYPE rows.
    Returns (request ids, per-request status)."""
    n = len(reqs)
    if isinstance(reqs, np.ndarray):
        assert reqs.dtype == _REQ_DTYPE and reqs.flags.c_contiguous
        arr = reqs.ctypes.data_as(ctypes.POINTER(AlignRequest))
    else:
        arr = (AlignRequest * n)(*reqs)
    ids = np.zeros(n, dtype=np.uint64)
    st = np.zeros(n, dtype=np.int32)
    rc = lib().align_submit_batch(ctx, n, arr, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                  st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc < 0 and n and bool(np.all(st != 0)):  # a context-level failure
        raise AlignError(rc, "align_submit_batch")
    return ids.tolist(), st.tolist()


def align_flush(ctx) -> None:
    _check(lib().align_flush(ctx), "align_flush")


def align_poll(ctx, request_id: int, timeout_ms: int = -1) -> tuple[int, int]:
    """Returns (ALIGN_OK or ALIGN_PENDING, request status)."""
    st = ctypes.c_int32(ALIGN_PENDING)
    rc = _check(lib().align_poll(ctx, request_id, timeout_ms, ctypes.byref(st)), "align_poll")
    return rc, st.value


def align_poll_done(ctx, max_n: int = 4096) -> list[tuple[int, int]]:
    """Finished (request id, result code) pairs, released; never waits."""
    ids = (ctypes.c_uint64 * max_n)()
    st = (ctypes.c_int32 * max_n)()
    n = ctypes.c_int32(0)
    _check(lib().align_poll_done(ctx, ids, st, max_n, ctypes.byref(n)), "align_poll_done")
    return [(ids[i], st[i]) for i in range(n.value)]


def align_join(ctx, stream_ptr: int | None = None) -> None:
    _check(lib().align_join(ctx, ctypes.c_void_p(stream_ptr) if stream_ptr else None), "align_join")


def align_get_stats(ctx, reset: bool = False) -> dict:
    s = AlignStats()
    _check(lib().align_get_stats(ctx, ctypes.byref(s), int(reset)), "align_get_stats")
    return {k: getattr(s, k) for k, _ in AlignStats._fields_}


def align_set_tuning(ctx, states_per_lane: int = 0, cta_warps: int = 0, max_cluster: int = 0) -> None:
    _check(lib().align_set_tuning(ctx, states_per_lane, cta_warps, max_cluster), "align_set_tuning")


def align_probe_frame_latency(device: int, warps: int, ctas: int, frames: int) -> float:
    """ns per frame of the null-work exchange pattern (see include/align.h)."""
    ns = ctypes.c_double(0.0)
    _check(lib().align_probe_frame_latency(device, warps, ctas, frames, ctypes.byref(ns)),
           "align_probe_frame_latency")
    return ns.value


def align_forced_noalloc(log_probs_ptr: int, T: int, C: int, targets, blank: int, out: AlignOut,
                         stream_ptr: int | None = None) -> tuple[int, int]:
    """Allocation-free alignment (see include/align.h). Returns (call code, request status);
    a negative call code comes with a message in align_noalloc_last_error()."""
    tg = _i32(targets)
    st = ctypes.c_int32(ALIGN_PENDING)
    rc = lib().align_forced_noalloc(ctypes.c_void_p(log_probs_ptr), T, C, tg.ctypes.data_as(ctypes.c_void_p),
                                    tg.size, blank, out, ctypes.c_void_p(stream_ptr) if stream_ptr else None,
                                    ctypes.byref(st))
    return rc, st.value


def align_noalloc_last_error() -> str:
    return lib().align_noalloc_last_error().decode()


def align_set_tuning_bucket(ctx, s_max: int, states_per_lane: int = 0, cta_warps: int = 0) -> None:
    _check(lib().align_set_tuning_bucket(ctx, s_max, states_per_lane, cta_warps), "align_set_tuning_bucket")


def align_token_spans(states, scores, frame_offsets, token_offsets, n: int, total_frames: int, total_tokens: int,
                      span_start, span_end, span_score, stream_ptr: int | None = None) -> None:
    """Same-named call: every pointer argument is a device address (int)."""
    _check(lib().align_token_spans(states, scores, frame_offsets, token_offsets, n, total_frames, total_tokens,
                                   span_start, span_end, span_score, stream_ptr), "align_token_spans")


def token_spans(states, scores, frame_offsets, token_offsets, stream=None, totals=None):
    """Token spans of packed alignments (CUDA tensors): states int32 [sum T],
    scores float32 [sum T], frame_offsets / token_offsets int64 [n+1], host
    arrays (copied to the device) or CUDA int64 tensors (then pass
    totals=(sum T, sum L) to avoid reading them back). Returns (start int32,
    end int32, score float32) CUDA tensors of [sum L]; frames relative to
    each utterance."""
    import torch
    dev = states.device

    def dev_offsets(x):
        if isinstance(x, torch.Tensor) and x.is_cuda:
            return x.to(torch.int64), None
        h = np.asarray(x.cpu() if isinstance(x, torch.Tensor) else x, dtype=np.int64)
        return torch.from_numpy(h).to(dev), h

    fo, fo_h = dev_offsets(frame_offsets)
    to, to_h = dev_offsets(token_offsets)
    n = fo.numel() - 1
    if totals is not None:
        total_T, total_L = int(totals[0]), int(totals[1])
    else:
        total_T = int(fo_h[-1]) if fo_h is not None else int(fo[-1].item())
        total_L = int(to_h[-1]) if to_h is not None else int(to[-1].item())
    if states.dtype != torch.int32 or scores.dtype != torch.float32 or states.numel() < total_T or \
            scores.numel() < total_T or not states.is_cuda or not scores.is_cuda:
        raise ValueError("states int32 / scores float32 CUDA tensors of sum T elements expected")
    start = torch.empty(total_L, dtype=torch.int32, device=dev)
    end = torch.empty(total_L, dtype=torch.int32, device=dev)
    score = torch.empty(total_L, dtype=torch.float32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    align_token_spans(states.data_ptr(), scores.data_ptr(), fo.data_ptr(), to.data_ptr(), n, total_T, total_L,
                      start.data_ptr(), end.data_ptr(), score.data_ptr(), st.cuda_stream)
    return start, end, score


def align_ctc_beam_workspace_bytes(n: int, total_frames: int, beam: int) -> int:
    return int(lib().align_ctc_beam_workspace_bytes(n, total_frames, beam))


def align_ctc_beam_decode(probs, frame_offsets, n: int, total_frames: int, V: int, blank: int, beam: int,
                          threshold: float, workspace, workspace_bytes: int, tokens, timesteps, lengths, totals,
                          scale_exp, scores, kept, stream_ptr: int | None = None) -> None:
    """Same-named call: every pointer argument is a device address (int)."""
    _check(lib().align_ctc_beam_decode(probs, frame_offsets, n, total_frames, V, blank, beam, threshold, workspace,
                                       workspace_bytes, tokens, timesteps, lengths, totals, scale_exp, scores, kept,
                                       stream_ptr), "align_ctc_beam_decode")


@dataclass
class BeamResult:
    """Outputs of ctc_beam_decode (CUDA tensors); hypothesis b of utterance u
    lives at tokens[offsets[u] * beam + b * T_u :][:lengths[u, b]]."""
    offsets: np.ndarray     # int64 [n+1] host copy of the frame offsets
    beam: int
    tokens: object          # int32 [sum T * beam]
    timesteps: object       # int32 [sum T * beam]
    lengths: object         # int32 [n, beam]
    totals: object          # float32 [n, beam]
    scale_exp: object       # int32 [n]
    scores: object          # float32 [n, beam]
    kept: object            # int32 [n]
    workspace: object

    def hypotheses(self, u: int) -> list[tuple[list[int], list[int], float]]:
        """(tokens, timesteps, score) of utterance u's hypotheses, best first (host)."""
        f0, f1 = int(self.offsets[u]), int(self.offsets[u + 1])
        T = f1 - f0
        lens = self.lengths[u].cpu().tolist()
        sc = self.scores[u].cpu().tolist()
        base = f0 * self.beam
        tk = self.tokens[base:base + self.beam * T].cpu().view(self.beam, T) if T else None
        tm = self.timesteps[base:base + self.beam * T].cpu().view(self.beam, T) if T else None
        out = []
        for b, L in enumerate(lens):
            if L < 0:
                continue
            out.append((tk[b, :L].tolist() if L else [], tm[b, :L].tolist() if L else [], sc[b]))
        return out


def ctc_beam_decode(probs, offsets, beam: int = 10, blank: int = 0, threshold: float = 1.0, stream=None,
                    workspace=None) -> BeamResult:
    """CTC prefix beam search with blank collapse over a packed batch:
    probs float32 CUDA tensor [sum T, V] (probabilities), offsets host int64
    [n+1]. threshold = the blank frame-skip threshold a (1.0: no collapse).
    One kernel launch on `stream` (default: current stream)."""
    import torch
    dev = probs.device
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    TT, V = probs.shape
    if off[-1] != TT:
        raise ValueError("offsets do not match the packed probabilities")
    fo = torch.from_numpy(off).to(dev)
    wb = align_ctc_beam_workspace_bytes(n, TT, beam)
    if workspace is None or workspace.numel() < wb:
        workspace = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    res = BeamResult(off, beam, torch.empty(max(TT * beam, 1), **i32), torch.empty(max(TT * beam, 1), **i32),
                     torch.empty((n, beam), **i32), torch.empty((n, beam), dtype=torch.float32, device=dev),
                     torch.empty(n, **i32), torch.empty((n, beam), dtype=torch.float32, device=dev),
                     torch.empty(n, **i32), workspace)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    align_ctc_beam_decode(probs.data_ptr(), fo.data_ptr(), n, TT, V, blank, beam, float(threshold),
                          workspace.data_ptr(), wb, res.tokens.data_ptr(), res.timesteps.data_ptr(),
                          res.lengths.data_ptr(), res.totals.data_ptr(), res.scale_exp.data_ptr(),
                          res.scores.data_ptr(), res.kept.data_ptr(), st.cuda_stream)
    res._keep = fo  # the offsets must outlive the launch
    return res


ALIGN_TUNE_LATENCY = 0
ALIGN_TUNE_THROUGHPUT = 1


def align_set_tuning_bucket_for(ctx, table: int, s_max: int, states_per_lane: int = 0, cta_warps: int = 0) -> None:
    _check(lib().align_set_tuning_bucket_for(ctx, table, s_max, states_per_lane, cta_warps),
           "align_set_tuning_bucket_for")


def align_validate(targets, C: int, blank: int, T: int) -> tuple[int, int]:
    tg = _i32(targets)
    rep = ctypes.c_int64(0)
    rc = lib().align_validate(tg.ctypes.data_as(ctypes.c_void_p), tg.size, C, blank, T, ctypes.byref(rep))
    return rc, rep.value


def align_plan(T: int, C: int, L: int, budget: int = 0, flags: int = 0, states_per_lane: int = 0,
               cta_warps: int = 0, max_cluster: int = 0) -> dict:
    info = AlignPlanInfo()
    _check(lib().align_plan(T, C, L, budget, flags, states_per_lane, cta_warps, max_cluster, ctypes.byref(info)),
           "align_plan")
    return {k: getattr(info, k) for k, _ in AlignPlanInfo._fields_ if k != "pad"}


# ------------------------------------------------------------ convenience --

@dataclass
class Result:
    request_id: int
    path: object      # torch tensor (device or host)
    scores: object
    total: object
    states: object
    status: int = ALIGN_PENDING


@dataclass
class PackedResult:
    """Requests of one packed batch (utterance i = rows offsets[i]:offsets[i+1])."""
    request_ids: np.ndarray   # uint64 [n]
    status: np.ndarray        # int32 [n], ALIGN_PENDING until waited for
    keep: tuple               # the packed buffers, kept alive until done


class Aligner:
    """Owns one context. Device submits take CUDA tensors and return CUDA tensors."""

    def __init__(self, device: int = 0, batched: bool = False, bp_budget_bytes: int = 0,
                 staging_bytes: int = 0, stream=None, force_checkpoint: bool = False,
                 wait_limit_ms: int = 0, max_inflight: int = 0, graphs: bool = True,
                 test_stall: bool = False, grid_teams: bool = True, debug_checks: bool = False,
                 generic_kernel: bool = False, persistent: bool = False, upload_descriptors: bool = False):
        import torch
        self.torch = torch
        self.device = device
        flags = (ALIGN_F_BATCHED if batched else 0) | (ALIGN_F_FORCE_CHECKPOINT if force_checkpoint else 0)
        flags |= 0 if graphs else ALIGN_F_NO_GRAPHS
        flags |= 0 if grid_teams else ALIGN_F_NO_GRID_TEAMS
        flags |= ALIGN_F_TEST_STALL if test_stall else 0
        flags |= ALIGN_F_DEBUG_CHECKS if debug_checks else 0
        flags |= ALIGN_F_GENERIC_KERNEL if generic_kernel else 0
        flags |= ALIGN_F_PERSISTENT if persistent else 0
        flags |= ALIGN_F_UPLOAD_DESCRIPTORS if upload_descriptors else 0
        cfg = AlignConfig(device=device, max_inflight=max_inflight, bp_budget_bytes=bp_budget_bytes,
                          staging_bytes=staging_bytes,
                          cuda_stream=(stream.cuda_stream if stream is not None else None), flags=flags,
                          wait_limit_ms=wait_limit_ms)
        self.ctx = align_create(cfg)
        self._live: dict[int, tuple] = {}
        self._ranges: list[list] = []  # packed batches: [first id, count, PackedResult, pending]

    def close(self) -> None:
        if self.ctx is not None:
            align_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, log_probs, targets, blank: int = 0, want_states: bool = False, out=None,
               logits: bool = False) -> Result:
        """Device tensors. logits=True: log_probs holds raw logits and the
        kernel applies log_softmax per frame while staging (ALIGN_REQ_LOGITS)."""
        torch = self.torch
        if not (log_probs.is_cuda and log_probs.dtype == torch.float32 and log_probs.dim() == 2
                and log_probs.is_contiguous()):
            raise ValueError("log_probs must be a contiguous CUDA float32 [T, C] tensor")
        T, C = log_probs.shape
        dev = log_probs.device
        if out is None:
            path = torch.empty(T, dtype=torch.int32, device=dev)
            scores = torch.empty(T, dtype=torch.float32, device=dev)
            total = torch.empty(1, dtype=torch.float32, device=dev)
            states = torch.empty(T, dtype=torch.int32, device=dev) if want_states else None
        else:
            path, scores, total, states = out
        if logits:
            (res,) = self.submit_batch([(log_probs, targets, blank, (path, scores, total, states))], logits=True)
            return res
        o = AlignOut(path.data_ptr(), scores.data_ptr(), total.data_ptr(),
                     states.data_ptr() if states is not None else None)
        rid = align_submit(self.ctx, log_probs.data_ptr(), T, C, targets, blank, o)
        res = Result(rid, path, scores, total, states)
        self._live[rid] = (log_probs, res)
        return res

    def submit_host(self, log_probs, targets, blank: int = 0, want_states: bool = False, out=None) -> Result:
        """log_probs: CPU float32 [T, C] tensor (pinned for asynchronous copies)."""
        torch = self.torch
        if log_probs.is_cuda or log_probs.dtype != torch.float32 or not log_probs.is_contiguous():
            raise ValueError("log_probs must be a contiguous CPU float32 [T, C] tensor")
        T, C = log_probs.shape
        if out is None:
            pin = log_probs.is_pinned()
            path = torch.empty(T, dtype=torch.int32, pin_memory=pin)
            scores = torch.empty(T, dtype=torch.float32, pin_memory=pin)
            total = torch.empty(1, dtype=torch.float32, pin_memory=pin)
            states = torch.empty(T, dtype=torch.int32, pin_memory=pin) if want_states else None
        else:
            path, scores, total, states = out
        o = AlignOut(path.data_ptr(), scores.data_ptr(), total.data_ptr(),
                     states.data_ptr() if states is not None else None)
        rid = align_submit_host(self.ctx, log_probs.data_ptr(), T, C, targets, blank, o)
        res = Result(rid, path, scores, total, states)
        self._live[rid] = (log_probs, res)
        return res

    def submit_batch(self, items, host: bool = False, logits: bool = False) -> list[Result]:
        """items: sequence of (log_probs, targets, blank, out) with out = (path, scores, total, states)
        tensors (device tensors, or host tensors when host=True). One C call for the whole batch."""
        n = len(items)
        reqs = np.zeros(n, dtype=_REQ_DTYPE)
        cols = {k: [0] * n for k in ("lp", "T", "C", "tg", "L", "blank", "path", "scores", "total", "states")}
        keep, results = [], []
        for i, (lp, tg, blank, out) in enumerate(items):
            tg = _i32(tg)
            path, scores, total, states = out
            T, C = lp.shape
            cols["lp"][i] = lp.data_ptr()
            cols["T"][i] = T
            cols["C"][i] = C
            cols["tg"][i] = tg.ctypes.data
            cols["L"][i] = tg.size
            cols["blank"][i] = blank
            cols["path"][i] = path.data_ptr()
            cols["scores"][i] = scores.data_ptr()
            cols["total"][i] = total.data_ptr()
            cols["states"][i] = states.data_ptr() if states is not None else 0
            keep.append((lp, tg))
            results.append(Result(0, path, scores, total, states))
        for k, v in cols.items():
            reqs[k] = v
        reqs["flags"] = (ALIGN_REQ_HOST if host else 0) | (ALIGN_REQ_LOGITS if logits else 0)
        ids, st = align_submit_batch(self.ctx, reqs)
        for r, rid, code, k in zip(results, ids, st, keep):
            if code < 0:
                raise AlignError(code, "align_submit_batch")
            r.request_id = rid
            self._live[rid] = (k, r)
        return results

    def flush(self) -> None:
        align_flush(self.ctx)

    def poll(self, res: Result, timeout_ms: int = -1) -> bool:
        rc, st = align_poll(self.ctx, res.request_id, timeout_ms)
        if rc == ALIGN_OK:
            res.status = st
            self._finish(res.request_id, st)
            return True
        return False

    def poll_done(self, max_n: int = 4096) -> list[Result]:
        """Results that finished since the last call (status filled in), without waiting."""
        out = []
        for rid, st in align_poll_done(self.ctx, max_n):
            res = self._finish(rid, st)
            if res is not None:
                out.append(res)
        return out

    def submit_packed(self, log_probs, offsets, targets, target_offsets, out, blank: int = 0,
                      host: bool = False, logits: bool = False) -> PackedResult:
        """A ragged batch in packed form, marshalled without a per-utterance
        Python loop. log_probs: float32 [sum T, C] (utterance i = rows
        offsets[i]:offsets[i+1]); targets: int32 [sum L] (utterance i =
        targets[target_offsets[i]:target_offsets[i+1]]), host memory;
        out = (path int32 [sum T], scores float32 [sum T], total float32 [n],
        states int32 [sum T] or None) in the same packing. Device tensors, or
        host tensors when host=True. One C call for the whole batch."""
        offsets = np.asarray(offsets, dtype=np.int64)
        target_offsets = np.asarray(target_offsets, dtype=np.int64)
        tg = _i32(targets)
        n = offsets.size - 1
        path, scores, total, states = out
        T, C = log_probs.shape
        if log_probs.dtype != self.torch.float32 or not log_probs.is_contiguous():
            raise ValueError("log_probs must be a contiguous float32 [sum T, C] tensor")
        if offsets[-1] != T or target_offsets.size != n + 1 or target_offsets[-1] != tg.size or total.numel() < n:
            raise ValueError("offsets / target_offsets do not match the packed tensors")
        f0 = offsets[:-1].astype(np.uint64)
        reqs = np.zeros(n, dtype=_REQ_DTYPE)
        reqs["lp"] = np.uint64(log_probs.data_ptr()) + f0 * np.uint64(4 * C)
        reqs["T"] = np.diff(offsets)
        reqs["C"] = C
        reqs["tg"] = np.uint64(tg.ctypes.data) + target_offsets[:-1].astype(np.uint64) * np.uint64(4)
        reqs["L"] = np.diff(target_offsets)
        reqs["blank"] = blank
        reqs["flags"] = (ALIGN_REQ_HOST if host else 0) | (ALIGN_REQ_LOGITS if logits else 0)
        reqs["path"] = np.uint64(path.data_ptr()) + f0 * np.uint64(4)
        reqs["scores"] = np.uint64(scores.data_ptr()) + f0 * np.uint64(4)
        reqs["total"] = np.uint64(total.data_ptr()) + np.arange(n, dtype=np.uint64) * np.uint64(4)
        if states is not None:
            reqs["states"] = np.uint64(states.data_ptr()) + f0 * np.uint64(4)
        ids, st = align_submit_batch(self.ctx, reqs)
        ids = np.asarray(ids, dtype=np.uint64)
        st = np.asarray(st, dtype=np.int32)
        bad = st < 0
        if bad.any():
            raise AlignError(int(st[bad][0]), "align_submit_batch")
        res = PackedResult(ids, np.full(n, ALIGN_PENDING, dtype=np.int32), (log_probs, tg, out))
        self._register_packed(res, ids)
        return res

    def _register_packed(self, res, ids) -> None:
        """The requests of a packed batch, live until finished: one range entry
        when their ids are consecutive (the usual case), else one per id."""
        n = ids.size
        if n and int(ids[-1]) - int(ids[0]) == n - 1:
            self._ranges.append([int(ids[0]), n, res, n])
        else:
            for i, rid in enumerate(ids.tolist()):
                self._live[rid] = (None, (res, i))

    def _waiter(self):
        """A stream of this context's device used only to wait for batches."""
        if getattr(self, "_wait_stream", None) is None:
            self._wait_stream = self.torch.cuda.Stream(self.device)
        return self._wait_stream

    def _finish(self, rid: int, code: int):
        """Record a finished request; returns its Result (None for a packed one)."""
        entry = self._live.pop(rid, None)
        if entry is None:
            for k, rg in enumerate(self._ranges):
                i = rid - rg[0]
                if 0 <= i < rg[1]:
                    if rg[2].status[i] == ALIGN_PENDING:
                        rg[2].status[i] = code
                        rg[3] -= 1
                        if rg[3] == 0:
                            del self._ranges[k]
                    break
            return None
        target = entry[1]
        if isinstance(target, tuple):
            target[0].status[target[1]] = code
            return None
        target.status = code
        return target

    def ctc_forward_packed(self, log_probs, offsets, targets, target_offsets, total, blank: int = 0,
                           host: bool = False) -> PackedResult:
        """Sum-product forward scores of a packed batch (ALIGN_REQ_SUM): total[i]
        = log of the total probability of utterance i's transcript (minus its
        CTC loss). Same packing as submit_packed; no path or scores outputs."""
        offsets = np.asarray(offsets, dtype=np.int64)
        target_offsets = np.asarray(target_offsets, dtype=np.int64)
        tg = _i32(targets)
        n = offsets.size - 1
        T, C = log_probs.shape
        if offsets[-1] != T or target_offsets.size != n + 1 or total.numel() < n:
            raise ValueError("offsets / target_offsets do not match the packed tensors")
        f0 = offsets[:-1].astype(np.uint64)
        reqs = np.zeros(n, dtype=_REQ_DTYPE)
        reqs["lp"] = np.uint64(log_probs.data_ptr()) + f0 * np.uint64(4 * C)
        reqs["T"] = np.diff(offsets)
        reqs["C"] = C
        reqs["tg"] = np.uint64(tg.ctypes.data) + target_offsets[:-1].astype(np.uint64) * np.uint64(4)
        reqs["L"] = np.diff(target_offsets)
        reqs["blank"] = blank
        reqs["flags"] = ALIGN_REQ_SUM | (ALIGN_REQ_HOST if host else 0)
        reqs["total"] = np.uint64(total.data_ptr()) + np.arange(n, dtype=np.uint64) * np.uint64(4)
        ids, st = align_submit_batch(self.ctx, reqs)
        ids = np.asarray(ids, dtype=np.uint64)
        st = np.asarray(st, dtype=np.int32)
        if (st < 0).any():
            raise AlignError(int(st[st < 0][0]), "align_submit_batch")
        res = PackedResult(ids, np.full(n, ALIGN_PENDING, dtype=np.int32), (log_probs, tg, total))
        self._register_packed(res, ids)
        return res

    def ctc_forward(self, log_probs, targets, blank: int = 0) -> tuple[int, float]:
        """Sum-product forward score of one utterance: (status, log total probability)."""
        dev = log_probs.is_cuda
        total = self.torch.empty(1, dtype=self.torch.float32, device=log_probs.device if dev else "cpu")
        if not dev:
            total = total.pin_memory()
        tg = _i32(targets)
        res = self.ctc_forward_packed(log_probs.contiguous(), [0, log_probs.shape[0]], tg, [0, tg.size], total,
                                      blank, host=not dev)
        self.flush()
        self.wait_packed(res)
        return int(res.status[0]), float(total.cpu()[0])

    def wait_packed(self, res: PackedResult) -> None:
        """Block until every request of a packed batch is done; fills res.status.
        Blocks on the batch of its last pending request only (batches launched
        after it keep running), then sweeps the finished statuses."""
        ids = res.request_ids
        while True:
            pend = np.nonzero(res.status == ALIGN_PENDING)[0]
            if pend.size == 0:
                return
            rid = int(ids[pend[-1]])
            rc, code = align_poll(self.ctx, rid, -1)
            if rc == ALIGN_OK:
                self._finish(rid, code)
            if (res.status == ALIGN_PENDING).any():
                for rid2, code2 in align_poll_done(self.ctx, max(4096, 2 * pend.size)):
                    self._finish(rid2, code2)

    def wait(self, results) -> None:
        """Block until every result in `results` is done: one device-side join
        and synchronisation, then one status sweep (align_poll_done) instead of
        one align_poll per request."""
        pending = {r.request_id: r for r in results if r.request_id in self._live}
        if not pending:
            return
        st = self._waiter()
        self.join(st)
        st.synchronize()
        while pending:
            for r in self.poll_done(max_n=max(4096, 2 * len(pending))):
                pending.pop(r.request_id, None)
            if pending:  # finished on the GPU but not yet reaped: poll the rest
                for rid in list(pending):
                    if self.poll(pending[rid], 0):
                        pending.pop(rid)

    def align(self, log_probs, targets, blank: int = 0, want_states: bool = False, logits: bool = False) -> Result:
        res = self.submit(log_probs, targets, blank, want_states, logits=logits)
        self.flush()
        self.poll(res)
        return res

    def join(self, stream=None) -> None:
        """Make a torch CUDA stream (default: current) wait for every launched batch."""
        st = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        align_join(self.ctx, st.cuda_stream)

    def stats(self, reset: bool = False) -> dict:
        return align_get_stats(self.ctx, reset)

    def set_tuning(self, states_per_lane: int = 0, cta_warps: int = 0, max_cluster: int = 0) -> None:
        align_set_tuning(self.ctx, states_per_lane, cta_warps, max_cluster)

    def set_tuning_table(self, table, mode: str = "latency") -> None:
        """table: iterable of (s_max, states_per_lane, cta_warps); replaces the
        latency (default) or throughput table."""
        which = {"latency": ALIGN_TUNE_LATENCY, "throughput": ALIGN_TUNE_THROUGHPUT}[mode]
        align_set_tuning_bucket_for(self.ctx, which, 0)
        for s_max, k, cw in table:
            align_set_tuning_bucket_for(self.ctx, which, int(s_max), int(k), int(cw))
