/*
 * align.h -- C ABI of the GB300 CTC forced-alignment library (libalign.so).
 *
 * The operation (TorchAudio 2.1 paper, Sec. 4, paragraph "CTC-based forced
 * alignment"): given the frame log-probabilities log_probs[T][C] of a
 * CTC-trained model, a transcript targets[L] and the blank id, compute the
 * frame-level alignment, i.e. the label per frame of the best-scoring CTC path
 * whose collapse (merge repeats, drop blanks) equals the transcript, and the
 * per-frame scores along it.
 *
 * Method: the Viterbi max-plus recursion over the trellis of S = 2L+1
 * blank-interleaved states of the CTC work the paper cites, followed by a
 * backtrack. Conventions fixed by this library where the paper is silent:
 *   - inside the max, ties keep the earlier candidate in the order
 *     stay (s), advance (s-1), skip (s-2);
 *   - a skip enters only an odd (label) state s >= 3 whose label differs from
 *     the label of state s-2;
 *   - the final state is S-1 (trailing blank) unless alpha_{T-1}(S-2) is
 *     strictly greater;
 *   - scores[t] = log_probs[t][path[t]]; total = alpha_{T-1}(final), which is
 *     the left-to-right binary32 sum of scores[0..T-1];
 *   - arithmetic is IEEE binary32, one round-to-nearest add per trellis cell
 *     after an exact max, no flush-to-zero, so results are deterministic and
 *     independent of the launch configuration.
 *
 * Threading: one align_ctx must be used by one host thread at a time.
 * Every call returns 0 (ALIGN_OK) or a status code below.
 */
#ifndef GB300_ALIGN_H
#define GB300_ALIGN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define ALIGN_OK 0
#define ALIGN_PENDING 1          /* align_poll: request not finished within the timeout */
#define ALIGN_E_INVAL (-1)       /* NULL pointer, T < 1, C < 2, L < 0, blank not in [0, C), bad config */
#define ALIGN_E_TARGET (-2)      /* a target outside [0, C) or equal to the blank */
#define ALIGN_E_INFEASIBLE (-3)  /* T < L + R, R = number of adjacent equal targets */
#define ALIGN_E_TOO_LARGE (-4)   /* the request cannot fit the memory budget even checkpointed */
#define ALIGN_E_AGAIN (-5)       /* too many requests in flight (max_inflight) */
#define ALIGN_E_NOPATH (-6)      /* feasible, but every path scores -inf (log 0 emissions) */
#define ALIGN_E_TIMEOUT (-7)     /* a device-side wait hit its time limit; the context stays usable */
#define ALIGN_E_CUDA (-8)        /* a CUDA runtime call failed (align_last_error has the text) */
#define ALIGN_E_NOTFOUND (-9)    /* unknown request id (never submitted or already polled) */
#define ALIGN_E_NOMEM (-10)      /* device or pinned allocation failed at create time */
#define ALIGN_E_NONFINITE (-11)  /* NaN or +inf in the emissions (found only under ALIGN_F_DEBUG_CHECKS) */

/* ---- configuration ----------------------------------------------------- */
#define ALIGN_F_BATCHED 0x1u          /* submit only queues; align_flush (or poll) launches the
                                         queued requests together as one ragged batch */
#define ALIGN_F_FORCE_CHECKPOINT 0x2u /* always use checkpointed recompute (no full backpointers) */
#define ALIGN_F_NO_GRAPHS 0x4u        /* batched launches without CUDA-graph capture */
#define ALIGN_F_NO_GRID_TEAMS 0x8u    /* transcripts beyond one thread-block cluster use larger
                                         K per lane instead of a grid team (a cooperative launch of
                                         one 16-warp CTA per SM linked through global memory) */
#define ALIGN_F_DEBUG_CHECKS 0x10u    /* every submit scans its [T, C] emissions for NaN and +inf
                                         (-inf, log 0, stays allowed) and returns ALIGN_E_NONFINITE;
                                         a device scan plus a synchronisation per request, or a host
                                         scan for host inputs. Off by default: without it such inputs
                                         give unspecified (but in-bounds) results. */
#define ALIGN_F_GENERIC_KERNEL 0x20u  /* run every Viterbi request on the generic trellis kernel
                                         (the one that also serves the sum-product, K >= 8 and
                                         C > 512) instead of the fast kernel for K = 2 or 4; same
                                         results, for comparison and testing */
#define ALIGN_F_PERSISTENT 0x40u      /* batches whose requests all qualify (log-probabilities on the
                                         device, one vocabulary with 16-byte rows, full backpointers
                                         within the budget, every team within the resident CTAs)
                                         run as ONE persistent launch: resident CTAs take the
                                         requests' seats from a device counter, longest first, with
                                         one kernel shape (the tuning table's for the batch's median
                                         S, K = 2 or 4); other batches launch per shape group */
#define ALIGN_F_UPLOAD_DESCRIPTORS 0x80u /* always copy a batch's descriptors and targets to device
                                         memory and its result codes back, as for batches that
                                         use other kernels; by default a batch that runs only the
                                         fast kernel (device inputs and outputs, full or grid-team
                                         backpointers) has its kernels read them from the pinned
                                         host image and write the result codes there, which saves
                                         two copies per batch (needs native host atomics) */
#define ALIGN_F_TEST_STALL 0x80000000u /* testing the device watchdog only: in every request whose
                                         trellis spans more than one warp, the first warp never
                                         hands its values on, so the next warp's bounded wait runs
                                         out and the request ends with ALIGN_E_TIMEOUT after about
                                         wait_limit_ms; single-warp requests are unaffected */

typedef struct align_ctx align_ctx;   /* opaque */

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    int32_t max_inflight;      /* requests submitted and not yet polled; 0 -> 8192 */
    uint64_t bp_budget_bytes;  /* device arena for backpointers and checkpoints; 0 -> 1 GiB.
                                  Requests are admitted while their footprint fits; a request
                                  whose full backpointers do not fit runs checkpointed */
    uint64_t staging_bytes;    /* device staging for align_submit_host inputs/outputs; 0 -> 64 MiB */
    void *cuda_stream;         /* cudaStream_t all work is ordered after/on; NULL -> own stream */
    uint32_t flags;            /* ALIGN_F_* */
    uint32_t wait_limit_ms;    /* limit of every device-side spin wait; 0 -> 2000 */
} align_config;

/* Outputs, caller-owned. For align_submit they are DEVICE pointers, for
   align_submit_host HOST pointers. path and scores: T elements; total: 1;
   states (optional, may be NULL): T trellis state indices. */
typedef struct {
    int32_t *path;
    float *scores;
    float *total;
    int32_t *states;
} align_out;

/* Create a context on cfg->device: allocates the backpointer arena, the staging
   buffers and descriptor tables once; no later call allocates device memory.
   cfg may be NULL (all defaults). Errors: ALIGN_E_INVAL, ALIGN_E_NOMEM, ALIGN_E_CUDA. */
int align_create(align_ctx **out, const align_config *cfg);

/* Finish all work in flight, then free everything the context owns.
   NULL is accepted (no-op). */
int align_destroy(align_ctx *ctx);

/* Submit one alignment.
   log_probs: DEVICE pointer, FP32 [T][C] row-major, contiguous.
   targets:   HOST pointer, int32 [L]; copied before return (may be freed after).
   out:       DEVICE pointers (see align_out).
   Ownership: log_probs and out.* must stay valid and unmodified until
   align_poll reports the request done (same rule as cudaMemcpyAsync).
   Validation (ALIGN_E_INVAL / ALIGN_E_TARGET / ALIGN_E_INFEASIBLE /
   ALIGN_E_TOO_LARGE) happens here on the host; on such an error no request is
   created. In plain mode the work is launched before return; with
   ALIGN_F_BATCHED it is queued until align_flush / align_poll. Work is ordered
   after everything already enqueued on cfg->cuda_stream at submit time.
   On success *request_id identifies the request for align_poll. */
int align_submit(align_ctx *ctx, const float *log_probs, int64_t T, int64_t C,
                 const int32_t *targets, int64_t L, int32_t blank, align_out out,
                 uint64_t *request_id);

/* Same as align_submit, but log_probs and out.* are HOST pointers. When the
   device can address all of them (page-locked mapped memory, or any host
   memory on a device that reads the host page tables), one batched copy
   kernel per batch moves the emissions in and one the results out; otherwise
   the library copies host->device and device->host with one copy per buffer. The host buffers must stay valid
   and unmodified until align_poll reports the request done. */
int align_submit_host(align_ctx *ctx, const float *log_probs, int64_t T, int64_t C,
                      const int32_t *targets, int64_t L, int32_t blank, align_out out,
                      uint64_t *request_id);

/* One request of a batch submission. */
#define ALIGN_REQ_HOST 0x1u  /* log_probs and out.* are HOST pointers (as align_submit_host) */
#define ALIGN_REQ_SUM 0x4u    /* sum-product instead of Viterbi: the same trellis with log-add in
                                 place of max (the forward score of the CTC work the paper cites);
                                 out.total = log of the total probability of every CTC path of the
                                 transcript (minus the CTC loss); out.path / scores / states are not
                                 used (may be NULL). FP32 with the fast exponential / logarithm
                                 intrinsics, the maximum factored out of every log-add; no
                                 backpointers (no backpointer memory). Not combined with
                                 ALIGN_REQ_LOGITS (ALIGN_E_INVAL). */
#define ALIGN_REQ_LOGITS 0x2u /* log_probs holds raw per-frame scores (logits): a pre-pass
                                 kernel computes each row's lse = m + logf(sum expf(x - m)), m
                                 the row maximum, and the trellis kernel uses x - lse in FP32
                                 as it reads the staged rows, so no log_softmax output [T][C]
                                 is written or read again; scores are then log-probabilities.
                                 Results equal an alignment of those FP32 log-probabilities;
                                 they may differ from one of log-probabilities computed
                                 elsewhere by the rounding of expf / logf. */
typedef struct {
    const float *log_probs;   /* [T][C] FP32 row-major, device (or host with ALIGN_REQ_HOST) */
    int64_t T, C;
    const int32_t *targets;   /* HOST int32 [L], copied during the call */
    int64_t L;
    int32_t blank;
    uint32_t flags;           /* ALIGN_REQ_* */
    align_out out;
} align_request;

/* Submit n requests in one call; they are queued together and, unless the
   context is in batched mode, launched together as one ragged batch before
   return. Each request is validated like align_submit: request_ids[i] gets its
   id (0 if rejected) and submit_status[i] (optional) its result code. Returns
   ALIGN_OK if all were accepted, else the first rejection code. */
int align_submit_batch(align_ctx *ctx, int32_t n, const align_request *reqs, uint64_t *request_ids,
                       int32_t *submit_status);

/* Launch every queued request that fits the memory budget (batched mode).
   Requests that do not fit yet stay queued and are launched by later calls
   once memory is released. No-op in plain mode when nothing is queued. */
int align_flush(align_ctx *ctx);

/* Wait up to timeout_ms (0 = just check, < 0 = forever) for a request.
   Returns ALIGN_OK when it is done, writing its result code to
   *request_status (ALIGN_OK, ALIGN_E_NOPATH, ALIGN_E_TIMEOUT, or ALIGN_E_CUDA
   if the kernel refused launch parameters that did not fit the request); the id is
   then released. Returns ALIGN_PENDING if it is still running, or
   ALIGN_E_NOTFOUND. Polling also launches queued work. */
int align_poll(align_ctx *ctx, uint64_t request_id, int32_t timeout_ms, int32_t *request_status);

/* Collect finished requests without waiting: launches queued work like
   align_poll, then writes up to `max` finished request ids and their result
   codes (ALIGN_OK, ALIGN_E_NOPATH or ALIGN_E_TIMEOUT) and releases them;
   *count gets the number written. Serving loops call this once per tick
   instead of polling every request. */
int align_poll_done(align_ctx *ctx, uint64_t *ids, int32_t *statuses, int32_t max, int32_t *count);

/* Make `stream` (a cudaStream_t; NULL = the context's stream) wait on the GPU
   for every batch launched so far, without blocking the host. Batches are not
   otherwise ordered before later work on the context's stream, so that new
   batches can overlap running ones; use this to time or order after them. */
int align_join(align_ctx *ctx, void *stream);

/* Counters of the context since creation (or the last reset). */
typedef struct {
    uint64_t kernel_launches;   /* kernels this library launched */
    uint64_t graph_launches;    /* CUDA graph replays */
    uint64_t requests_done;
    uint64_t cells;             /* sum of T * S over finished requests */
    uint64_t checkpointed;      /* requests that ran with checkpointed recompute */
    uint64_t bp_bytes_peak;     /* peak arena use */
    uint64_t throughput_batches; /* batches planned with the throughput tuning table */
    uint64_t grid_teams;        /* finished requests that ran as a grid team */
    uint64_t sum_requests;      /* finished sum-product (ALIGN_REQ_SUM) requests */
    uint64_t persistent_batches; /* batches launched as one persistent launch (ALIGN_F_PERSISTENT) */
} align_stats;

int align_get_stats(align_ctx *ctx, align_stats *out, int32_t reset);

/* Human-readable name of a status code (static string). */
const char *align_status_string(int32_t code);

/* Text of the last CUDA error seen by this thread (static buffer). */
const char *align_last_error(void);

/* Tuning of the trellis kernel for requests submitted after the call:
   states per lane K (2, 4, 8 or 16), warps per CTA before a transcript is
   split over a thread-block cluster (1..32), and the largest cluster (1..16).
   0 leaves a value unchanged. Every choice gives bit-identical results. */
int align_set_tuning(align_ctx *ctx, int32_t states_per_lane, int32_t cta_warps, int32_t max_cluster);

/* Measurement helper: time per frame of the irreducible per-frame chain of
   the recursion at warp scope with null work around it (shared-memory
   emission read, neighbour shuffle, one max, one add), run by `ctas` CTAs of
   `warps` warps for `frames` frames. Allocates a 24-byte result buffer on
   `device` and synchronises. This is the per-frame synchronisation bound of
   the roofline; it is not part of the alignment path. */
int align_probe_frame_latency(int32_t device, int32_t warps, int32_t ctas, int32_t frames,
                              double *ns_per_frame);

/* Per-range tuning measured on this GPU: transcripts with S <= s_max states
   use states_per_lane (2, 4, 8 or 16) and cta_warps (1..16); the smallest
   matching s_max wins; ranges not covered use align_set_tuning's values.
   s_max <= 0 clears the table. Up to 16 ranges (ALIGN_E_AGAIN beyond). The
   autotuner of the Python package fills this table from timed trials. */
int align_set_tuning_bucket(align_ctx *ctx, int32_t s_max, int32_t states_per_lane, int32_t cta_warps);

/* Tuning tables: ALIGN_TUNE_LATENCY holds the shapes that finish one
   utterance soonest (short chains of few-state lanes); ALIGN_TUNE_THROUGHPUT
   the shapes that finish many utterances soonest when the GPU is
   oversubscribed (more states per lane and warps per CTA). When a throughput
   table is set, each batch of two or more requests is planned with it if its
   work exceeds what the GPU runs concurrently: sum over requests of
   T * ceil(S / 64) above T_max * 8 * (number of SMs); otherwise with the
   latency table. Grid teams (see ALIGN_F_NO_GRID_TEAMS) are planned for
   latency batches only. Same
   arguments as align_set_tuning_bucket (which sets the latency table);
   s_max <= 0 clears the given table. ALIGN_E_INVAL for an unknown table. */
#define ALIGN_TUNE_LATENCY 0
#define ALIGN_TUNE_THROUGHPUT 1
int align_set_tuning_bucket_for(align_ctx *ctx, int32_t table, int32_t s_max, int32_t states_per_lane,
                                int32_t cta_warps);

/* ---- CTC prefix beam search with blank collapse -------------------------- */

/* Beam search decoding of CTC outputs (paper Sec. 5, "CUDA CTC decoder": beam
   search parallel over batch, hypotheses and vocabulary, with the blank
   collapse of the cited work, frame-skip threshold a; no language model).
   Blank collapse: frame t is a blank frame when probs[t][blank] > threshold;
   a blank frame right after a blank frame is skipped (threshold >= 1 keeps
   every frame). Prefix beam search over the kept frames: each hypothesis is
   a label prefix with pb (paths ending in blank) and pnb (ending in its last
   label z); per frame with probabilities y it stays (pb' = (pb + pnb) *
   y[blank], pnb' = pnb * y[z]) or grows by a non-blank label c (pnb = (pb +
   pnb) * y[c], or pb * y[c] when c == z); a growth equal to a hypothesis of
   the beam adds into its pnb; the beam keeps the `beam` largest totals pb +
   pnb, ties to the smaller candidate index (stays by beam slot first, then
   growths by slot and label). Binary32, one rounding per operation in that
   order; after each frame every probability is multiplied by the power of
   two that brings the largest total into [0.5, 1), the exponents summed.
   Inputs (DEVICE pointers): probs float32 [total_frames][V] (probabilities,
   finite and >= 0; rows need not sum to 1), frame_offsets int64 [n+1]
   (utterance u = rows frame_offsets[u] .. frame_offsets[u+1]-1,
   frame_offsets[n] = total_frames). 2 <= V, 0 <= blank < V, 1 <= beam <= 16.
   workspace: at least align_ctc_beam_workspace_bytes(n, total_frames, beam)
   device bytes (kept frame lists and the prefix tree), owned by the caller.
   Outputs (DEVICE, caller-owned): for utterance u with T_u frames and
   hypothesis b (beam order, largest total first): tokens / timesteps int32
   at [frame_offsets[u] * beam + b * T_u, + lengths[u*beam + b]) = labels and
   the frame of each label's emission (frame index within the utterance);
   lengths int32 [n*beam] (-1: no hypothesis in that slot); totals float32
   [n*beam] = pb + pnb after the last rescale; scale_exp int32 [n] = E, so
   the probability of a hypothesis is totals * 2^E; scores float32 [n*beam]
   = logf(total) + E ln 2 (-inf for a zero total); kept int32 [n] = frames
   kept by blank collapse. Two kernels on cuda_stream, asynchronous: the
   B most probable labels of every frame (one warp per frame), then the
   search (one CTA per utterance). ALIGN_E_INVAL for bad sizes, pointers or a small workspace,
   ALIGN_E_TOO_LARGE when V is beyond the shared memory, ALIGN_E_CUDA if the
   launch fails. Results for NaN, negative or infinite probabilities are
   unspecified (the kernel stays within its buffers). */
uint64_t align_ctc_beam_workspace_bytes(int32_t n, int64_t total_frames, int32_t beam);
int align_ctc_beam_decode(const float *probs, const int64_t *frame_offsets, int32_t n, int64_t total_frames,
                          int32_t V, int32_t blank, int32_t beam, float threshold, void *workspace,
                          uint64_t workspace_bytes, int32_t *tokens, int32_t *timesteps, int32_t *lengths,
                          float *totals, int32_t *scale_exp, float *scores, int32_t *kept, void *cuda_stream);

/* ---- token spans: the alignment per transcript token -------------------- */

/* Token spans of one or more finished alignments, packed: utterance u owns
   frames frame_offsets[u] .. frame_offsets[u+1]-1 of states / scores and
   tokens token_offsets[u] .. token_offsets[u+1]-1 of the outputs (paper
   Sec. 4: forced alignment gives the alignment between audio frames and
   transcript tokens; this collapses it to one span per token). Transcript
   token i occupies the frames whose trellis state is 2i + 1 (the states
   output of align_submit); span_start[k] = first such frame, span_end[k] =
   one past the last (frames relative to the utterance's first frame), and
   span_score[k] = the FP32 sum of those frames' scores, added in frame order,
   divided by the span length (IEEE division). A token with no frame (not a
   valid alignment) gets -1, -1, 0.
   All pointers are DEVICE pointers: states int32 [total_frames], scores
   float32 [total_frames], frame_offsets / token_offsets int64 [n+1] with
   frame_offsets[n] = total_frames and token_offsets[n] = total_tokens;
   outputs int32 / int32 / float32 [total_tokens]. Runs asynchronously on
   cuda_stream (NULL = legacy default stream): two memsets and two kernels.
   ALIGN_E_INVAL for negative sizes or missing pointers, ALIGN_E_CUDA if a
   launch fails. */
int align_token_spans(const int32_t *states, const float *scores, const int64_t *frame_offsets,
                      const int64_t *token_offsets, int32_t n, int64_t total_frames, int64_t total_tokens,
                      int32_t *span_start, int32_t *span_end, float *span_score, void *cuda_stream);

/* ---- allocation-free entry point ---------------------------------------- */

/* Align one utterance without allocating any memory, for callers that cannot
   allocate device memory when they need an alignment (a real-time thread that
   must not risk the device-wide synchronisation of cudaMalloc, or a host that
   gives the library a fixed device-memory budget up front). The paper has no
   counterpart; this is an interface choice of this library.
   log_probs: DEVICE FP32 [T][C]; targets: HOST int32 [L]; out: DEVICE pointers;
   cuda_stream: stream to run on (NULL = legacy default stream). Same results
   as align_submit. All scratch (descriptor, status, targets copy, backpointers,
   anchor rows) lives in one fixed 32 MiB device array built into the library,
   held on every device where the library is loaded until the process exits.
   Requests needing more scratch than that return ALIGN_E_TOO_LARGE (message
   in align_noalloc_last_error, which every non-OK return fills).
   log_probs and the outputs must be device (or managed) memory of the current
   device: other pointers return ALIGN_E_INVAL. The first call on a device
   looks up the array's address and, under CUDA's lazy module loading, is where
   the library's device code and the array are loaded onto the device (which
   allocates and may synchronise): make it outside the allocation-sensitive
   path and before any stream capture on that device. The call copies from
   host memory and synchronises its stream, so on a stream that is being
   captured it returns ALIGN_E_INVAL and does nothing. Every
   call shares the array and keeps the previous call's contents: calls that
   overlap on the GPU race, so never issue two at once. The call synchronises
   `cuda_stream` before it returns and writes the request's result code
   (ALIGN_OK, ALIGN_E_NOPATH or ALIGN_E_TIMEOUT) to *request_status. */
int align_forced_noalloc(const float *log_probs, int64_t T, int64_t C, const int32_t *targets, int64_t L,
                         int32_t blank, align_out out, void *cuda_stream, int32_t *request_status);

/* Text of the last align_forced_noalloc failure on this thread (static buffer). */
const char *align_noalloc_last_error(void);

/* ---- host-only helpers (no GPU needed) -------------------------------- */

/* Step A1 alone: checks T >= 1, C >= 2, 0 <= blank < C, every target in [0, C)
   and != blank, and feasibility T >= L + R. Writes R (adjacent equal targets)
   to *repeats when non-NULL. Returns ALIGN_OK or the error of align_submit. */
int align_validate(const int32_t *targets, int64_t L, int64_t C, int32_t blank, int64_t T,
                   int64_t *repeats);

/* Kernel shape and memory footprint align_submit would choose. */
typedef struct {
    int32_t states_per_lane;    /* K: trellis states held by one lane */
    int32_t warps_per_cta;
    int32_t cluster_ctas;       /* 1: a single CTA */
    int32_t frames_per_stage;   /* emission rows per shared-memory stage */
    int32_t checkpointed;       /* 1: backpointers recomputed per segment */
    int32_t checkpoint_every;   /* frames between alpha checkpoints */
    int32_t checkpoints;        /* number of segments */
    int32_t pad;
    uint64_t backpointer_bytes; /* footprint of full backpointers */
    uint64_t checkpoint_bytes;  /* footprint of the checkpointed form */
} align_plan_info;

/* Plan a request of T frames, C classes and L targets for a context with the
   given budget (0 = default), flags and tuning (0 = defaults, see align_set_tuning).
   Returns ALIGN_OK, ALIGN_E_INVAL or ALIGN_E_TOO_LARGE. */
int align_plan(int64_t T, int64_t C, int64_t L, uint64_t bp_budget_bytes, uint32_t flags,
               int32_t states_per_lane, int32_t cta_warps, int32_t max_cluster, align_plan_info *out);

#ifdef __cplusplus
}
#endif
#endif /* GB300_ALIGN_H */
