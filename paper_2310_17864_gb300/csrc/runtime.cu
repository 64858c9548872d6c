// Host runtime behind the C ABI in include/align.h.
//
// Responsibilities:
//   * validation of a request (step A1 of the hot path: targets in range,
//     no blank target, T >= L + R), on the host, O(L);
//   * planning: kernel shape (states per lane K, warps per CTA, cluster size)
//     from the number of trellis states S = 2L+1, and the memory footprint of
//     full backpointers or of checkpointed recompute;
//   * memory: one device arena for backpointers / checkpoints (the budget),
//     one for per-request metadata, one for host-I/O staging, and a pinned host
//     arena for descriptor uploads -- all allocated once in align_create;
//   * scheduling: requests are queued, admitted while their footprint fits,
//     grouped by kernel shape and launched as ragged batches (one launch per
//     shape group, longest first) on a pool of streams so batches overlap;
//     completion is tracked by events and released memory admits more work
//     (continuous batching);
//   * checkpointed recompute for requests whose backpointers do not fit.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/align.h"
#include "align_internal.h"
#include "trellis.cuh"

using namespace gb300_align;

namespace {

thread_local char g_last_error[512] = "";

void set_error(const char* what, cudaError_t e) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", what, cudaGetErrorString(e),
                static_cast<int>(e));
}

#define CU(call)                         \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) {             \
      set_error(#call, e_);              \
      return ALIGN_E_CUDA;               \
    }                                    \
  } while (0)

constexpr uint64_t kAlign = 256;
constexpr size_t kMaxStreams = 128;  // worker streams of a context
constexpr size_t kMaxGraphs = 16;    // cached batch graphs of a context
inline uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, cap) with coalescing frees.
class Arena {
 public:
  void init(uint64_t cap) {
    cap_ = cap;
    free_.clear();
    if (cap) free_[0] = cap;
    used_ = peak_ = 0;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = round_up(std::max<uint64_t>(bytes, 1), kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes;
        const uint64_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = round_up(std::max<uint64_t>(bytes, 1), kAlign);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t cap() const { return cap_; }
  uint64_t used() const { return used_; }
  uint64_t peak() const { return peak_; }
  void reset_peak() { peak_ = used_; }

 private:
  uint64_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

struct Alloc {
  uint64_t off = 0, bytes = 0;
  bool live = false;
};

// Metadata block per request in device memory: status, state_io, final2[2].
struct MetaBlock {
  int32_t status;
  int32_t state_io;
  float final2[2];
};
static_assert(sizeof(MetaBlock) == 16, "meta");

enum class ReqState { Queued, Launched, Done };

struct Request {
  uint64_t id = 0;
  ReqState state = ReqState::Queued;
  const float* lp = nullptr;  // device emissions (or host, when host_io)
  bool host_io = false;
  // host_io: device-addressable aliases of the host buffers (mapped pinned
  // memory, or system memory the device reaches through the host page
  // tables); then one batched copy kernel moves them instead of one
  // cudaMemcpyAsync per buffer. Null when any buffer is not addressable.
  const void* lp_alias = nullptr;
  align_out out_alias{};
  bool logits = false;  // lp holds raw logits (ALIGN_REQ_LOGITS)
  bool sum = false;     // sum-product forward score only (ALIGN_REQ_SUM)
  align_out out{};            // caller outputs (device or host)
  int64_t T = 0, C = 0, L = 0;
  int32_t blank = 0;
  std::vector<int32_t> targets;
  Plan plan{};
  int plan_table = ALIGN_TUNE_LATENCY;  // tuning table the plan was made with
  Alloc bp;                   // backpointers or checkpoints + segment buffer
  Alloc stage;                // host-I/O device staging
  int batch = -1;
  int meta_index = -1;        // index of its metadata block in the batch
  int32_t status = ALIGN_PENDING;
};

// A captured batch launch, replayed for later batches with the same launch
// structure. Its descriptor image lives at fixed addresses (device and pinned
// host regions taken from the context's arenas), so a replay only rewrites the
// host image and calls cudaGraphLaunch.
struct GraphEntry {
  std::vector<int64_t> key;
  Alloc meta, pinned;
  cudaGraphExec_t exec = nullptr;
  bool busy = false;  // a batch using the fixed image has not been reaped yet
  int seen = 0;       // batches with this structure so far (captured on the second)
};

struct Batch {
  int id = 0;
  int graph = -1;  // index of the GraphEntry whose image this batch uses
  cudaEvent_t done = nullptr;
  Alloc meta;      // device: descriptors + per-request metadata + targets
  Alloc pinned;    // host pinned: upload image + status download
  std::vector<uint64_t> reqs;
  MetaBlock* h_meta = nullptr;  // pinned copy of the requests' metadata blocks
  bool finished = false;
  std::vector<cudaEvent_t> events;     // pooled events used by this batch
  Alloc xlink;     // persistent launches: the teams' CTA links (backpointer arena)
};

}  // namespace

struct align_ctx {
  int device = 0;
  cudaStream_t main = nullptr;
  bool own_main = false;
  std::vector<cudaStream_t> workers;
  cudaStream_t grid_stream = nullptr;   // every grid-team launch, in order: two teams never
                                        // compete for the SMs each needs all of at once
  std::vector<cudaEvent_t> fork_events;
  std::vector<cudaEvent_t> event_pool;  // reusable events for batch joins and completion
  int next_worker = 0;
  uint32_t flags = 0;
  uint64_t wait_limit_ns = 2000000000ull;
  int max_inflight = 8192;

  char* d_bp = nullptr;
  Arena bp_arena;
  char* d_meta = nullptr;
  Arena meta_arena;
  char* d_stage = nullptr;
  Arena stage_arena;
  char* h_pinned = nullptr;
  char* d_pinned = nullptr;  // device address of h_pinned (direct images), or nullptr
  Arena pinned_arena;
  int32_t* d_check = nullptr;  // ALIGN_F_DEBUG_CHECKS: result word of the emission scan
  int32_t* h_check = nullptr;

  std::vector<GraphEntry> graphs;
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> queued;
  std::map<int, Batch> batches;
  uint64_t next_id = 1;
  int next_batch = 1;

  bool host_ats = false;  // the device reads pageable host memory through the host page tables
  TuneTable tune;     // latency shapes (also the defaults)
  TuneTable tune_tp;  // throughput shapes (nbuckets == 0: not set)
  int num_sms = 0;
  int smem_optin = 0;
  std::map<std::tuple<int, int, int>, int> persist_ctas;  // (K, warps, C) -> resident CTAs of that shape
  align_stats stats{};
};

namespace {

uint64_t inflight_count(const align_ctx* ctx) { return ctx->reqs.size(); }

// Plan of a request with one tuning table. Logits requests get a per-frame
// shift buffer (written by the lse pre-pass before their trellis launch).
int plan_request(const align_ctx* ctx, const TuneTable& table, int64_t T, int64_t C, int64_t L, bool logits,
                 Plan* out, bool sum = false) {
  TuneTable t = table;
  // Throughput batches with wide rows (C > 64: stages of 8 KB per few frames):
  // CTAs of at most four warps, so that several share an SM (a wider CTA
  // needs a stage ring that leaves room for one).
  if (&table == &ctx->tune_tp && C > 64) t.max_warps = std::min(t.max_warps, 4);
  const int rc = make_plan(t, T, C, L, sum ? ~0ull : ctx->bp_arena.cap(),
                           !sum && (ctx->flags & ALIGN_F_FORCE_CHECKPOINT) != 0, out);
  if (rc != ALIGN_OK) return rc;
  if (ctx->flags & ALIGN_F_GENERIC_KERNEL) out->shape.fast = 0;
  if (sum) {  // the forward pass only: no backpointers, anchor rows or checkpoints
    out->shape.sum = 1;
    out->shape.fast = 0;  // the sum-product runs on the generic kernel
    out->checkpointed = false;
    out->bp_bytes = 0;
    out->z_off = 0;
    if (plan_device_bytes(*out) > ctx->bp_arena.cap()) return ALIGN_E_TOO_LARGE;
  }
  if (logits) {
    // Per-frame shifts of the lse pre-pass (generic kernel) or per-warp partial
    // sums of the scores (fast kernel): T or team-warps floats.
    out->shape.norm = 1;
    const uint64_t team_warps = static_cast<uint64_t>(out->shape.warps) * static_cast<uint64_t>(out->shape.ncta);
    out->lse_bytes = (std::max(static_cast<uint64_t>(T), team_warps) * 4 + 255) & ~255ull;
    if (plan_device_bytes(*out) > ctx->bp_arena.cap()) return ALIGN_E_TOO_LARGE;
  }
  return ALIGN_OK;
}

// A device-addressable alias of host memory, or nullptr.
void* device_alias(const align_ctx* ctx, const void* p) {
  if (!p) return nullptr;
  // The device reads any host address through the host page tables: no query.
  if (ctx->host_ats) return const_cast<void*>(p);
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
  if (a.type == cudaMemoryTypeManaged) return const_cast<void*>(p);
  return nullptr;
}


cudaEvent_t take_event(align_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

int finish_batch(align_ctx* ctx, Batch& b) {
  for (size_t i = 0; i < b.reqs.size(); ++i) {
    auto it = ctx->reqs.find(b.reqs[i]);
    if (it == ctx->reqs.end()) continue;
    Request& r = it->second;
    r.state = ReqState::Done;
    r.status = b.h_meta[i].status;
    if (r.status == ALIGN_PENDING) r.status = ALIGN_E_TIMEOUT;
    if (r.bp.live) ctx->bp_arena.release(r.bp.off, r.bp.bytes), r.bp.live = false;
    if (r.stage.live) ctx->stage_arena.release(r.stage.off, r.stage.bytes), r.stage.live = false;
    ctx->stats.requests_done++;
    ctx->stats.cells += static_cast<uint64_t>(r.T) * static_cast<uint64_t>(2 * r.L + 1);
    if (r.plan.checkpointed) ctx->stats.checkpointed++;
    if (r.plan.shape.grid && !r.plan.shape.persist) ctx->stats.grid_teams++;
    if (r.sum) ctx->stats.sum_requests++;
  }
  if (b.meta.live) ctx->meta_arena.release(b.meta.off, b.meta.bytes), b.meta.live = false;
  if (b.pinned.live) ctx->pinned_arena.release(b.pinned.off, b.pinned.bytes), b.pinned.live = false;
  if (b.xlink.live) ctx->bp_arena.release(b.xlink.off, b.xlink.bytes), b.xlink.live = false;
  if (b.graph >= 0) ctx->graphs[static_cast<size_t>(b.graph)].busy = false;
  b.finished = true;
  return ALIGN_OK;
}

// Retire finished batches; returns ALIGN_E_CUDA on a failed query.
int reap(align_ctx* ctx) {
  for (auto it = ctx->batches.begin(); it != ctx->batches.end();) {
    Batch& b = it->second;
    cudaError_t q = cudaEventQuery(b.done);
    if (q == cudaSuccess) {
      finish_batch(ctx, b);
      for (cudaEvent_t e : b.events) ctx->event_pool.push_back(e);
      it = ctx->batches.erase(it);
    } else if (q == cudaErrorNotReady) {
      ++it;
    } else {
      set_error("cudaEventQuery", q);
      return ALIGN_E_CUDA;
    }
  }
  return ALIGN_OK;
}

uint64_t request_bp_bytes(const Plan& p) { return plan_device_bytes(p); }

// Launch as many queued requests as fit, as one batch. Returns ALIGN_OK even
// if nothing could be launched (they stay queued).
// Plans the queued requests with the throughput table when there are several
// and their work exceeds what the GPU runs at once (T * ceil(S/64)
// warp-frames, summed, above T_max * 8 warps * SMs), else with the latency
// table. Plans are only
// remade for requests whose table changes; a request keeps its plan if the
// other table cannot place it.
bool want_throughput(const align_ctx* ctx) {
  if (ctx->tune_tp.nbuckets == 0) return false;
  uint64_t work = 0;
  int64_t tmax = 0;
  for (uint64_t id : ctx->queued) {
    const Request& r = ctx->reqs.at(id);
    work += static_cast<uint64_t>(r.T) * static_cast<uint64_t>((2 * r.L + 1 + 63) / 64);
    tmax = std::max(tmax, r.T);
  }
  // One request alone is a latency problem whatever its size.
  return ctx->queued.size() >= 2 &&
         work > static_cast<uint64_t>(tmax) * 8ull * static_cast<uint64_t>(std::max(1, ctx->num_sms));
}

bool choose_tables(align_ctx* ctx) {
  const bool tp = want_throughput(ctx);
  const int want = tp ? ALIGN_TUNE_THROUGHPUT : ALIGN_TUNE_LATENCY;
  for (uint64_t id : ctx->queued) {
    Request& r = ctx->reqs.at(id);
    if (r.plan_table == want) continue;
    Plan p{};
    if (plan_request(ctx, tp ? ctx->tune_tp : ctx->tune, r.T, r.C, r.L, r.logits, &p, r.sum) == ALIGN_OK) {
      p.shape.occ = tp ? 1 : 0;
      r.plan = p;
      r.plan_table = want;
    }
  }
  return tp;
}

constexpr int kPersistTable = 2;  // plan_table of a request planned for a persistent launch

// Resident CTAs of a persistent launch of shape (K, warps) over rows of C
// classes (cached per context), or 0.
int persist_ctas(align_ctx* ctx, const LaunchShape& shape, int C, int F) {
  const auto key = std::make_tuple(shape.K, shape.warps, C);
  auto it = ctx->persist_ctas.find(key);
  if (it != ctx->persist_ctas.end()) return it->second;
  const FwdParams P = plan_params(shape, C, F, ctx->wait_limit_ns);
  int n = 0;
  if (persist_max_ctas(shape, P, ctx->device, &n) != 0) {
    (void)cudaGetLastError();
    n = 0;
  }
  ctx->persist_ctas[key] = n;
  return n;
}

// Whether the queued requests run as one persistent launch; if so, every
// queued request is planned with the batch's one shape: K states per lane and
// W compute warps from the tuning table's entry for the median S (K = 2 or 4,
// W <= 15), ceil(S / (32 K W)) CTAs per team. Every request must align
// log-probabilities in device memory with 16-byte rows of one vocabulary
// C <= 512, keep full backpointers within the budget, and have a team of at
// most the resident CTAs of that shape. Otherwise plans made for a persistent
// launch are remade by choose_tables.
bool choose_persist(align_ctx* ctx, bool tp) {
  if (!(ctx->flags & ALIGN_F_PERSISTENT) || (ctx->flags & (ALIGN_F_GENERIC_KERNEL | ALIGN_F_FORCE_CHECKPOINT)) ||
      ctx->queued.size() < 2)
    return false;
  const int64_t C = ctx->reqs.at(ctx->queued.front()).C;
  std::vector<int64_t> S;
  S.reserve(ctx->queued.size());
  for (uint64_t id : ctx->queued) {
    const Request& r = ctx->reqs.at(id);
    if (r.sum || r.logits || r.host_io || r.C != C || C > 512 || !rows_bulk_ok(r.lp, r.C)) return false;
    S.push_back(2 * r.L + 1);
  }
  std::nth_element(S.begin(), S.begin() + static_cast<std::ptrdiff_t>(S.size() / 2), S.end());
  const TuneTable t = resolve_tuning(tp ? ctx->tune_tp : ctx->tune, S[S.size() / 2]);
  const int K = (t.K == 2) ? 2 : 4;
  const int W = std::max(1, std::min({t.cta_warps, t.max_warps, 15}));
  std::vector<std::pair<Request*, Plan>> plans;
  plans.reserve(ctx->queued.size());
  for (uint64_t id : ctx->queued) {
    Request& r = ctx->reqs.at(id);
    Plan p{};
    if (r.plan_table == kPersistTable && r.plan.shape.K == K && r.plan.shape.warps == W) {
      p = r.plan;
    } else if (make_persist_plan(K, W, r.T, r.C, r.L, ctx->bp_arena.cap(), &p) != ALIGN_OK) {
      return false;
    }
    plans.emplace_back(&r, p);
  }
  LaunchShape one = plans.front().second.shape;
  one.ncta = 1;
  const int ctas = persist_ctas(ctx, one, static_cast<int>(C), plans.front().second.frames_per_stage);
  for (const auto& rp : plans)
    if (rp.second.shape.ncta > ctas) return false;
  for (auto& rp : plans) {
    rp.first->plan = rp.second;
    rp.first->plan_table = kPersistTable;
  }
  return true;
}

int launch_persistent(align_ctx* ctx, std::vector<Request*>& take);

int launch_queued(align_ctx* ctx) {
  if (ctx->queued.empty()) return ALIGN_OK;
  const bool tp_want = want_throughput(ctx);
  const bool persist = choose_persist(ctx, tp_want);
  const bool tp_batch = persist ? tp_want : choose_tables(ctx);
  std::vector<Request*> take;
  std::deque<uint64_t> keep;
  uint64_t meta_est = 0;  // descriptor + metadata + targets bytes of the batch
  const uint64_t meta_room = std::min(ctx->meta_arena.cap() - ctx->meta_arena.used(),
                                      ctx->pinned_arena.cap() - ctx->pinned_arena.used());
  while (!ctx->queued.empty()) {
    const uint64_t id = ctx->queued.front();
    Request& r = ctx->reqs.at(id);
    uint64_t m = (1 + static_cast<uint64_t>(r.plan.nck)) * sizeof(FwdJob) + 64 +
                 static_cast<uint64_t>(r.L) * 4 + 16 + static_cast<uint64_t>(r.plan.shape.ncta) * 4;
    if (r.host_io && r.lp_alias) {  // batched-copy chunks of this request
      const uint64_t T = static_cast<uint64_t>(r.T);
      m += (T * static_cast<uint64_t>(r.C) * 4 / kCopyChunk + 3 * (T * 4 / kCopyChunk) + 5) * sizeof(CopyChunk);
    }
    if (meta_est + m + 4 * kAlign > meta_room) break;  // the rest waits for the next batch
    ctx->queued.pop_front();
    // Admission: backpointer / checkpoint footprint, plus staging for host I/O.
    Plan& p = r.plan;
    uint64_t need = request_bp_bytes(p);
    if (!p.checkpointed && !ctx->bp_arena.alloc(need, &r.bp.off)) {
      if (p.shape.persist) {  // persistent launches keep full backpointers: wait for memory
        keep.push_back(id);
        continue;
      }
      // Full backpointers do not fit now: fall back to checkpointed recompute
      // if that fits, otherwise wait for memory to be released.
      const uint64_t ck_need = p.ckpt_bytes + p.seg_bp_bytes + p.x_bytes;
      if (ck_need <= ctx->bp_arena.cap() - ctx->bp_arena.used() && ctx->bp_arena.alloc(ck_need, &r.bp.off)) {
        p.checkpointed = true;
        need = ck_need;
      } else {
        keep.push_back(id);
        continue;
      }
    } else if (p.checkpointed && !ctx->bp_arena.alloc(need, &r.bp.off)) {
      keep.push_back(id);
      continue;
    }
    r.bp.bytes = need;
    r.bp.live = true;
    meta_est += m;
    if (r.host_io) {
      const uint64_t sb = host_stage_bytes(r.T, r.C);
      if (!ctx->stage_arena.alloc(sb, &r.stage.off)) {
        ctx->bp_arena.release(r.bp.off, r.bp.bytes);
        r.bp.live = false;
        keep.push_back(id);
        continue;
      }
      r.stage.bytes = sb;
      r.stage.live = true;
    }
    // Checkpointed logits requests take the generic kernel (its score pass
    // reads the per-frame shifts of the lse pre-pass).
    if (r.plan.checkpointed && r.plan.shape.norm) r.plan.shape.fast = 0;
    take.push_back(&r);
  }
  for (auto it = keep.rbegin(); it != keep.rend(); ++it) ctx->queued.push_front(*it);
  if (take.empty()) return ALIGN_OK;
  ctx->stats.bp_bytes_peak = std::max(ctx->stats.bp_bytes_peak, ctx->bp_arena.peak());

  // Longest first (trellis cells), then group by kernel shape.
  std::stable_sort(take.begin(), take.end(), [](const Request* a, const Request* b) {
    return a->T * (2 * a->L + 1) > b->T * (2 * b->L + 1);
  });
  if (persist) {
    if (tp_batch) ctx->stats.throughput_batches++;
    return launch_persistent(ctx, take);
  }

  // Descriptor image: full-mode jobs grouped by shape; checkpointed requests
  // get 1 + nck descriptors each.
  // (K, warps, ncta, F, C) -> request indices. C is part of the key: the launch
  // parameters (emission stage size) depend on it.
  std::map<std::tuple<int, int, int, int, int, int, int, int>, std::vector<int>> groups;
  size_t njobs = 0;
  for (size_t i = 0; i < take.size(); ++i) {
    const Plan& p = take[i]->plan;
    if (p.checkpointed || p.shape.grid) {  // a launch sequence of its own
      njobs += p.checkpointed ? 1 + static_cast<size_t>(p.nck) : 1;
    } else {
      groups[{p.shape.K, p.shape.warps, p.shape.ncta, p.frames_per_stage, static_cast<int>(take[i]->C), p.shape.occ,
              p.shape.norm, p.shape.sum}].push_back(
          static_cast<int>(i));
      njobs += 1;
    }
  }
  uint64_t tgt_words = 0;
  for (auto* r : take) tgt_words += round_up(static_cast<uint64_t>(std::max<int64_t>(r->L, 1)), 4);
  // Batched host copies: chunks of the emissions in, of the outputs out.
  const auto nch = [](uint64_t bytes) { return bytes ? (bytes + kCopyChunk - 1) / kCopyChunk : 0; };
  uint64_t n_h2d = 0, n_d2h = 0;
  for (auto* r : take) {
    if (!r->host_io || !r->lp_alias) continue;
    const uint64_t T = static_cast<uint64_t>(r->T);
    n_h2d += nch(T * static_cast<uint64_t>(r->C) * 4);
    n_d2h += 2 * nch(T * 4) + 1 + (r->out.states ? nch(T * 4) : 0);
  }
  const uint64_t off_jobs = 0;
  const uint64_t off_metas = round_up(njobs * sizeof(FwdJob), kAlign);
  const uint64_t off_tgts = round_up(off_metas + take.size() * sizeof(MetaBlock), kAlign);
  const uint64_t off_h2d = round_up(off_tgts + tgt_words * 4, kAlign);
  const uint64_t off_d2h = round_up(off_h2d + n_h2d * sizeof(CopyChunk), kAlign);
  const uint64_t up_bytes = round_up(off_d2h + n_d2h * sizeof(CopyChunk), kAlign);
  const uint64_t off_status = up_bytes;  // pinned only: metadata download (status of every request)
  const uint64_t pin_bytes = up_bytes + round_up(take.size() * sizeof(MetaBlock), kAlign);

  // CUDA graph for this launch structure (not for host-buffer requests, whose
  // copies have per-batch host addresses).
  bool any_host = false;
  for (auto* r : take) any_host = any_host || r->host_io;
  // Direct image: when every launch is the fast kernel (device buffers, or
  // host buffers the copy kernels reach), the kernels read the descriptors,
  // targets and copy lists from the pinned image (each CTA copies its
  // descriptor to shared memory once) and update the result codes there: no
  // upload or download copy, no graph.
  bool direct = ctx->d_pinned != nullptr;
  for (auto* r : take) direct = direct && r->plan.shape.fast != 0 && (!r->host_io || r->lp_alias != nullptr);
  int gi = -1;
  bool need_capture = false;
  uint64_t up_copy = up_bytes;
  uint64_t off_meta_dl = off_status;
  if (!(ctx->flags & ALIGN_F_NO_GRAPHS) && !any_host && !direct) {
    uint64_t up_bucket = 64 << 10;
    while (up_bucket < up_bytes) up_bucket <<= 1;
    std::vector<int64_t> key{static_cast<int64_t>(take.size()), static_cast<int64_t>(up_bucket)};
    for (auto& kv : groups) {
      key.insert(key.end(), {std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                             std::get<3>(kv.first), std::get<4>(kv.first), std::get<5>(kv.first),
                             std::get<6>(kv.first), std::get<7>(kv.first), static_cast<int64_t>(kv.second.size())});
    }
    for (auto* r : take) {
      const Plan& p = r->plan;
      if (!p.checkpointed && !p.shape.grid) continue;
      key.insert(key.end(), {-1, p.shape.K, p.shape.warps, p.shape.ncta, p.shape.occ, p.shape.grid, p.shape.norm,
                             p.shape.sum, p.frames_per_stage, p.checkpointed ? p.nck : -1, r->C});
    }
    for (size_t k = 0; k < ctx->graphs.size(); ++k)
      if (ctx->graphs[k].key == key) gi = static_cast<int>(k);
    if (gi < 0) {
      // First batch with this structure: remember it, launch directly.
      if (ctx->graphs.size() < kMaxGraphs) {
        GraphEntry ge;
        ge.key = key;
        ge.seen = 1;
        ctx->graphs.push_back(ge);
      }
    } else if (ctx->graphs[static_cast<size_t>(gi)].busy) {
      gi = -1;  // its image is in use: launch this batch directly
    } else if (!ctx->graphs[static_cast<size_t>(gi)].meta.live) {
      // Second batch with this structure: fix its image regions and capture.
      GraphEntry& ge = ctx->graphs[static_cast<size_t>(gi)];
      const uint64_t pin_need = up_bucket + round_up(take.size() * sizeof(MetaBlock), kAlign);
      bool ok = false;
      if (ctx->meta_arena.alloc(up_bucket, &ge.meta.off)) {
        if (ctx->pinned_arena.alloc(pin_need, &ge.pinned.off)) {
          ge.meta.bytes = up_bucket;
          ge.meta.live = true;
          ge.pinned.bytes = pin_need;
          ge.pinned.live = true;
          ok = true;
        } else {
          ctx->meta_arena.release(ge.meta.off, up_bucket);
        }
      }
      if (!ok) gi = -1;
    }
    if (gi >= 0 && !ctx->graphs[static_cast<size_t>(gi)].meta.live) gi = -1;
    if (gi >= 0) {
      GraphEntry& ge = ctx->graphs[static_cast<size_t>(gi)];
      ge.seen++;
      need_capture = ge.exec == nullptr;
      up_copy = up_bucket;
      off_meta_dl = up_bucket;
    }
  }

  if (tp_batch) ctx->stats.throughput_batches++;
  Batch b;
  b.id = ctx->next_batch++;
  auto unwind = [&]() {
    for (auto* r : take) {
      if (r->bp.live) ctx->bp_arena.release(r->bp.off, r->bp.bytes), r->bp.live = false;
      if (r->stage.live) ctx->stage_arena.release(r->stage.off, r->stage.bytes), r->stage.live = false;
      ctx->queued.push_front(r->id);
    }
  };
  char* h = nullptr;
  char* d = nullptr;
  if (gi >= 0) {
    GraphEntry& ge = ctx->graphs[static_cast<size_t>(gi)];
    ge.busy = true;
    b.graph = gi;
    h = ctx->h_pinned + ge.pinned.off;
    d = ctx->d_meta + ge.meta.off;
  } else if (direct) {
    if (!ctx->pinned_arena.alloc(up_bytes, &b.pinned.off)) {
      unwind();
      return ALIGN_OK;  // retried after other batches release their images
    }
    b.pinned.bytes = up_bytes;
    b.pinned.live = true;
    h = ctx->h_pinned + b.pinned.off;
    d = ctx->d_pinned + b.pinned.off;
    off_meta_dl = off_metas;  // the result codes are read where the kernels write them
  } else {
    if (!ctx->meta_arena.alloc(up_bytes, &b.meta.off)) {
      unwind();
      return ALIGN_OK;  // retried after other batches release metadata
    }
    b.meta.bytes = up_bytes;
    b.meta.live = true;
    if (!ctx->pinned_arena.alloc(pin_bytes, &b.pinned.off)) {
      ctx->meta_arena.release(b.meta.off, b.meta.bytes);
      unwind();
      return ALIGN_OK;
    }
    b.pinned.bytes = pin_bytes;
    b.pinned.live = true;
    h = ctx->h_pinned + b.pinned.off;
    d = ctx->d_meta + b.meta.off;
  }
  FwdJob* hjobs = reinterpret_cast<FwdJob*>(h + off_jobs);
  MetaBlock* hmeta = reinterpret_cast<MetaBlock*>(h + off_metas);
  int32_t* htgt = reinterpret_cast<int32_t*>(h + off_tgts);
  const FwdJob* djobs = reinterpret_cast<const FwdJob*>(d + off_jobs);
  MetaBlock* dmeta = reinterpret_cast<MetaBlock*>(d + off_metas);
  const int32_t* dtgt = reinterpret_cast<const int32_t*>(d + off_tgts);
  b.h_meta = reinterpret_cast<MetaBlock*>(h + off_meta_dl);

  // Per-request metadata, targets and device views of inputs / outputs.
  std::vector<const int32_t*> req_tgt(take.size());
  std::vector<const float*> req_lp(take.size());
  std::vector<align_out> req_out(take.size());
  CopyChunk* hh2d = reinterpret_cast<CopyChunk*>(h + off_h2d);
  CopyChunk* hd2h = reinterpret_cast<CopyChunk*>(h + off_d2h);
  const CopyChunk* dh2d = reinterpret_cast<const CopyChunk*>(d + off_h2d);
  const CopyChunk* dd2h = reinterpret_cast<const CopyChunk*>(d + off_d2h);
  size_t ih2d = 0, id2h = 0;
  const auto add_chunks = [](CopyChunk* list, size_t& n, const void* src, void* dst, uint64_t bytes) {
    for (uint64_t o = 0; o < bytes; o += kCopyChunk) {
      list[n++] = CopyChunk{static_cast<const char*>(src) + o, static_cast<char*>(dst) + o,
                            std::min(kCopyChunk, bytes - o), 0};
    }
  };
  uint64_t tw = 0;
  for (size_t i = 0; i < take.size(); ++i) {
    Request& r = *take[i];
    r.state = ReqState::Launched;
    r.batch = b.id;
    r.meta_index = static_cast<int>(i);
    b.reqs.push_back(r.id);
    hmeta[i].status = ALIGN_PENDING;
    hmeta[i].state_io = 0;
    hmeta[i].final2[0] = hmeta[i].final2[1] = -INFINITY;
    b.h_meta[i].status = ALIGN_PENDING;
    if (r.L) std::memcpy(htgt + tw, r.targets.data(), static_cast<size_t>(r.L) * 4);
    req_tgt[i] = dtgt + tw;
    tw += round_up(static_cast<uint64_t>(std::max<int64_t>(r.L, 1)), 4);
    if (r.host_io) {
      char* sbase = ctx->d_stage + r.stage.off;
      HostStage hs = host_stage_layout(r.T, r.C);
      req_lp[i] = reinterpret_cast<const float*>(sbase + hs.lp);
      req_out[i].path = reinterpret_cast<int32_t*>(sbase + hs.path);
      req_out[i].scores = reinterpret_cast<float*>(sbase + hs.scores);
      req_out[i].total = reinterpret_cast<float*>(sbase + hs.total);
      req_out[i].states = r.out.states ? reinterpret_cast<int32_t*>(sbase + hs.states) : nullptr;
    } else {
      req_lp[i] = r.lp;
      req_out[i] = r.out;
    }
  }

  auto base_job = [&](size_t i) {
    const Request& r = *take[i];
    FwdJob j{};
    j.lp = req_lp[i];
    j.tgt = req_tgt[i];
    j.status = &dmeta[i].status;
    j.state_io = &dmeta[i].state_io;
    j.final2 = dmeta[i].final2;
    j.path = req_out[i].path;
    j.scores = req_out[i].scores;
    j.total = req_out[i].total;
    j.states = req_out[i].states;
    j.T = static_cast<int32_t>(r.T);
    j.C = static_cast<int32_t>(r.C);
    j.blank = r.blank;
    j.L = static_cast<int32_t>(r.L);
    j.S = static_cast<int32_t>(2 * r.L + 1);
    j.flags = (rows_bulk_ok(j.lp, r.C) ? kJobBulkRows : 0u) | ((ctx->flags & ALIGN_F_TEST_STALL) ? kJobTestStall : 0u);
    j.lse = r.logits ? reinterpret_cast<float*>(ctx->d_bp + r.bp.off + plan_lse_off(r.plan)) : nullptr;
    return j;
  };

  // Fill descriptors: shape groups first (contiguous ranges), then the
  // checkpointed sequences.
  // Copy chunks of a launch's host-buffer requests: [first, first + count) of
  // the emission (in) and output (out) lists, moved on the launch's own stream
  // so that copies of one group overlap the kernels of others.
  struct CopyRange {
    size_t in_first = 0, in_count = 0, out_first = 0, out_count = 0;
  };
  const auto add_request_chunks = [&](size_t i, CopyRange& cr) {
    const Request& r = *take[i];
    if (!r.host_io || !r.lp_alias) return;
    const uint64_t T = static_cast<uint64_t>(r.T);
    add_chunks(hh2d, ih2d, r.lp_alias, const_cast<float*>(req_lp[i]), T * static_cast<uint64_t>(r.C) * 4);
    if (r.out.path) add_chunks(hd2h, id2h, req_out[i].path, r.out_alias.path, T * 4);
    if (r.out.scores) add_chunks(hd2h, id2h, req_out[i].scores, r.out_alias.scores, T * 4);
    add_chunks(hd2h, id2h, req_out[i].total, r.out_alias.total, 4);
    if (r.out.states) add_chunks(hd2h, id2h, req_out[i].states, r.out_alias.states, T * 4);
    cr.in_count = ih2d - cr.in_first;
    cr.out_count = id2h - cr.out_first;
  };
  struct GroupLaunch {
    LaunchShape shape;
    int F;
    size_t first, count;
    CopyRange cr;
    int64_t t_max;  // longest job of the group (frames): its chain sets the launch's duration
  };
  std::vector<GroupLaunch> glaunch;
  // Requests with a launch sequence of their own: checkpointed (pass 1, then
  // the segments last to first) and grid teams (one cooperative launch each).
  struct CkLaunch {
    size_t req, first, count;
    uint64_t* xlink;  // grid team links (zeroed before every launch), or nullptr
    CopyRange cr;
  };
  std::vector<CkLaunch> cklaunch;
  size_t jn = 0;
  for (auto& kv : groups) {
    GroupLaunch gl{};
    gl.shape = LaunchShape{std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), std::get<5>(kv.first)};
    gl.shape.norm = std::get<6>(kv.first);
    gl.shape.sum = std::get<7>(kv.first);
    gl.shape.fast = take[static_cast<size_t>(kv.second[0])]->plan.shape.fast;  // implied by K, C and sum
    gl.F = std::get<3>(kv.first);
    gl.first = jn;
    gl.count = kv.second.size();
    gl.t_max = 0;
    gl.cr.in_first = ih2d;
    gl.cr.out_first = id2h;
    for (int i : kv.second) {
      add_request_chunks(static_cast<size_t>(i), gl.cr);
      const Request& r = *take[static_cast<size_t>(i)];
      gl.t_max = std::max(gl.t_max, r.T);
      FwdJob j = base_job(static_cast<size_t>(i));
      j.bp = r.sum ? nullptr : reinterpret_cast<uint32_t*>(ctx->d_bp + r.bp.off);
      j.ztab = r.sum ? nullptr : reinterpret_cast<uint8_t*>(ctx->d_bp + r.bp.off + r.plan.z_off);
      j.zstride = r.plan.zstride;
      j.t_begin = 0;
      j.t_end = j.T;
      j.bp_rows = std::max(j.T - 1, 0);
      j.flags |= kJobWriteFinal | (r.sum ? 0u : kJobChase);
      hjobs[jn++] = j;
    }
    glaunch.push_back(gl);
  }
  // Launch the groups with the longest chains first: when the batch fills the
  // GPU, later launches wait for room, and the longest job must not wait.
  std::stable_sort(glaunch.begin(), glaunch.end(),
                   [](const GroupLaunch& x, const GroupLaunch& y) { return x.t_max > y.t_max; });
  for (size_t i = 0; i < take.size(); ++i) {
    const Request& r = *take[i];
    const Plan& p = r.plan;
    if (!p.checkpointed && !p.shape.grid) continue;
    uint64_t* xl = p.shape.grid ? reinterpret_cast<uint64_t*>(ctx->d_bp + r.bp.off + plan_x_off(p)) : nullptr;
    CkLaunch cl{i, jn, p.checkpointed ? static_cast<size_t>(p.nck) + 1 : 1, xl, CopyRange{}};
    cl.cr.in_first = ih2d;
    cl.cr.out_first = id2h;
    add_request_chunks(i, cl.cr);
    if (!p.checkpointed) {  // grid team, full backpointers (none for the sum-product)
      FwdJob j = base_job(i);
      j.bp = r.sum ? nullptr : reinterpret_cast<uint32_t*>(ctx->d_bp + r.bp.off);
      j.ztab = r.sum ? nullptr : reinterpret_cast<uint8_t*>(ctx->d_bp + r.bp.off + p.z_off);
      j.zstride = p.zstride;
      j.t_begin = 0;
      j.t_end = j.T;
      j.bp_rows = std::max(j.T - 1, 0);
      j.flags |= kJobWriteFinal | (r.sum ? 0u : kJobChase);
      j.xlink = xl;
      hjobs[jn++] = j;
      cklaunch.push_back(cl);
      continue;
    }
    float* ck = reinterpret_cast<float*>(ctx->d_bp + r.bp.off);
    uint32_t* seg = reinterpret_cast<uint32_t*>(ctx->d_bp + r.bp.off + p.ckpt_bytes);
    FwdJob j = base_job(i);  // pass 1: checkpoints every Kc frames, final state, no backpointers
    j.t_begin = 0;
    j.t_end = j.T;
    j.ckpt = ck;
    j.ck_every = p.ck_every;
    j.ck_stride = p.ck_stride;
    j.flags |= kJobWriteFinal;
    j.xlink = xl;
    hjobs[jn++] = j;
    for (int c = p.nck - 1; c >= 0; --c) {  // pass 2: segments, last first
      FwdJob s = base_job(i);
      const int t0 = c * p.ck_every;
      const int e = std::min(t0 + p.ck_every, s.T - 1);
      s.t_begin = t0;
      s.t_end = e + 1;
      s.alpha_in = ck + static_cast<size_t>(c) * p.ck_stride;
      s.final2 = nullptr;
      s.bp = seg;
      s.bp_rows = e - t0;
      s.ztab = reinterpret_cast<uint8_t*>(ctx->d_bp + r.bp.off + p.ckpt_bytes + p.seg_z_off);
      s.zstride = p.zstride;
      s.flags |= kJobChase;
      s.xlink = xl;
      hjobs[jn++] = s;
    }
    cklaunch.push_back(cl);
  }

  // Streams: the batch forks from the main stream; each group / checkpointed
  // sequence runs on its own worker stream; everything joins on the first.
  cudaEvent_t fork = ctx->fork_events[static_cast<size_t>(b.id) % ctx->fork_events.size()];
  CU(cudaEventRecord(fork, ctx->main));
  // Idle streams first, so a new batch never queues behind a long kernel of an
  // earlier batch (head-of-line blocking); the pool grows when all are busy.
  size_t ngrid = 0;  // grid teams: all on the context's grid stream
  for (const CkLaunch& cl : cklaunch) ngrid += cl.xlink ? 1 : 0;
  const size_t nlanes = std::max<size_t>(1, glaunch.size() + cklaunch.size() - ngrid);
  std::vector<cudaStream_t> used;
  for (size_t k = 0; k < ctx->workers.size() && used.size() < nlanes; ++k) {
    cudaStream_t s = ctx->workers[(static_cast<size_t>(ctx->next_worker) + k) % ctx->workers.size()];
    if (cudaStreamQuery(s) == cudaSuccess) used.push_back(s);
  }
  ctx->next_worker = static_cast<int>((static_cast<size_t>(ctx->next_worker) + 1) % ctx->workers.size());
  while (used.size() < nlanes && ctx->workers.size() < kMaxStreams) {
    cudaStream_t s;
    CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ctx->workers.push_back(s);
    used.push_back(s);
  }
  for (size_t k = 0; used.size() < nlanes && k < ctx->workers.size(); ++k) {
    cudaStream_t s = ctx->workers[(static_cast<size_t>(ctx->next_worker) + k) % ctx->workers.size()];
    if (std::find(used.begin(), used.end(), s) == used.end()) used.push_back(s);
  }
  const size_t nwork = used.size();
  if (ngrid) used.push_back(ctx->grid_stream);
  cudaStream_t s0 = used[0];
  for (cudaStream_t s : used) CU(cudaStreamWaitEvent(s, fork, 0));
  uint64_t nkernels = 0;
  // Everything from the descriptor upload to the status download; issued
  // directly, or captured once into the batch graph.
  auto body = [&]() -> int {
  if (!direct) CU(cudaMemcpyAsync(d, h, up_copy, cudaMemcpyHostToDevice, s0));
  for (size_t i = 0; i < take.size(); ++i) {
    Request& r = *take[i];
    if (r.host_io && !r.lp_alias) {
      CU(cudaMemcpyAsync(const_cast<float*>(req_lp[i]), r.lp, static_cast<size_t>(r.T * r.C) * 4,
                         cudaMemcpyHostToDevice, s0));
    }
  }

  // Copy kernels of one launch's host-buffer requests, in or out, on its stream.
  const auto copy_range = [&](const CopyChunk* list, size_t first, size_t count, cudaStream_t s) -> int {
    if (!count) return ALIGN_OK;
    const cudaError_t e =
        static_cast<cudaError_t>(launch_copy_chunks(list + first, static_cast<int>(count), ctx->num_sms, s));
    if (e != cudaSuccess) {
      set_error("copy_chunks", e);
      return ALIGN_E_CUDA;
    }
    ++nkernels;
    return ALIGN_OK;
  };
  // Large host batches move each launch's buffers on its own stream (copies
  // overlap other launches' kernels); small ones in one copy kernel each way.
  uint64_t in_bytes = 0;
  for (size_t k = 0; k < ih2d; ++k) in_bytes += hh2d[k].bytes;
  const bool split_copies = in_bytes > (64ull << 20);
  if (!split_copies && copy_range(dh2d, 0, ih2d, s0) != ALIGN_OK) return ALIGN_E_CUDA;
  cudaEvent_t ready = take_event(ctx);
  b.events.push_back(ready);
  CU(cudaEventRecord(ready, s0));
  size_t lane_i = 0;
  // Checkpointed sequences first (the longest utterances), then the groups.
  for (const CkLaunch& cl : cklaunch) {
    cudaStream_t s = cl.xlink ? ctx->grid_stream : used[lane_i++ % nwork];
    if (s != s0) CU(cudaStreamWaitEvent(s, ready, 0));
    const Plan& p = take[cl.req]->plan;
    const FwdParams P = plan_params(p.shape, static_cast<int>(take[cl.req]->C), p.frames_per_stage, ctx->wait_limit_ns);
    if (split_copies && copy_range(dh2d, cl.cr.in_first, cl.cr.in_count, s) != ALIGN_OK) return ALIGN_E_CUDA;
    for (size_t k = 0; k < cl.count; ++k) {
      if (cl.xlink) CU(cudaMemsetAsync(cl.xlink, 0, p.x_bytes, s));
      cudaError_t e = static_cast<cudaError_t>(launch_trellis(p.shape, P, djobs + cl.first + k, 1, s));
      if (e != cudaSuccess) {
        set_error("launch_trellis", e);
        return ALIGN_E_CUDA;
      }
      ++nkernels;
    }
    if (split_copies && copy_range(dd2h, cl.cr.out_first, cl.cr.out_count, s) != ALIGN_OK) return ALIGN_E_CUDA;
  }
  for (const GroupLaunch& gl : glaunch) {
    cudaStream_t s = used[lane_i++ % nwork];
    if (s != s0) CU(cudaStreamWaitEvent(s, ready, 0));
    const int C = hjobs[gl.first].C;
    const FwdParams P = plan_params(gl.shape, C, gl.F, ctx->wait_limit_ns);
    if (split_copies && copy_range(dh2d, gl.cr.in_first, gl.cr.in_count, s) != ALIGN_OK) return ALIGN_E_CUDA;
    cudaError_t e = static_cast<cudaError_t>(launch_trellis(gl.shape, P, djobs + gl.first, static_cast<int>(gl.count), s));
    if (e != cudaSuccess) {
      set_error("launch_trellis", e);
      return ALIGN_E_CUDA;
    }
    ++nkernels;
    if (split_copies && copy_range(dd2h, gl.cr.out_first, gl.cr.out_count, s) != ALIGN_OK) return ALIGN_E_CUDA;
  }
  // Join, download statuses and host outputs, record completion.
  for (cudaStream_t s : used) {
    if (s == s0) continue;
    cudaEvent_t j = take_event(ctx);
    b.events.push_back(j);
    CU(cudaEventRecord(j, s));
    CU(cudaStreamWaitEvent(s0, j, 0));
  }
  if (!split_copies && copy_range(dd2h, 0, id2h, s0) != ALIGN_OK) return ALIGN_E_CUDA;
  if (!direct) CU(cudaMemcpyAsync(b.h_meta, dmeta, take.size() * sizeof(MetaBlock), cudaMemcpyDeviceToHost, s0));

  for (size_t i = 0; i < take.size(); ++i) {
    Request& r = *take[i];
    if (!r.host_io || r.lp_alias) continue;
    const size_t T = static_cast<size_t>(r.T);
    if (r.out.path) CU(cudaMemcpyAsync(r.out.path, req_out[i].path, T * 4, cudaMemcpyDeviceToHost, s0));
    if (r.out.scores) CU(cudaMemcpyAsync(r.out.scores, req_out[i].scores, T * 4, cudaMemcpyDeviceToHost, s0));
    CU(cudaMemcpyAsync(r.out.total, req_out[i].total, 4, cudaMemcpyDeviceToHost, s0));
    if (r.out.states) CU(cudaMemcpyAsync(r.out.states, req_out[i].states, T * 4, cudaMemcpyDeviceToHost, s0));
  }
  return ALIGN_OK;
  };

  if (gi >= 0 && !need_capture) {
    const uint64_t nk = glaunch.size() + [&] {
      uint64_t c = 0;
      for (const CkLaunch& cl : cklaunch) c += cl.count;
      return c;
    }();
    CU(cudaGraphLaunch(ctx->graphs[static_cast<size_t>(gi)].exec, s0));
    ctx->stats.graph_launches++;
    ctx->stats.kernel_launches += nk;
  } else if (gi >= 0) {
    GraphEntry& ge = ctx->graphs[static_cast<size_t>(gi)];
    cudaGraph_t graph = nullptr;
    int rc = ALIGN_E_CUDA;
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      rc = body();
      const cudaError_t ce = cudaStreamEndCapture(s0, &graph);
      if (ce != cudaSuccess) rc = ALIGN_E_CUDA;
    }
    if (rc == ALIGN_OK && graph && cudaGraphInstantiate(&ge.exec, graph, 0) == cudaSuccess) {
      cudaGraphDestroy(graph);
      CU(cudaGraphLaunch(ge.exec, s0));
      ctx->stats.graph_launches++;
      ctx->stats.kernel_launches += nkernels;
    } else {
      // Capture not possible here: forget the entry's key and launch directly.
      if (graph) cudaGraphDestroy(graph);
      (void)cudaGetLastError();
      ge.exec = nullptr;
      ge.key.clear();
      nkernels = 0;
      rc = body();
      if (rc != ALIGN_OK) return rc;
      ctx->stats.kernel_launches += nkernels;
    }
  } else {
    const int rc = body();
    if (rc != ALIGN_OK) return rc;
    ctx->stats.kernel_launches += nkernels;
  }
  b.done = take_event(ctx);
  b.events.push_back(b.done);
  CU(cudaEventRecord(b.done, s0));
  ctx->batches.emplace(b.id, b);
  return ALIGN_OK;
}

// One persistent launch over the admitted requests (all planned by
// choose_persist with one shape): descriptors in seat order (longest chain
// first), the seat table and the seat counter in one upload; the teams' CTA
// links in one zeroed region of the backpointer arena.
int launch_persistent(align_ctx* ctx, std::vector<Request*>& take) {
  std::stable_sort(take.begin(), take.end(), [](const Request* a, const Request* b) { return a->T > b->T; });
  const size_t n = take.size();
  const LaunchShape shape = [&] {
    LaunchShape sh = take[0]->plan.shape;
    sh.ncta = 1;
    return sh;
  }();
  const int C = static_cast<int>(take[0]->C);
  const int F = take[0]->plan.frames_per_stage;
  const FwdParams P = plan_params(shape, C, F, ctx->wait_limit_ns);
  int64_t total_seats = 0;
  uint64_t x_bytes = 0, tgt_words = 0;
  std::vector<uint64_t> x_off(n, 0);
  for (size_t i = 0; i < n; ++i) {
    const int ncta = take[i]->plan.shape.ncta;
    total_seats += ncta;
    if (ncta > 1) {
      x_off[i] = x_bytes;
      x_bytes += fast_xlink_bytes(ncta, P.kb);
    }
    tgt_words += round_up(static_cast<uint64_t>(std::max<int64_t>(take[i]->L, 1)), 4);
  }
  const uint64_t off_jobs = 0;
  const uint64_t off_metas = round_up(n * sizeof(FwdJob), kAlign);
  const uint64_t off_tgts = round_up(off_metas + n * sizeof(MetaBlock), kAlign);
  const uint64_t off_seats = round_up(off_tgts + tgt_words * 4, kAlign);
  const uint64_t up_bytes = round_up(off_seats + static_cast<uint64_t>(total_seats) * 4, kAlign);
  // Direct image (as for shape-group batches): the kernel reads the
  // descriptors, targets and seat table from the pinned image and writes the
  // result codes there. Otherwise the image is uploaded and the codes copied back.
  const bool direct = ctx->d_pinned != nullptr;
  const uint64_t pin_bytes = direct ? up_bytes : up_bytes + round_up(n * sizeof(MetaBlock), kAlign);
  // Device region zeroed before the launch: the teams' CTA links, then the seat counter.
  const uint64_t off_counter = round_up(x_bytes, kAlign);
  const uint64_t dev_bytes = off_counter + kAlign;

  Batch b;
  b.id = ctx->next_batch++;
  auto unwind = [&]() {
    if (b.meta.live) ctx->meta_arena.release(b.meta.off, b.meta.bytes), b.meta.live = false;
    if (b.pinned.live) ctx->pinned_arena.release(b.pinned.off, b.pinned.bytes), b.pinned.live = false;
    if (b.xlink.live) ctx->bp_arena.release(b.xlink.off, b.xlink.bytes), b.xlink.live = false;
    for (auto it = take.rbegin(); it != take.rend(); ++it) {
      Request* r = *it;
      if (r->bp.live) ctx->bp_arena.release(r->bp.off, r->bp.bytes), r->bp.live = false;
      ctx->queued.push_front(r->id);
    }
    return ALIGN_OK;  // retried after other batches release memory
  };
  if (!direct) {
    if (!ctx->meta_arena.alloc(up_bytes, &b.meta.off)) return unwind();
    b.meta.bytes = up_bytes;
    b.meta.live = true;
  }
  if (!ctx->pinned_arena.alloc(pin_bytes, &b.pinned.off)) return unwind();
  b.pinned.bytes = pin_bytes;
  b.pinned.live = true;
  if (!ctx->bp_arena.alloc(dev_bytes, &b.xlink.off)) return unwind();
  b.xlink.bytes = dev_bytes;
  b.xlink.live = true;
  char* h = ctx->h_pinned + b.pinned.off;
  char* d = direct ? ctx->d_pinned + b.pinned.off : ctx->d_meta + b.meta.off;
  FwdJob* hjobs = reinterpret_cast<FwdJob*>(h + off_jobs);
  MetaBlock* hmeta = reinterpret_cast<MetaBlock*>(h + off_metas);
  int32_t* htgt = reinterpret_cast<int32_t*>(h + off_tgts);
  int32_t* hseat = reinterpret_cast<int32_t*>(h + off_seats);
  MetaBlock* dmeta = reinterpret_cast<MetaBlock*>(d + off_metas);
  const int32_t* dtgt = reinterpret_cast<const int32_t*>(d + off_tgts);
  b.h_meta = reinterpret_cast<MetaBlock*>(direct ? h + off_metas : h + up_bytes);
  char* d_x = ctx->d_bp + b.xlink.off;
  uint64_t tw = 0;
  int32_t seat = 0;
  for (size_t i = 0; i < n; ++i) {
    Request& r = *take[i];
    const Plan& p = r.plan;
    r.state = ReqState::Launched;
    r.batch = b.id;
    r.meta_index = static_cast<int>(i);
    b.reqs.push_back(r.id);
    hmeta[i].status = ALIGN_PENDING;
    hmeta[i].state_io = 0;
    hmeta[i].final2[0] = hmeta[i].final2[1] = -INFINITY;
    b.h_meta[i].status = ALIGN_PENDING;
    if (r.L) std::memcpy(htgt + tw, r.targets.data(), static_cast<size_t>(r.L) * 4);
    FwdJob j{};
    j.lp = r.lp;
    j.tgt = dtgt + tw;
    tw += round_up(static_cast<uint64_t>(std::max<int64_t>(r.L, 1)), 4);
    j.status = &dmeta[i].status;
    j.state_io = &dmeta[i].state_io;
    j.final2 = dmeta[i].final2;
    j.path = r.out.path;
    j.scores = r.out.scores;
    j.total = r.out.total;
    j.states = r.out.states;
    j.T = static_cast<int32_t>(r.T);
    j.C = static_cast<int32_t>(r.C);
    j.blank = r.blank;
    j.L = static_cast<int32_t>(r.L);
    j.S = static_cast<int32_t>(2 * r.L + 1);
    j.flags = kJobBulkRows | kJobWriteFinal | kJobChase | ((ctx->flags & ALIGN_F_TEST_STALL) ? kJobTestStall : 0u);
    j.bp = reinterpret_cast<uint32_t*>(ctx->d_bp + r.bp.off);
    j.ztab = reinterpret_cast<uint8_t*>(ctx->d_bp + r.bp.off + p.z_off);
    j.zstride = p.zstride;
    j.t_begin = 0;
    j.t_end = j.T;
    j.bp_rows = std::max(j.T - 1, 0);
    j.xlink = p.shape.ncta > 1 ? reinterpret_cast<uint64_t*>(d_x + x_off[i]) : nullptr;
    j.team_ctas = p.shape.ncta;
    j.first_seat = seat;
    for (int c = 0; c < p.shape.ncta; ++c) hseat[seat++] = static_cast<int32_t>(i);
    hjobs[i] = j;
  }

  // One idle worker stream (the batch forks from the main stream).
  cudaStream_t s0 = nullptr;
  for (size_t k = 0; k < ctx->workers.size() && !s0; ++k) {
    cudaStream_t s = ctx->workers[(static_cast<size_t>(ctx->next_worker) + k) % ctx->workers.size()];
    if (cudaStreamQuery(s) == cudaSuccess) s0 = s;
  }
  ctx->next_worker = static_cast<int>((static_cast<size_t>(ctx->next_worker) + 1) % ctx->workers.size());
  if (!s0 && ctx->workers.size() < kMaxStreams) {
    CU(cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking));
    ctx->workers.push_back(s0);
  }
  if (!s0) s0 = ctx->workers[static_cast<size_t>(ctx->next_worker) % ctx->workers.size()];
  cudaEvent_t fork = ctx->fork_events[static_cast<size_t>(b.id) % ctx->fork_events.size()];
  CU(cudaEventRecord(fork, ctx->main));
  CU(cudaStreamWaitEvent(s0, fork, 0));
  if (!direct) CU(cudaMemcpyAsync(d, h, up_bytes, cudaMemcpyHostToDevice, s0));
  CU(cudaMemsetAsync(d_x, 0, dev_bytes, s0));
  const int ctas = persist_ctas(ctx, shape, C, F);
  const cudaError_t e = static_cast<cudaError_t>(
      launch_trellis_persist(shape, P, reinterpret_cast<const FwdJob*>(d + off_jobs),
                             reinterpret_cast<const int32_t*>(d + off_seats), static_cast<int32_t>(total_seats),
                             reinterpret_cast<int32_t*>(d_x + off_counter), ctas, s0));
  if (e != cudaSuccess) {
    set_error("launch_trellis_persist", e);
    return ALIGN_E_CUDA;
  }
  if (!direct) CU(cudaMemcpyAsync(b.h_meta, dmeta, n * sizeof(MetaBlock), cudaMemcpyDeviceToHost, s0));
  ctx->stats.kernel_launches += 1;
  ctx->stats.persistent_batches++;
  ctx->stats.bp_bytes_peak = std::max(ctx->stats.bp_bytes_peak, ctx->bp_arena.peak());
  b.done = take_event(ctx);
  b.events.push_back(b.done);
  CU(cudaEventRecord(b.done, s0));
  ctx->batches.emplace(b.id, b);
  return ALIGN_OK;
}

int pump(align_ctx* ctx, bool launch) {
  int rc = reap(ctx);
  if (rc != ALIGN_OK) return rc;
  if (launch) {
    rc = launch_queued(ctx);
    if (rc != ALIGN_OK) return rc;
  }
  return ALIGN_OK;
}

// Queues one request; then (unless `pump_after` is false, as for the
// requests of one batch call, which pump once at its end) retires finished
// batches and, outside batched mode, launches.
// `tp_plan`: plan with the throughput table (the table the batch will be
// launched with), so that the launch need not plan the request again.
int submit_common(align_ctx* ctx, const float* lp, int64_t T, int64_t C, const int32_t* targets, int64_t L,
                  int32_t blank, align_out out, uint64_t* request_id, bool host_io, bool logits = false,
                  bool sum = false, bool pump_after = true, bool tp_plan = false) {
  if (!ctx || !lp || !request_id || !out.total || (!sum && (!out.path || !out.scores))) return ALIGN_E_INVAL;
  if (sum && logits) return ALIGN_E_INVAL;  // the sum-product path takes log-probabilities
  if (sum) out.path = nullptr, out.scores = nullptr, out.states = nullptr;
  if (L > 0 && !targets) return ALIGN_E_INVAL;
  // Frame tags in the ring words have 24 bits; 2^24 frames of 20 ms are 93 hours.
  if (T >= (1ll << kTagBits) || L > INT32_MAX / 4) return ALIGN_E_TOO_LARGE;
  int64_t R = 0;
  int rc = validate_request(targets, L, C, blank, T, &R);
  if (rc != ALIGN_OK) return rc;
  if (ctx->flags & ALIGN_F_DEBUG_CHECKS) {  // NaN / +inf scan of the emissions
    const int64_t nv = T * C;
    const float* dv = host_io ? static_cast<const float*>(device_alias(ctx, lp)) : lp;
    if (host_io && !dv) {
      for (int64_t i = 0; i < nv; ++i)
        if (std::isnan(lp[i]) || lp[i] == INFINITY) return ALIGN_E_NONFINITE;
    } else {
      const int e = launch_scan_nonfinite(dv, nv, ctx->d_check, ctx->num_sms, ctx->main);
      if (e != cudaSuccess) return set_error("scan_nonfinite", static_cast<cudaError_t>(e)), ALIGN_E_CUDA;
      CU(cudaMemcpyAsync(ctx->h_check, ctx->d_check, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->main));
      CU(cudaStreamSynchronize(ctx->main));
      if (*ctx->h_check) return ALIGN_E_NONFINITE;
    }
  }
  if (static_cast<int64_t>(inflight_count(ctx)) >= ctx->max_inflight) {
    rc = pump(ctx, true);
    if (rc != ALIGN_OK) return rc;
    if (static_cast<int64_t>(inflight_count(ctx)) >= ctx->max_inflight) return ALIGN_E_AGAIN;
  }
  Plan p{};
  tp_plan = tp_plan && ctx->tune_tp.nbuckets != 0;
  rc = plan_request(ctx, tp_plan ? ctx->tune_tp : ctx->tune, T, C, L, logits, &p, sum);
  if (rc != ALIGN_OK && tp_plan) {  // the throughput table cannot place it: the latency table's plan
    tp_plan = false;
    rc = plan_request(ctx, ctx->tune, T, C, L, logits, &p, sum);
  }
  if (rc != ALIGN_OK) return rc;
  if (tp_plan) p.shape.occ = 1;
  Request r;
  r.logits = logits;
  r.sum = sum;
  if (host_io) {
    align_out al{};
    const void* la = device_alias(ctx, lp);
    al.path = static_cast<int32_t*>(device_alias(ctx, out.path));
    al.scores = static_cast<float*>(device_alias(ctx, out.scores));
    al.total = static_cast<float*>(device_alias(ctx, out.total));
    al.states = out.states ? static_cast<int32_t*>(device_alias(ctx, out.states)) : nullptr;
    if (la && (al.path || !out.path) && (al.scores || !out.scores) && al.total && (!out.states || al.states)) {
      r.lp_alias = la;
      r.out_alias = al;
    }
    if (host_stage_bytes(T, C) > ctx->stage_arena.cap()) return ALIGN_E_TOO_LARGE;
  }
  r.id = ctx->next_id++;
  r.lp = lp;
  r.host_io = host_io;
  r.out = out;
  r.T = T;
  r.C = C;
  r.L = L;
  r.blank = blank;
  r.targets.assign(targets, targets + L);
  r.plan = p;
  r.plan_table = tp_plan ? ALIGN_TUNE_THROUGHPUT : ALIGN_TUNE_LATENCY;
  *request_id = r.id;
  ctx->reqs.emplace(r.id, std::move(r));
  ctx->queued.push_back(*request_id);
  if (!pump_after) return ALIGN_OK;
  const bool launch_now = !(ctx->flags & ALIGN_F_BATCHED);
  return pump(ctx, launch_now);
}

}  // namespace

// ------------------------------------------------------------------ C ABI --
extern "C" {

int align_create(align_ctx** out, const align_config* cfg_in) {
  if (!out) return ALIGN_E_INVAL;
  *out = nullptr;
  align_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (cfg.device < 0 || cfg.device >= ndev) return ALIGN_E_INVAL;
  CU(cudaSetDevice(cfg.device));
  std::unique_ptr<align_ctx> ctx(new align_ctx());
  ctx->device = cfg.device;
  ctx->flags = cfg.flags;
  ctx->max_inflight = cfg.max_inflight > 0 ? cfg.max_inflight : 8192;
  ctx->wait_limit_ns = static_cast<uint64_t>(cfg.wait_limit_ms ? cfg.wait_limit_ms : 2000) * 1000000ull;
  CU(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, cfg.device));
  ctx->smem_optin = max_smem_optin(cfg.device);
  ctx->tune = default_tune_table();
  int coop = 0;
  CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, cfg.device));
  int ats = 0;
  CU(cudaDeviceGetAttribute(&ats, cudaDevAttrPageableMemoryAccessUsesHostPageTables, cfg.device));
  ctx->host_ats = ats != 0;
  // Grid teams for latency-planned batches only: a team holds whole SMs, and
  // batches that oversubscribe the GPU are better served by clusters.
  if (coop && !(cfg.flags & ALIGN_F_NO_GRID_TEAMS)) ctx->tune.max_grid = ctx->num_sms;
  const uint64_t bp_bytes = cfg.bp_budget_bytes ? cfg.bp_budget_bytes : (1ull << 30);
  const uint64_t stage_bytes = cfg.staging_bytes ? cfg.staging_bytes : (64ull << 20);
  const uint64_t meta_bytes = 64ull << 20;
  const uint64_t pin_bytes = 64ull << 20;
  if (cudaMalloc(&ctx->d_bp, bp_bytes) != cudaSuccess) return ALIGN_E_NOMEM;
  ctx->bp_arena.init(bp_bytes);
  if (cudaMalloc(&ctx->d_meta, meta_bytes) != cudaSuccess) {
    cudaFree(ctx->d_bp);
    return ALIGN_E_NOMEM;
  }
  ctx->meta_arena.init(meta_bytes);
  if (cudaMalloc(&ctx->d_stage, stage_bytes) != cudaSuccess) {
    cudaFree(ctx->d_bp);
    cudaFree(ctx->d_meta);
    return ALIGN_E_NOMEM;
  }
  ctx->stage_arena.init(stage_bytes);
  if (cudaMallocHost(&ctx->h_pinned, pin_bytes) != cudaSuccess) {
    cudaFree(ctx->d_bp);
    cudaFree(ctx->d_meta);
    cudaFree(ctx->d_stage);
    return ALIGN_E_NOMEM;
  }
  ctx->pinned_arena.init(pin_bytes);
  {
    // Direct images: kernels read a batch's descriptors from the pinned
    // arena and update its result codes there (atomics on host memory).
    void* alias = nullptr;
    int host_atomics = 0;
    if (!(cfg.flags & ALIGN_F_UPLOAD_DESCRIPTORS) &&
        cudaDeviceGetAttribute(&host_atomics, cudaDevAttrHostNativeAtomicSupported, cfg.device) == cudaSuccess &&
        host_atomics && cudaHostGetDevicePointer(&alias, ctx->h_pinned, 0) == cudaSuccess)
      ctx->d_pinned = static_cast<char*>(alias);
    (void)cudaGetLastError();
  }
  if (cudaMalloc(&ctx->d_check, 256) != cudaSuccess || cudaMallocHost(&ctx->h_check, 256) != cudaSuccess) {
    cudaFree(ctx->d_bp);
    cudaFree(ctx->d_meta);
    cudaFree(ctx->d_stage);
    cudaFree(ctx->d_check);
    cudaFreeHost(ctx->h_pinned);
    return ALIGN_E_NOMEM;
  }
  if (cfg.cuda_stream) {
    ctx->main = static_cast<cudaStream_t>(cfg.cuda_stream);
  } else {
    CU(cudaStreamCreateWithFlags(&ctx->main, cudaStreamNonBlocking));
    ctx->own_main = true;
  }
  for (int i = 0; i < 16; ++i) {
    cudaStream_t s;
    CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ctx->workers.push_back(s);
  }
  CU(cudaStreamCreateWithFlags(&ctx->grid_stream, cudaStreamNonBlocking));
  for (int i = 0; i < 64; ++i) {
    cudaEvent_t e;
    CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->fork_events.push_back(e);
  }
  *out = ctx.release();
  return ALIGN_OK;
}

int align_destroy(align_ctx* ctx) {
  if (!ctx) return ALIGN_OK;
  cudaSetDevice(ctx->device);
  for (auto& kv : ctx->batches) cudaEventSynchronize(kv.second.done);
  for (auto& kv : ctx->batches)
    for (cudaEvent_t e : kv.second.events) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  for (GraphEntry& ge : ctx->graphs)
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
  for (cudaStream_t s : ctx->workers) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (ctx->grid_stream) {
    cudaStreamSynchronize(ctx->grid_stream);
    cudaStreamDestroy(ctx->grid_stream);
  }
  for (cudaEvent_t e : ctx->fork_events) cudaEventDestroy(e);
  if (ctx->own_main) {
    cudaStreamSynchronize(ctx->main);
    cudaStreamDestroy(ctx->main);
  }
  cudaFree(ctx->d_bp);
  cudaFree(ctx->d_meta);
  cudaFree(ctx->d_stage);
  cudaFreeHost(ctx->h_pinned);
  cudaFree(ctx->d_check);
  cudaFreeHost(ctx->h_check);
  delete ctx;
  return ALIGN_OK;
}

int align_submit(align_ctx* ctx, const float* log_probs, int64_t T, int64_t C, const int32_t* targets, int64_t L,
                 int32_t blank, align_out out, uint64_t* request_id) {
  if (ctx) cudaSetDevice(ctx->device);
  return submit_common(ctx, log_probs, T, C, targets, L, blank, out, request_id, false);
}

int align_submit_host(align_ctx* ctx, const float* log_probs, int64_t T, int64_t C, const int32_t* targets,
                      int64_t L, int32_t blank, align_out out, uint64_t* request_id) {
  if (ctx) cudaSetDevice(ctx->device);
  return submit_common(ctx, log_probs, T, C, targets, L, blank, out, request_id, true);
}

int align_submit_batch(align_ctx* ctx, int32_t n, const align_request* reqs, uint64_t* request_ids,
                       int32_t* submit_status) {
  if (!ctx || n < 0 || (n > 0 && (!reqs || !request_ids))) return ALIGN_E_INVAL;
  cudaSetDevice(ctx->device);
  // Queue every request without launching, then launch once: one batch.
  // The table the batch will most likely be launched with (the rule of
  // want_throughput over the queued requests and these) plans them at once.
  bool tp_plan = false;
  if (ctx->tune_tp.nbuckets != 0 && ctx->queued.size() + static_cast<size_t>(n) >= 2) {
    uint64_t work = 0;
    int64_t tmax = 0;
    for (uint64_t id : ctx->queued) {
      const Request& r = ctx->reqs.at(id);
      work += static_cast<uint64_t>(r.T) * static_cast<uint64_t>((2 * r.L + 1 + 63) / 64);
      tmax = std::max(tmax, r.T);
    }
    for (int32_t i = 0; i < n; ++i) {
      if (reqs[i].T < 1 || reqs[i].L < 0) continue;
      work += static_cast<uint64_t>(reqs[i].T) * static_cast<uint64_t>((2 * reqs[i].L + 1 + 63) / 64);
      tmax = std::max<int64_t>(tmax, reqs[i].T);
    }
    tp_plan = work > static_cast<uint64_t>(tmax) * 8ull * static_cast<uint64_t>(std::max(1, ctx->num_sms));
  }
  const uint32_t saved = ctx->flags;
  ctx->flags |= ALIGN_F_BATCHED;
  int first_err = ALIGN_OK;
  for (int32_t i = 0; i < n; ++i) {
    const align_request& q = reqs[i];
    int rc = (q.flags & ~(ALIGN_REQ_HOST | ALIGN_REQ_LOGITS | ALIGN_REQ_SUM))
                 ? ALIGN_E_INVAL
                 : submit_common(ctx, q.log_probs, q.T, q.C, q.targets, q.L, q.blank, q.out, &request_ids[i],
                                 (q.flags & ALIGN_REQ_HOST) != 0, (q.flags & ALIGN_REQ_LOGITS) != 0,
                                 (q.flags & ALIGN_REQ_SUM) != 0, /*pump_after=*/false, tp_plan);
    if (rc != ALIGN_OK) request_ids[i] = 0;
    if (submit_status) submit_status[i] = rc;
    if (rc != ALIGN_OK && first_err == ALIGN_OK) first_err = rc;
  }
  ctx->flags = saved;
  // One retire pass for the whole call (and the launch, outside batched mode).
  const int rc = pump(ctx, !(saved & ALIGN_F_BATCHED));
  if (rc != ALIGN_OK) return rc;
  return first_err;
}

int align_flush(align_ctx* ctx) {
  if (!ctx) return ALIGN_E_INVAL;
  cudaSetDevice(ctx->device);
  return pump(ctx, true);
}

int align_poll(align_ctx* ctx, uint64_t request_id, int32_t timeout_ms, int32_t* request_status) {
  if (!ctx) return ALIGN_E_INVAL;
  cudaSetDevice(ctx->device);
  auto it = ctx->reqs.find(request_id);
  if (it == ctx->reqs.end()) return ALIGN_E_NOTFOUND;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    int rc = pump(ctx, true);
    if (rc != ALIGN_OK) return rc;
    Request& r = ctx->reqs.at(request_id);
    if (r.state == ReqState::Done) {
      if (request_status) *request_status = r.status;
      ctx->reqs.erase(request_id);
      return ALIGN_OK;
    }
    if (timeout_ms == 0) return ALIGN_PENDING;
    if (timeout_ms > 0) {
      const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
      if (el.count() >= timeout_ms) return ALIGN_PENDING;
    }
    if (r.state == ReqState::Launched) {
      Batch& b = ctx->batches.at(r.batch);
      // Block on the event for up to the remaining time (spin-sleep keeps the timeout honoured).
      if (timeout_ms < 0) {
        cudaError_t e = cudaEventSynchronize(b.done);
        if (e != cudaSuccess) {
          set_error("cudaEventSynchronize", e);
          return ALIGN_E_CUDA;
        }
      } else {
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    } else if (r.state == ReqState::Queued) {
      // Waiting for memory held by running batches; with nothing running it can never fit.
      if (ctx->batches.empty()) {
        ctx->queued.erase(std::remove(ctx->queued.begin(), ctx->queued.end(), request_id), ctx->queued.end());
        ctx->reqs.erase(request_id);
        return ALIGN_E_TOO_LARGE;
      }
      if (timeout_ms < 0) {
        cudaEventSynchronize(ctx->batches.begin()->second.done);
      } else {
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    }
  }
}

int align_probe_frame_latency(int32_t device, int32_t warps, int32_t ctas, int32_t frames, double* ns_per_frame) {
  if (!ns_per_frame || warps < 1 || warps > 32 || ctas < 1 || ctas > 16 || frames < 2) return ALIGN_E_INVAL;
  CU(cudaSetDevice(device));
  uint64_t* d = nullptr;
  CU(cudaMalloc(&d, 3 * sizeof(uint64_t)));
  uint64_t h[3] = {0, 0, 0};
  cudaError_t e = static_cast<cudaError_t>(launch_frame_probe(warps, ctas, frames, 2000000000ull, d, nullptr));
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("frame probe", e);
    return ALIGN_E_CUDA;
  }
  if (h[1]) return ALIGN_E_TIMEOUT;
  *ns_per_frame = static_cast<double>(h[0]) / static_cast<double>(frames);
  return ALIGN_OK;
}

int align_poll_done(align_ctx* ctx, uint64_t* ids, int32_t* statuses, int32_t max, int32_t* count) {
  if (!ctx || !count || max < 0 || (max > 0 && (!ids || !statuses))) return ALIGN_E_INVAL;
  cudaSetDevice(ctx->device);
  const int rc = pump(ctx, true);
  if (rc != ALIGN_OK) return rc;
  int32_t n = 0;
  for (auto it = ctx->reqs.begin(); it != ctx->reqs.end() && n < max;) {
    if (it->second.state == ReqState::Done) {
      ids[n] = it->first;
      statuses[n] = it->second.status;
      ++n;
      it = ctx->reqs.erase(it);
    } else {
      ++it;
    }
  }
  *count = n;
  return ALIGN_OK;
}

int align_join(align_ctx* ctx, void* stream) {
  if (!ctx) return ALIGN_E_INVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->main;
  for (auto& kv : ctx->batches) CU(cudaStreamWaitEvent(s, kv.second.done, 0));
  return ALIGN_OK;
}

int align_get_stats(align_ctx* ctx, align_stats* out, int32_t reset) {
  if (!ctx || !out) return ALIGN_E_INVAL;
  ctx->stats.bp_bytes_peak = std::max(ctx->stats.bp_bytes_peak, ctx->bp_arena.peak());
  *out = ctx->stats;
  if (reset) {
    ctx->stats = align_stats{};
    ctx->bp_arena.reset_peak();
  }
  return ALIGN_OK;
}

const char* align_status_string(int32_t code) {
  switch (code) {
    case ALIGN_OK: return "ALIGN_OK";
    case ALIGN_PENDING: return "ALIGN_PENDING";
    case ALIGN_E_INVAL: return "ALIGN_E_INVAL";
    case ALIGN_E_TARGET: return "ALIGN_E_TARGET";
    case ALIGN_E_INFEASIBLE: return "ALIGN_E_INFEASIBLE";
    case ALIGN_E_TOO_LARGE: return "ALIGN_E_TOO_LARGE";
    case ALIGN_E_AGAIN: return "ALIGN_E_AGAIN";
    case ALIGN_E_NOPATH: return "ALIGN_E_NOPATH";
    case ALIGN_E_TIMEOUT: return "ALIGN_E_TIMEOUT";
    case ALIGN_E_CUDA: return "ALIGN_E_CUDA";
    case ALIGN_E_NOTFOUND: return "ALIGN_E_NOTFOUND";
    case ALIGN_E_NOMEM: return "ALIGN_E_NOMEM";
    case ALIGN_E_NONFINITE: return "ALIGN_E_NONFINITE";
    default: return "ALIGN_E_UNKNOWN";
  }
}

const char* align_last_error(void) { return g_last_error; }

int align_set_tuning_bucket(align_ctx* ctx, int32_t s_max, int32_t states_per_lane, int32_t cta_warps) {
  return align_set_tuning_bucket_for(ctx, ALIGN_TUNE_LATENCY, s_max, states_per_lane, cta_warps);
}

int align_set_tuning_bucket_for(align_ctx* ctx, int32_t table, int32_t s_max, int32_t states_per_lane,
                                int32_t cta_warps) {
  if (!ctx || (table != ALIGN_TUNE_LATENCY && table != ALIGN_TUNE_THROUGHPUT)) return ALIGN_E_INVAL;
  TuneTable& t = (table == ALIGN_TUNE_LATENCY) ? ctx->tune : ctx->tune_tp;
  if (s_max <= 0) {  // clear the table
    t.nbuckets = 0;
    return ALIGN_OK;
  }
  if ((states_per_lane != 2 && states_per_lane != 4 && states_per_lane != 8 && states_per_lane != 16) ||
      cta_warps < 1 || cta_warps > 16)
    return ALIGN_E_INVAL;
  for (int i = 0; i < t.nbuckets; ++i) {
    if (t.buckets[i].s_max == s_max) {
      t.buckets[i] = TuneBucket{s_max, states_per_lane, cta_warps};
      return ALIGN_OK;
    }
  }
  if (t.nbuckets >= 16) return ALIGN_E_AGAIN;
  t.buckets[t.nbuckets++] = TuneBucket{s_max, states_per_lane, cta_warps};
  std::sort(t.buckets, t.buckets + t.nbuckets, [](const TuneBucket& a, const TuneBucket& b) { return a.s_max < b.s_max; });
  return ALIGN_OK;
}

int align_set_tuning(align_ctx* ctx, int32_t states_per_lane, int32_t cta_warps, int32_t max_cluster) {
  if (!ctx) return ALIGN_E_INVAL;
  if (states_per_lane && states_per_lane != 2 && states_per_lane != 4 && states_per_lane != 8 &&
      states_per_lane != 16)
    return ALIGN_E_INVAL;
  if (cta_warps < 0 || cta_warps > 32 || max_cluster < 0 || max_cluster > 16) return ALIGN_E_INVAL;
  for (TuneTable* t : {&ctx->tune, &ctx->tune_tp}) {  // the defaults of both tables
    if (states_per_lane) t->K = states_per_lane;
    if (cta_warps) t->cta_warps = cta_warps;
    if (max_cluster) t->max_cluster = max_cluster;
  }
  return ALIGN_OK;
}

}  // extern "C"
