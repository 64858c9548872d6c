// Validation (step A1) and planning of a request: kernel shape, emission
// staging depth and memory footprint of full or checkpointed backpointers.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "../../include/align.h"
#include "align_internal.h"

namespace gb300_align {

namespace {
inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline uint64_t round_up(uint64_t v, uint64_t a) { return ceil_div(v, a) * a; }
}  // namespace

TuneTable default_tune_table() { return TuneTable{}; }

TuneTable resolve_tuning(const TuneTable& t, int64_t S) {
  TuneTable r = t;
  for (int i = 0; i < t.nbuckets; ++i) {
    if (S <= t.buckets[i].s_max) {
      r.K = t.buckets[i].K;
      r.cta_warps = t.buckets[i].cta_warps;
      break;
    }
  }
  return r;
}

int validate_request(const int32_t* targets, int64_t L, int64_t C, int32_t blank, int64_t T, int64_t* repeats) {
  if (T < 1 || C < 2 || L < 0 || blank < 0 || blank >= C) return ALIGN_E_INVAL;
  if (L > 0 && targets == nullptr) return ALIGN_E_INVAL;
  int64_t R = 0;
  for (int64_t i = 0; i < L; ++i) {
    const int32_t v = targets[i];
    if (v < 0 || v >= C || v == blank) return ALIGN_E_TARGET;
    if (i > 0 && v == targets[i - 1]) ++R;
  }
  if (repeats) *repeats = R;
  if (T < L + R) return ALIGN_E_INFEASIBLE;
  return ALIGN_OK;
}

int make_plan(const TuneTable& tune_in, int64_t T, int64_t C, int64_t L, uint64_t budget, bool force_checkpoint,
              Plan* out) {
  Plan p{};
  const int64_t S = 2 * L + 1;
  const TuneTable tune = resolve_tuning(tune_in, S);
  // Shape: one CTA of up to cta_warps warps, else a cluster of CTAs of at most
  // cta_warps warps (portable sizes first), else wider CTAs and larger K.
  const int K = tune.K;
  // The fast kernel (K = 2 or 4, C <= 512) adds a producer warp to each CTA of
  // compute warps, so it takes at most 15 of them; the generic kernel 16.
  const auto warp_cap = [&](int k) {
    const bool fast_k = (k == 2 || k == 4) && C <= 512;
    return std::min(fast_k ? 15 : 16, tune.max_warps);
  };
  const int portable = std::min(8, tune.max_cluster);
  // Transcripts beyond a cluster of the tuned K become grid teams (one CTA
  // per SM, linked through global memory) when the device has the SMs, before
  // K grows to 8 or 16 states per lane. A grid team spreads over as many SMs
  // as it can: the fewest warps per CTA (at most 16) that fit on max_grid SMs,
  // since the warps of one SM share its issue slots.
  struct Try {
    int k, wcap, cmax, grid;
  };
  const int cw = std::max(1, std::min(tune.cta_warps, warp_cap(K)));
  const Try tries[] = {{K, cw, portable, 0},
                       {K, cw, tune.max_cluster, 0},
                       {K, warp_cap(K), tune.max_grid, 1},
                       {K, warp_cap(K), portable, 0},
                       {K, warp_cap(K), tune.max_cluster, 0},
                       {8, warp_cap(8), portable, 0},
                       {8, warp_cap(8), tune.max_cluster, 0},
                       {8, warp_cap(8), tune.max_grid, 1},
                       {16, warp_cap(16), tune.max_cluster, 0},
                       {16, warp_cap(16), tune.max_grid, 1}};
  bool found = false;
  for (const Try& tr : tries) {
    if (tr.k < K || tr.cmax < 1) continue;
    const uint64_t G = ceil_div(static_cast<uint64_t>(S), 32ull * tr.k);
    const uint64_t wcap = tr.grid ? std::min<uint64_t>(static_cast<uint64_t>(tr.wcap),
                                                       std::max<uint64_t>(1, ceil_div(G, static_cast<uint64_t>(tr.cmax))))
                                  : static_cast<uint64_t>(tr.wcap);
    const uint64_t ncta = ceil_div(G, wcap);
    if (ncta <= static_cast<uint64_t>(tr.cmax)) {
      p.shape = LaunchShape{tr.k, static_cast<int>(ceil_div(G, ncta)), static_cast<int>(ncta)};
      p.shape.grid = tr.grid;
      found = true;
      break;
    }
  }
  if (!found) return ALIGN_E_TOO_LARGE;
  return plan_footprint(T, C, L, budget, force_checkpoint, &p, out);
}

int make_persist_plan(int K, int warps, int64_t T, int64_t C, int64_t L, uint64_t budget, Plan* out) {
  if ((K != 2 && K != 4) || warps < 1 || warps > 15 || C > 512) return ALIGN_E_INVAL;
  Plan p{};
  const uint64_t S = static_cast<uint64_t>(2 * L + 1);
  const uint64_t ncta = ceil_div(S, 32ull * K * static_cast<uint64_t>(warps));
  p.shape = LaunchShape{K, warps, static_cast<int>(ncta)};
  p.shape.grid = 1;  // CTAs of a team link through global memory
  const int rc = plan_footprint(T, C, L, budget, false, &p, out);
  if (rc != ALIGN_OK) return rc;
  if (out->checkpointed) return ALIGN_E_TOO_LARGE;  // persistent launches keep full backpointers
  out->shape.persist = 1;
  out->x_bytes = 0;  // the links of a persistent batch are one region of the batch
  return ALIGN_OK;
}

// Footprint and staging of a request whose kernel shape (K, warps, CTAs,
// grid) is set in *p.
int plan_footprint(int64_t T, int64_t C, int64_t L, uint64_t budget, bool force_checkpoint, Plan* pp, Plan* out) {
  Plan& p = *pp;
  const int64_t S = 2 * L + 1;
  // The fast Viterbi kernel serves K = 2 or 4 with at least 4 frames per
  // emission stage (C <= 512); its stages are 8 KB. Other shapes (and the
  // sum-product, and logits requests that run checkpointed) use the generic
  // kernel.
  const bool fast = (p.shape.K == 2 || p.shape.K == 4) && C <= 512;
  p.shape.fast = fast ? 1 : 0;
  // Emission staging: stages of 4 KB (32 frames of a 32-class row), up to 8 KB
  // for wide rows; frames per stage a power of two dividing the anchor window.
  const int64_t stage_budget = (fast || p.shape.warps >= 2) ? 8192 : 4096;
  const int64_t fmax = std::clamp<int64_t>(stage_budget / (4 * C), 1, kAnchorD);
  p.frames_per_stage = 1;
  while (p.frames_per_stage * 2 <= fmax) p.frames_per_stage *= 2;
  const uint64_t warps = static_cast<uint64_t>(p.shape.warps) * p.shape.ncta;
  const uint64_t row_bytes = warps * bp_words(p.shape.K) * 4ull;
  // Anchor rows: one row of S bytes (rounded to 16) per kAnchorD frames.
  p.zstride = static_cast<int>(round_up(static_cast<uint64_t>(S), 16));
  const auto zrows = [](int64_t frames) { return static_cast<uint64_t>((frames + kAnchorD - 1) / kAnchorD); };
  // Backpointer words: per frame (generic layout) or per whole window of
  // kAnchorD frames (fast layout); sized for whole windows, which covers both.
  p.z_off = round_up(row_bytes * zrows(T - 1) * kAnchorD, 256);
  p.bp_bytes = p.z_off + round_up(zrows(T - 1) * p.zstride, 256);
  p.x_bytes = p.shape.grid ? std::max({xlink_bytes(p.shape.ncta), fast_xlink_bytes(p.shape.ncta, kAnchorD), fast_xlink_bytes(p.shape.ncta, 4)}) : 0;
  p.ck_stride = static_cast<int>(round_up(static_cast<uint64_t>(S), 4));
  // Checkpoint segments: every segment of the recompute pass is a new pass
  // through the team's pipeline of warps, which fills with up to a 32-frame
  // window of lag per warp boundary (two per CTA boundary of a grid team). So
  // a segment spans at least about twice that fill (then the recompute pass
  // costs about one forward pass plus the fills), and at least sqrt(T)
  // frames; rounded up to whole anchor windows so that checkpoint frames end
  // windows. A budget that cannot hold such a segment gets shorter ones, down
  // to sqrt(T) frames.
  const uint64_t team_warps = static_cast<uint64_t>(p.shape.warps) * p.shape.ncta;
  const uint64_t fill = static_cast<uint64_t>(kAnchorD) * (team_warps - 1 + (p.shape.grid ? p.shape.ncta - 1 : 0));
  const uint64_t ck_min =
      round_up(static_cast<uint64_t>(std::max(1.0, std::ceil(std::sqrt(static_cast<double>(T))))), kAnchorD);
  const auto set_segments = [&](uint64_t every) {
    p.ck_every = static_cast<int>(every);
    p.nck = static_cast<int>((T - 1) / p.ck_every + 1);
    p.ckpt_bytes = round_up(static_cast<uint64_t>(p.nck) * p.ck_stride * 4ull, 256);
    p.seg_z_off = round_up(row_bytes * every, 256);
    p.seg_bp_bytes = p.seg_z_off + round_up(zrows(static_cast<int64_t>(every)) * p.zstride, 256);
  };
  uint64_t every = std::max(ck_min, round_up(std::min<uint64_t>(2 * fill, static_cast<uint64_t>(T)), kAnchorD));
  set_segments(every);
  while (every > ck_min && p.ckpt_bytes + p.seg_bp_bytes + p.x_bytes > budget) {
    every = std::max(ck_min, round_up(every / 2, kAnchorD));
    set_segments(every);
  }
  p.checkpointed = force_checkpoint || p.bp_bytes + p.x_bytes > budget;
  if (p.checkpointed && p.ckpt_bytes + p.seg_bp_bytes + p.x_bytes > budget) return ALIGN_E_TOO_LARGE;
  *out = p;
  return ALIGN_OK;
}

HostStage host_stage_layout(int64_t T, int64_t C) {
  HostStage h{};
  const uint64_t t4 = round_up(static_cast<uint64_t>(T) * 4, 256);
  h.lp = 0;
  h.path = round_up(static_cast<uint64_t>(T) * static_cast<uint64_t>(C) * 4, 256);
  h.scores = h.path + t4;
  h.states = h.scores + t4;
  h.total = h.states + t4;
  h.bytes = h.total + 256;
  return h;
}

bool rows_bulk_ok(const float* lp, int64_t C) {
  return (C % 4) == 0 && (reinterpret_cast<uintptr_t>(lp) % 16) == 0;
}

}  // namespace gb300_align

using namespace gb300_align;

extern "C" {

int align_validate(const int32_t* targets, int64_t L, int64_t C, int32_t blank, int64_t T, int64_t* repeats) {
  return validate_request(targets, L, C, blank, T, repeats);
}

int align_plan(int64_t T, int64_t C, int64_t L, uint64_t bp_budget_bytes, uint32_t flags, int32_t states_per_lane,
               int32_t cta_warps, int32_t max_cluster, align_plan_info* out) {
  if (!out || T < 1 || C < 2 || L < 0) return ALIGN_E_INVAL;
  TuneTable tune = default_tune_table();
  if (states_per_lane) tune.K = states_per_lane;
  if (cta_warps) tune.cta_warps = cta_warps;
  if (max_cluster) tune.max_cluster = max_cluster;
  Plan p{};
  const int rc = make_plan(tune, T, C, L, bp_budget_bytes ? bp_budget_bytes : (1ull << 30),
                           (flags & ALIGN_F_FORCE_CHECKPOINT) != 0, &p);
  if (rc != ALIGN_OK) return rc;
  out->states_per_lane = p.shape.K;
  out->warps_per_cta = p.shape.warps;
  out->cluster_ctas = p.shape.ncta;
  out->frames_per_stage = p.frames_per_stage;
  out->checkpointed = p.checkpointed ? 1 : 0;
  out->checkpoint_every = p.ck_every;
  out->checkpoints = p.nck;
  out->backpointer_bytes = p.bp_bytes;
  out->checkpoint_bytes = p.ckpt_bytes + p.seg_bp_bytes;
  return ALIGN_OK;
}

}  // extern "C"
