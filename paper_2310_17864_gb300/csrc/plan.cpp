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

int make_plan(const TuneTable& tune, int64_t T, int64_t C, int64_t L, uint64_t budget, bool force_checkpoint,
              Plan* out) {
  Plan p{};
  const int64_t S = 2 * L + 1;
  // Shape: one CTA of up to max_warps warps, else a cluster of CTAs.
  // The K = 16 kernel keeps 2x more state in registers and is built for 512 threads.
  const int K = tune.K;
  const auto warp_cap = [&](int k) { return k == 16 ? std::min(16, tune.max_warps) : tune.max_warps; };
  const uint64_t G1 = ceil_div(static_cast<uint64_t>(S), 32ull * K);
  if (G1 <= static_cast<uint64_t>(warp_cap(K))) {
    p.shape = LaunchShape{K, static_cast<int>(G1), 1};
  } else {
    // Prefer portable clusters (<= 8 CTAs), then larger K, then non-portable sizes.
    bool found = false;
    const int portable = std::min(8, tune.max_cluster);
    const std::pair<int, int> tries[] = {{K, portable}, {8, portable}, {K, tune.max_cluster},
                                         {8, tune.max_cluster}, {16, tune.max_cluster}};
    for (auto [k, cmax] : tries) {
      if (k < K) continue;
      const int wmax = warp_cap(k);
      const uint64_t G = ceil_div(static_cast<uint64_t>(S), 32ull * k);
      const uint64_t ncta = ceil_div(G, static_cast<uint64_t>(wmax));
      if (ncta <= static_cast<uint64_t>(cmax)) {
        p.shape = LaunchShape{k, static_cast<int>(ceil_div(G, ncta)), static_cast<int>(ncta)};
        found = true;
        break;
      }
    }
    if (!found) return ALIGN_E_TOO_LARGE;
  }
  // Emission staging: stages of about 8 KB (16 frames of a 32-class row).
  p.frames_per_stage = static_cast<int>(std::clamp<int64_t>(8192 / (4 * C), 1, 16));
  const uint64_t warps = static_cast<uint64_t>(p.shape.warps) * p.shape.ncta;
  const uint64_t row_bytes = warps * bp_words(p.shape.K) * 4ull;
  p.bp_bytes = row_bytes * static_cast<uint64_t>(std::max<int64_t>(T - 1, 0));
  p.ck_every = std::max(1, static_cast<int>(std::ceil(std::sqrt(static_cast<double>(T)))));
  p.nck = static_cast<int>((T - 1) / p.ck_every + 1);
  p.ck_stride = static_cast<int>(round_up(static_cast<uint64_t>(S), 4));
  p.ckpt_bytes = round_up(static_cast<uint64_t>(p.nck) * p.ck_stride * 4ull, 256);
  p.seg_bp_bytes = row_bytes * static_cast<uint64_t>(p.ck_every);
  p.checkpointed = force_checkpoint || p.bp_bytes > budget;
  if (p.checkpointed && p.ckpt_bytes + p.seg_bp_bytes > budget) return ALIGN_E_TOO_LARGE;
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
               int32_t max_cluster, align_plan_info* out) {
  if (!out || T < 1 || C < 2 || L < 0) return ALIGN_E_INVAL;
  TuneTable tune = default_tune_table();
  if (states_per_lane) tune.K = states_per_lane;
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
