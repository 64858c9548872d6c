// Host-only planning and validation shared by the runtime and the C ABI.
#pragma once
#include <cstdint>

#include "trellis.cuh"

namespace gb300_align {

// Kernel-shape choices (replaced by measurements through align_set_tuning).
struct TuneBucket {
  int s_max;      // applies to transcripts with S <= s_max states
  int K;          // states per lane
  int cta_warps;  // warps per CTA before the team is split over a cluster
};

struct TuneTable {
  int K = 4;             // states per lane (when no bucket matches)
  int cta_warps = 4;     // warps per CTA before a team is split over a cluster
  int max_warps = 16;    // hard limit of warps per CTA (the kernel is built for 512 threads)
  int max_cluster = 16;  // CTAs per cluster for long transcripts
  int max_grid = 0;      // CTAs of a grid team (one per SM) beyond a cluster; 0: no grid teams
  int nbuckets = 0;      // measured choices per range of S, sorted by s_max
  TuneBucket buckets[16];
};
// The (K, cta_warps) that apply to a transcript of S states.
TuneTable resolve_tuning(const TuneTable& t, int64_t S);
TuneTable default_tune_table();

struct Plan {
  LaunchShape shape{};
  int frames_per_stage = 16;
  uint64_t bp_bytes = 0;      // full backpointers: warps * (T-1) * words * 4
  bool checkpointed = false;
  int ck_every = 0;           // frames between alpha checkpoints
  int nck = 0;                // number of checkpoints (segments)
  int ck_stride = 0;          // floats per checkpoint row
  uint64_t ckpt_bytes = 0;    // nck * ck_stride * 4
  uint64_t seg_bp_bytes = 0;  // backpointers + anchor rows of one segment
  int zstride = 0;            // bytes per anchor row (S rounded up to 16)
  uint64_t z_off = 0;         // offset of the anchor rows inside the full-mode allocation
  uint64_t seg_z_off = 0;     // offset of the anchor rows inside the segment buffer
  uint64_t x_bytes = 0;       // grid teams: CTA links, after the backpointers (or the segment buffer)
  uint64_t lse_bytes = 0;     // logits inputs: the per-frame log_softmax shift, after the links
};
// Device bytes of a request: backpointers (or checkpoints + one segment), the
// CTA links of a grid team (from plan_x_off), the per-frame shift of a
// logits request (from plan_lse_off).
inline uint64_t plan_x_off(const Plan& p) { return p.checkpointed ? p.ckpt_bytes + p.seg_bp_bytes : p.bp_bytes; }
inline uint64_t plan_lse_off(const Plan& p) { return plan_x_off(p) + p.x_bytes; }
inline uint64_t plan_device_bytes(const Plan& p) { return plan_lse_off(p) + p.lse_bytes; }

// Step A1: 0, ALIGN_E_INVAL, ALIGN_E_TARGET or ALIGN_E_INFEASIBLE; *repeats = R.
int validate_request(const int32_t* targets, int64_t L, int64_t C, int32_t blank, int64_t T, int64_t* repeats);

// Shape and footprint of a request; ALIGN_E_TOO_LARGE if it cannot run within budget.
int make_plan(const TuneTable& tune, int64_t T, int64_t C, int64_t L, uint64_t budget, bool force_checkpoint,
              Plan* out);
// Footprint and staging of a request whose shape is already set in *shape_plan.
int plan_footprint(int64_t T, int64_t C, int64_t L, uint64_t budget, bool force_checkpoint, Plan* shape_plan,
                   Plan* out);
// Plan of a request in a persistent launch: the fixed shape (K states per
// lane, `warps` compute warps per CTA), ceil(S / (32 K warps)) CTAs per team,
// full backpointers (ALIGN_E_TOO_LARGE otherwise; no CTA links of its own).
int make_persist_plan(int K, int warps, int64_t T, int64_t C, int64_t L, uint64_t budget, Plan* out);

// Device staging of a host-I/O request: emissions, then outputs.
struct HostStage {
  uint64_t lp, path, scores, states, total, bytes;
};
HostStage host_stage_layout(int64_t T, int64_t C);
inline uint64_t host_stage_bytes(int64_t T, int64_t C) { return host_stage_layout(T, C).bytes; }

// Emission rows may be staged with bulk copies (16-byte aligned rows).
bool rows_bulk_ok(const float* lp, int64_t C);

}  // namespace gb300_align
