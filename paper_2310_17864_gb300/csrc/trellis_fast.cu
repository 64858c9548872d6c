// Fast Viterbi trellis kernel for CTC forced alignment on sm_103a.
//
// The same hot path as trellis_kernel (Viterbi forward over the CTC trellis
// of the TorchAudio 2.1 paper's forced-alignment feature, Sec. 4 "CTC-based
// forced alignment", on the trellis of the cited CTC work; final state,
// windowed backtrack, scores), for K = 2 or 4 states per lane, with a frame
// loop built for a short dependent chain and few instructions per frame:
//
//   * a window of 32 frames is one straight-line block of code (blocks of kB
//     frames, every frame index a compile-time constant);
//   * one comparison per (blank, label) pair of states decides the blank
//     state's advance and the label state's best move other than staying;
//   * backpointers: each lane collects, per state, one bit per frame of the
//     window ("advance won" for a blank state, "stay lost" for a label
//     state) in a register and stores its words once per window (coalesced,
//     128 bytes per word and warp), instead of per-frame warp ballots;
//   * neighbour hand-off: the last lane of a warp writes, for each frame, a
//     64-bit word (alpha of its last state, frame tag, anchor offset) into
//     the next warp's link (shared memory, the next CTA's shared memory over
//     DSMEM, or global memory for grid teams), two words per store; the
//     receiver checks the tags of a whole block once and lane 0 reads one
//     word per frame; a consumption counter written back bounds the sender's
//     lead (flow control, one check per block);
//   * emission rows are staged by a producer warp with bulk copies; rows of
//     32 classes sit at compile-time offsets (kC).
//
// Arithmetic is the definition's (strict '>' in the order stay, advance,
// skip; one FP32 add after an exact max), so results are bit-identical to the
// generic kernel and the oracle for every team shape.
//
// Backpointer layout (per pass): window m (frames t_begin+1+32m ..
// t_begin+32m+32, bit i = frame t_begin+1+32m+i), warp g, word w, lane l at
//   bp[((m * G + g) * NW + w) * 32 + l],   NW = 3K/2 (words K+1.. unused):
//   word j < K, j even : "advance won" bits of blank state 32Kg + Kl + j,
//   word j < K, j odd  : "stay lost" bits of label state 32Kg + Kl + j,
//   word K             : the lane's skip permissions (bit i: label state
//                        32Kg + Kl + 2i + 1 may skip), the same every window.
// A label state's advance and skip candidates are also the two candidates of
// the blank state below it, so one comparison serves both: when the label
// state does not stay, it skips exactly when skipping is allowed and the
// blank state below advanced at the same frame (strict '>' keeps the order
// stay, advance, skip), and the backtrack reads that bit back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "trellis.cuh"
#include "trellis_common.cuh"

namespace gb300_align {
namespace {

// ------------------------------------------------- link memory operations --
// Scopes of one link: kLinkCta (two warps of a CTA, shared memory),
// kLinkCluster (CTAs of a cluster, DSMEM), kLinkGpu (CTAs of a grid team,
// global memory). Every link access is a relaxed (morally strong) access at
// the link's scope: a package word carries its own frame tag, so a reader
// that sees the tag sees the value (64-bit single-copy atomicity) and no
// fence is needed; the consumption counter is written after the reader has
// checked the tags of the words it read (a control dependency), so the
// sender never overwrites a word that is still to be read.
enum LinkScope { kLinkCta = 0, kLinkCluster = 1, kLinkGpu = 2 };

// Two package words (relaxed, 16-byte aligned).
__device__ __forceinline__ void st_words(int scope, uint32_t addr, uint64_t* p, uint64_t x, uint64_t y) {
  if (scope == kLinkGpu)
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(x), "l"(y) : "memory");
  else if (scope == kLinkCluster)
    asm volatile("st.relaxed.cluster.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(x), "l"(y) : "memory");
  else
    asm volatile("st.relaxed.cta.shared::cta.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(x), "l"(y) : "memory");
}
__device__ __forceinline__ void ld_words(int scope, uint32_t addr, const uint64_t* p, uint64_t& x, uint64_t& y) {
  if (scope == kLinkGpu)
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "l"(p) : "memory");
  else if (scope == kLinkCluster)
    asm volatile("ld.relaxed.cluster.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "r"(addr) : "memory");
  else
    asm volatile("ld.relaxed.cta.shared::cta.v2.u64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "r"(addr) : "memory");
}
// The consumption counter (u32).
__device__ __forceinline__ void st_count(int scope, uint32_t addr, uint32_t* p, uint32_t v) {
  if (scope == kLinkGpu)
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
  else if (scope == kLinkCluster)
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
  else
    asm volatile("st.relaxed.cta.shared::cta.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_count(int scope, uint32_t addr, const uint32_t* p) {
  uint32_t v;
  if (scope == kLinkGpu)
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  else if (scope == kLinkCluster)
    asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  else
    asm volatile("ld.relaxed.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Bounded wait by lane 31 until the consumption counter reaches `need`; the
// result is uniform over the warp. False on timeout (the CTA abort flag is
// raised) or when another warp of the CTA aborted.
__device__ __noinline__ bool count_wait(int scope, uint32_t addr, const uint32_t* p, uint32_t need,
                                        volatile int32_t* abort, uint64_t limit) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  if (lane == 31) {
    const uint64_t t0 = gtimer();
    for (;;) {
      if (ld_count(scope, addr, p) >= need) break;
      if (*abort != 0 || gtimer() - t0 > limit) {
        *abort = 1;
        ok = 0;
        break;
      }
    }
  }
  return __shfl_sync(kFull, ok, 31) != 0;
}

// Package of kB words read by lane 0: word i = alpha bits | (tag << 8 | anchor
// offset) << 32, tag = (frame + 1) mod 2^24 of the frame whose alpha it is.
// Returns true when the tags of words 0 .. n-1 (the frames of the block; a
// block at the end of a pass may be partial, and the sender's later words are
// then meaningless) are the expected ones (`e0` = the tag of word 0, shifted
// left by 8); on success off[i] = the anchor offsets.
template <int kB>
__device__ __forceinline__ bool read_package(int scope, uint32_t addr, const uint64_t* p, uint32_t e0, int n,
                                             float (&pa)[kB], uint32_t (&off)[kB]) {
  uint64_t w[kB];
#pragma unroll
  for (int q = 0; q < kB / 2; ++q) ld_words(scope, addr + q * 16, p + 2 * q, w[2 * q], w[2 * q + 1]);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    pa[i] = __uint_as_float(static_cast<uint32_t>(w[i]));
    off[i] = static_cast<uint32_t>(w[i] >> 32) - (e0 + (static_cast<uint32_t>(i) << 8));
    ok = ok & ((i >= n) | (off[i] < 256u));
  }
  return ok;
}

// Slow path of a package read: lane 0 re-reads until every tag matches
// (bounded); uniform result. The caller then reads the package again.
template <int kB>
__device__ __noinline__ bool package_wait(int scope, uint32_t addr, const uint64_t* p, uint32_t e0, int n,
                                          volatile int32_t* abort, uint64_t limit) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  if (lane == 0) {
    const uint64_t t0 = gtimer();
    float pa[kB];
    uint32_t off[kB];
    while (!read_package<kB>(scope, addr, p, e0, n, pa, off)) {
      if (*abort != 0 || gtimer() - t0 > limit) {
        *abort = 1;
        ok = 0;
        break;
      }
    }
  }
  return __shfl_sync(kFull, ok, 0) != 0;
}

// Two 64-bit words stored by the lanes where `pred` holds (predicated PTX, no
// branch): relaxed at cluster scope in shared memory, or at gpu scope through
// a generic address.
__device__ __forceinline__ void st_cluster_v2u64_if(uint32_t addr, uint64_t x, uint64_t y, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.relaxed.cluster.shared::cluster.v2.u64 [%0], {%1, %2};\n\t}" ::"r"(
          addr),
      "l"(x), "l"(y), "r"(static_cast<uint32_t>(pred))
      : "memory");
}
__device__ __forceinline__ void st_gpu_v2u64_if(uint64_t* p, uint64_t x, uint64_t y, bool pred) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.relaxed.gpu.v2.u64 [%0], {%1, %2};\n\t}" ::"l"(p),
               "l"(x), "l"(y), "r"(static_cast<uint32_t>(pred))
               : "memory");
}

// log(sum_c exp(row[c])) of one row of raw logits (max factored out; CUDA's
// expf / logf). -inf for a row of -inf. Rows of 16-byte aligned, 4-float
// multiples are read as float4s, 8 at a time, so the loads are in flight
// together.
__device__ float row_lse(const float* __restrict__ row, int C, bool vec4) {
  float m = -INFINITY;
  if (vec4) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const int n4 = C >> 2;
    for (int c = 0; c < n4; c += 8) {
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = (c + k < n4) ? __ldg(r4 + c + k) : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
#pragma unroll
      for (int k = 0; k < 8; ++k) m = fmaxf(m, fmaxf(fmaxf(v[k].x, v[k].y), fmaxf(v[k].z, v[k].w)));
    }
    if (m == -INFINITY) return -INFINITY;
    float s = 0.0f;
    for (int c = 0; c < n4; c += 8) {
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = (c + k < n4) ? __ldg(r4 + c + k) : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        s += expf(v[k].x - m);
        s += expf(v[k].y - m);
        s += expf(v[k].z - m);
        s += expf(v[k].w - m);
      }
    }
    return m + logf(s);
  }
  for (int c = 0; c < C; ++c) m = fmaxf(m, __ldg(row + c));
  if (m == -INFINITY) return -INFINITY;
  float s = 0.0f;
  for (int c = 0; c < C; ++c) s += expf(__ldg(row + c) - m);
  return m + logf(s);
}

// ------------------------------------------------------------------ kernel --
// kGrid: the team is P.grid_ctas consecutive CTAs of a cooperative launch (one
// per SM), linked through global memory (J.xlink); otherwise a thread-block
// cluster (or one CTA) linked through shared memory and DSMEM.
// kNorm: log_probs hold raw logits. log_softmax subtracts one value per frame
// from every state of that frame, so the Viterbi choices over the logits
// equal those over the log-probabilities: the frame loop runs on the logits
// unchanged, and the score pass subtracts each chosen frame's log-sum-exp.
// The dynamic shared memory of the fast kernels.
__device__ __forceinline__ unsigned char* fast_smem() {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  return smem_dyn;
}

// Positions in the ring of emission stages, kept across the jobs a
// persistent CTA runs: the producer's next stage and round, and the compute
// warps' current ones (the mbarrier phases follow the rounds).
struct StageRing {
  int p_stage = 0;
  uint32_t p_round = 0;
  int c_stage = 0;
  uint32_t c_round = 0;
  uint32_t t_round = 0;  // completed phases of the backtrack's copy barrier (warp 0)
};

// The whole hot path of one job for one CTA of its team: this CTA is rank
// `crank` of `ncta` CTAs. The stage barriers are initialised by the caller.
// kC: 0, or the vocabulary of every job of the launch when it is 32 (window
// mode): emission rows then sit at compile-time offsets in a stage.
template <int K, int kB, bool kGrid, bool kNorm, int kC>
__device__ __forceinline__ void team_job(const FwdJob& J, const FwdParams& P, const uint32_t ncta, const uint32_t crank,
                                         StageRing& ring) {
  static_assert(K == 2 || K == 4, "fast kernel: K = 2 or 4");
  static_assert(kC == 0 || (kC == 32 && kB == kAnchorD), "fixed rows of 32 classes in window mode only");
  static_assert(kB == 4 || kB == 8 || kB == kAnchorD, "fast kernel: blocks of 4 or 8 frames, or whole windows");
  constexpr int NW = bp_words(K);
  constexpr int kWin = kAnchorD;
  unsigned char* const smem = fast_smem();
  SmemHead* head = reinterpret_cast<SmemHead*>(smem);
  unsigned char* stages = smem + P.off_stage;
  volatile int32_t* abort = &head->abort;

  const int W = (blockDim.x >> 5) - 1;  // compute warps; warp W stages the emission rows
  const int warp = threadIdx.x >> 5;
  const bool producer = (warp == W);
  const int lane = threadIdx.x & 31;
  const int g = static_cast<int>(crank) * W + warp;  // warp index in the team
  const int G = static_cast<int>(ncta) * W;
  const int S = J.S, C = J.C, blank = J.blank;
  const int t_begin = J.t_begin, t_end = J.t_end;
  const int s0 = (g * 32 + lane) * K;
  const int F = P.frames_per_stage;
  const uint64_t limit = P.wait_limit_ns;
  const float* __restrict__ lp = J.lp;
  uint32_t* __restrict__ bp = J.bp;
  float* __restrict__ ckpt = J.ckpt;
  const int ck_every = J.ck_every;
  const int ck_stride = J.ck_stride;
  int32_t* const path = J.path;
  float* const scores_out = J.scores;
  int32_t* const states_out = J.states;
  const int32_t* const tgt = J.tgt;
  const int R = P.pkgs;
  const int Rg = P.gpkgs;

  // Launch parameters must fit the job (uniform over the team, checked before
  // any barrier): stages hold F >= kB rows, the team holds every state,
  // package rings are powers of two, checkpoint frames end windows.
  const bool ck_ok = ckpt == nullptr || (ck_every > 0 && ck_every % kAnchorD == 0 && t_begin % ck_every == 0);
  if (F * C * 4 > P.stage_bytes || (kC != 0 && C != kC) || static_cast<int64_t>(ncta) * W * 32 * K < S || P.stages < kLead ||
      P.stages > kMaxStages || F < kB || F > kAnchorD || (F & (F - 1)) != 0 || P.kb != kB || R < 2 ||
      (R & (R - 1)) != 0 || P.link_stride < 16 + R * kB * 8 || !ck_ok ||
      (kGrid && ncta > 1 && (J.xlink == nullptr || Rg < 2 || (Rg & (Rg - 1)) != 0))) {
    if (threadIdx.x == 0 && crank == 0) atomicExch(J.status, kStBadLaunch);
    return;
  }

  // ---- shared state: links zeroed (counters and package slots: a slot left
  // by an earlier kernel could hold a matching tag), barriers initialised ----
  {
    uint4* lk = reinterpret_cast<uint4*>(smem + P.link_off);
    const int n16 = W * P.link_stride / 16;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) lk[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  const bool bulk = (J.flags & kJobBulkRows) != 0;
  if (threadIdx.x == 0) {
    head->abort = 0;
    head->team_bad = 0u;
  }
  __syncthreads();
  if (!kGrid && ncta > 1) cluster_sync();  // every CTA's links and flags are zero before any remote store

  // ---- emission staging (a dedicated producer warp) ----
  // Chunk c holds the rows of frames t_begin+1+c*F .. t_begin+(c+1)*F in
  // stage c mod stages. F divides the window, kB divides F.
  const int nfr = t_end - 1 - t_begin;  // frames computed in this pass
  const int nchunks = (nfr + F - 1) / F;
  int issued = 0;
  int& p_stage = ring.p_stage;
  uint32_t& p_round = ring.p_round;
  auto issue_next = [&]() {
    const int f0 = t_begin + 1 + issued * F;
    const int nf = min(F, t_end - f0);
    const float* src = lp + static_cast<size_t>(f0) * C;
    float* dst = reinterpret_cast<float*>(stages + p_stage * P.stage_bytes);
    if (bulk) {
      if (lane == 0) {
        const uint32_t bytes = static_cast<uint32_t>(nf * C * 4);
        mbar_arrive_expect_tx(&head->full[p_stage], bytes);
        bulk_g2s(dst, src, bytes, &head->full[p_stage]);
      }
    } else {
      const int n = nf * C;
      for (int i = lane; i < n; i += 32) cp_async4(dst + i, src + i);
      cp_async_mbar_arrive(&head->full[p_stage]);
    }
    ++issued;
    if (++p_stage == P.stages) {
      p_stage = 0;
      ++p_round;
    }
  };
  const int nwin = (nfr + kWin - 1) / kWin;  // anchor rows / backpointer windows of this pass
  uint8_t* const ztab = J.ztab;
  const int zstride = J.zstride;
  // Grid teams: the team barrier follows the CTA links in global memory.
  uint32_t* const xbar = kGrid ? reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(J.xlink) +
                                                            static_cast<size_t>(ncta - 1) * (16 + Rg * kB * 8))
                               : nullptr;
  // Team block in device memory (grid teams of several CTAs): words 0-1 the
  // barrier, 2-3 the final alphas, 4 the timeout flag.
  const bool xteam = kGrid && ncta > 1;
  if (producer) {
    // Every chunk as soon as its stage is free (released by every compute
    // warp); then every copy in flight lands before the shared memory is
    // reused. The compute warps only release stages and wait for rows, so
    // no copy is issued on the recursion's path.
    for (int c = 0; c < nchunks; ++c) {
      if (p_round > 0 && !warp_wait_phase(&head->empty[p_stage], (p_round - 1) & 1u, abort, limit, lane)) break;
      issue_next();
    }
    if (lane == 0) {
      // Chunk x of the ring (counted over every job of this CTA) used stage
      // x mod stages in round x / stages.
      const int64_t next = static_cast<int64_t>(p_round) * P.stages + p_stage;
      for (int64_t x = next - min(issued, P.stages); x < next; ++x)
        (void)wait_phase(&head->full[x % P.stages], static_cast<uint32_t>(x / P.stages) & 1u, abort, limit, false);
    }
  } else {

  // ---- per-lane constants: label columns and skip permissions ----
  int col[K / 2];
  bool skok[K / 2];
#pragma unroll
  for (int i = 0; i < K / 2; ++i) {
    const int s = s0 + 2 * i + 1;
    int lab = 0;
    bool skip = false;
    if (s < S) {
      lab = tgt[(s - 1) >> 1];
      skip = (s >= 3) && (lab != tgt[(s - 3) >> 1]);
    }
    col[i] = lab;
    skok[i] = skip;
  }

  uint32_t skmask = 0u;  // bit i: label state s0 + 2i + 1 may skip
#pragma unroll
  for (int i = 0; i < K / 2; ++i) skmask |= skok[i] ? (1u << i) : 0u;

  // ---- frame t_begin ----
  float a[K];
  int A[K];  // anchor: state at the last window end on the best path to each state
  if (J.alpha_in == nullptr) {
    const float* row = lp + static_cast<size_t>(t_begin) * C;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int s = s0 + j;
      a[j] = (s == 0) ? __ldg(row + blank) : ((s == 1 && S > 1) ? __ldg(row + col[0]) : -INFINITY);
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) a[j] = (s0 + j < S) ? __ldg(J.alpha_in + s0 + j) : -INFINITY;
  }
#pragma unroll
  for (int j = 0; j < K; ++j) A[j] = s0 + j;
  if (ckpt != nullptr && (t_begin % ck_every) == 0) {
    float* dst = ckpt + static_cast<size_t>(t_begin / ck_every) * ck_stride;
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (s0 + j < S) dst[s0 + j] = a[j];
  }

  // ---- links ----
  // Warp w's link (shared memory at link_off + w * link_stride): word 1 counts
  // w's packages consumed by its right neighbour; from 16 bytes on, R package
  // slots of kB words written by w's left neighbour. Grid teams: the link
  // between CTA b's last warp and CTA b+1's warp 0 is in global memory at
  // xlink + b * gstride (same layout, Rg slots); the team barrier follows the
  // last link.
  const int gstride = 16 + Rg * kB * 8;
  unsigned char* const xl = kGrid ? reinterpret_cast<unsigned char*>(J.xlink) : nullptr;
  const bool recv_left = g > 0;
  const bool send_local = warp < W - 1;
  const bool send_remote = (warp == W - 1) && (crank + 1 < ncta);
  const bool has_next = send_local || send_remote;
  const uint32_t my_link = smem_addr(smem + P.link_off + warp * P.link_stride);
  // Receiving side.
  const bool recv_remote = recv_left && warp == 0;
  const int rscope = !recv_remote ? kLinkCta : (kGrid ? kLinkGpu : kLinkCluster);
  const int rslots = (rscope == kLinkGpu) ? Rg : R;
  uint32_t* const rg = (kGrid && recv_remote) ? reinterpret_cast<uint32_t*>(xl + static_cast<size_t>(crank - 1) * gstride)
                                             : nullptr;
  const uint32_t r_data = my_link + 16;
  const uint64_t* const rg_data = rg ? reinterpret_cast<const uint64_t*>(rg + 4) : nullptr;
  // Where the receiver reports consumption: the left neighbour's word 1.
  const uint32_t r_cons = !recv_left ? 0u
                          : (warp > 0)  ? smem_addr(smem + P.link_off + (warp - 1) * P.link_stride) + 4u
                          : kGrid       ? 0u
                                        : mapa_rank(smem_addr(smem + P.link_off + (W - 1) * P.link_stride), crank - 1) + 4u;
  // Sending side.
  const int sscope = !send_remote ? kLinkCta : (kGrid ? kLinkGpu : kLinkCluster);
  const int sslots = (sscope == kLinkGpu) ? Rg : R;
  uint32_t* const sg = (kGrid && send_remote) ? reinterpret_cast<uint32_t*>(xl + static_cast<size_t>(crank) * gstride)
                                             : nullptr;
  uint64_t* const sg_data = sg ? reinterpret_cast<uint64_t*>(sg + 4) : nullptr;
  const uint32_t s_link = send_local    ? smem_addr(smem + P.link_off + (warp + 1) * P.link_stride)
                          : (send_remote && !kGrid) ? mapa_rank(smem_addr(smem + P.link_off), crank + 1)
                                                    : 0u;
  const uint32_t s_cons = my_link + 4u;  // own word 1 (cluster scope when the receiver is remote)
  uint32_t cons_seen = 0;                // packages of this warp consumed, as last observed
  uint32_t pk = 0;                       // packages exchanged so far (same count on both sides)
  const int s_last = s0 + K - 1;
  const bool is_l0 = (lane == 0);
  const bool stall = (J.flags & kJobTestStall) && g == 0;  // test hook: the first warp never publishes
  bool dead = false;                                       // a bounded wait ran out (or another warp aborted)

  // One frame of this lane's states, as (blank j-1, label j) pairs in
  // descending order (a[j-1], a[j-2] still hold frame t-1). The blank state
  // advances when its left neighbour is strictly greater; the label state's
  // best move other than staying is then that same candidate when it may
  // skip, else the blank state below, and it leaves its state only when that
  // candidate is strictly greater (stay > advance > skip on ties). Selects
  // for the values; a chosen move's bit is set by a predicated OR.
  auto step_pairs = [&](const float left, const int Aleft, const float eb, const float (&el)[K / 2],
                        uint32_t (&bw)[NW], const uint32_t bit) {
#pragma unroll
    for (int j = K - 1; j >= 1; j -= 2) {
      const float p = (j == 1) ? left : a[j - 2];
      const int qp = (j == 1) ? Aleft : A[j - 2];
      const bool adv = p > a[j - 1];
      const float mb = adv ? p : a[j - 1];
      const int Ab = adv ? qp : A[j - 1];
      const bool sk = skok[j >> 1];
      const float mv = sk ? mb : a[j - 1];
      const int Am = sk ? Ab : A[j - 1];
      const bool moved = mv > a[j];
      a[j] = (moved ? mv : a[j]) + el[j >> 1];
      A[j] = moved ? Am : A[j];
      if (moved) bw[j] |= bit;
      a[j - 1] = mb + eb;
      A[j - 1] = Ab;
      if (adv) bw[j - 1] |= bit;
    }
  };

  // ---- frames t_begin+1 .. t_end-1 ----
  float carry_a = a[K - 1];  // block mode: alpha of the last state at the first frame of the next package
  int carry_A = A[K - 1];
  // Window end: backpointer words, anchor row m, anchors reset, checkpoint.
  auto end_window_bits = [&](uint32_t (&bits)[NW], const int m, const int t_last) {
    if (bp != nullptr) {
      uint32_t* dst = bp + (static_cast<size_t>(m) * G + g) * NW * 32 + lane;
#pragma unroll
      for (int w = 0; w < K; ++w) dst[w * 32] = bits[w];
      dst[K * 32] = skmask;
    }
    if (ztab != nullptr && s0 < zstride) {
      uint8_t* dst = ztab + static_cast<size_t>(m) * zstride + s0;
      uint32_t packed = 0u;
#pragma unroll
      for (int j = 0; j < K; ++j) packed |= (static_cast<uint32_t>(s0 + j - A[j]) & 0xffu) << (8 * j);
      if constexpr (K == 2)
        *reinterpret_cast<uint16_t*>(dst) = static_cast<uint16_t>(packed);
      else
        *reinterpret_cast<uint32_t*>(dst) = packed;
    }
    if (ckpt != nullptr && (t_last % ck_every) == 0) {
      float* dst = ckpt + static_cast<size_t>(t_last / ck_every) * ck_stride;
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (s0 + j < S) dst[s0 + j] = a[j];
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) bits[w] = 0u;
#pragma unroll
    for (int j = 0; j < K; ++j) A[j] = s0 + j;
    carry_A = s0 + K - 1;
  };

  const int nwin_full = nfr / kWin;
  const int rem = nfr - nwin_full * kWin;
  if constexpr (kB == kWin) {
    // ---- window mode (32-frame chunks): the hand-off is one tagged word per
    // frame. The last lane of the left neighbour stores, with a predicated
    // relaxed 64-bit store (no branch), the word of each frame it computes
    // into this warp's ring: slot m (R slots of 32 words) holds the
    // neighbour's alpha / anchor offset at frames t_begin+32m .. +31, word i
    // tagged (t_begin + 32m + i + 1) << 8. At the start of window m every
    // lane checks one word's tag (all 32 frames of the window must be there),
    // then each frame reads lane 0's word with a broadcast load; the
    // consumption count is published at the window end. A window of 32 frames
    // is straight-line code with no branch.
    // The first warp of the team reads its own ring, filled with -inf.
    if (!recv_left) {
      const uint64_t ninf = static_cast<uint64_t>(__float_as_uint(-INFINITY));
      for (int i = lane; i < R * kWin / 2; i += 32) st_words(kLinkCta, r_data + i * 16, nullptr, ninf, ninf);
    }
    __syncwarp();
    // Word 0 of slot 0: this warp's last state at t_begin (tag t_begin + 1).
    const uint32_t s_store_pred = (has_next && !stall && lane == 31) ? 1u : 0u;
    auto slot_addr_s = [&](int m) -> uint32_t { return s_link + 16u + static_cast<uint32_t>((m & (sslots - 1)) * kWin * 8); };
    auto slot_ptr_s = [&](int m) -> uint64_t* { return sg_data ? sg_data + (m & (sslots - 1)) * kWin : nullptr; };
    // kGrid: every send is a generic-address relaxed store at gpu scope
    // (shared memory for a local link, global memory for the next CTA);
    // clusters: a relaxed store at cluster scope (local or remote).
    uint64_t* const s_gen_local = (kGrid && send_local)
                                      ? reinterpret_cast<uint64_t*>(smem + P.link_off + (warp + 1) * P.link_stride + 16)
                                      : nullptr;
    // Words k, k+1 (k even) of slot m of the right neighbour's ring, in one
    // 16-byte store by the last lane: a store per frame would sit in the
    // shared-memory pipe ahead of the next frame's shuffles.
    auto send_pair = [&](int m, int k, uint64_t w0, uint64_t w1) {
      if constexpr (kGrid) {
        uint64_t* base = send_remote ? slot_ptr_s(m) : s_gen_local + (m & (sslots - 1)) * kWin;
        st_gpu_v2u64_if(base + k, w0, w1, s_store_pred != 0u);
      } else {
        st_cluster_v2u64_if(slot_addr_s(m) + static_cast<uint32_t>(k * 8), w0, w1, s_store_pred != 0u);
      }
    };
    // The word of the previous frame (at first this warp's last state at
    // t_begin, tag t_begin + 1); stored with the next even frame's word.
    uint64_t prev_w;
    {
      const uint32_t hb0 = (static_cast<uint32_t>(t_begin + 1) << 8) + static_cast<uint32_t>(s_last);
      prev_w = (static_cast<uint64_t>(hb0 - static_cast<uint32_t>(A[K - 1])) << 32) | __float_as_uint(a[K - 1]);
    }
    uint32_t bits[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) bits[w] = 0u;
    auto end_window = [&](const int m, const int t_last) { end_window_bits(bits, m, t_last); };
    const int nwin_all = nwin_full + (rem > 0 ? 1 : 0);
    uint64_t pf0 = 0ull, pf1 = 0ull;  // grid teams: window pf_m's words, loaded one window ahead
    int pf_m = -1;
    int& c_stage = ring.c_stage;
    uint32_t& c_round = ring.c_round;
    const float* stage_f = reinterpret_cast<const float*>(stages);
    const int stage_floats = P.stage_bytes / 4;

    // Start of window m (nf frames): emission chunk, flow control of this
    // warp's sends, the neighbour's words for the window. False when a
    // bounded wait ran out.
    auto window_begin = [&](const int m, const int nf) -> bool {
      if (m > 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&head->empty[c_stage]);
        if (++c_stage == P.stages) {
          c_stage = 0;
          ++c_round;
        }
      }
      if (!warp_wait_phase(&head->full[c_stage], c_round & 1u, abort, limit, lane)) return false;
      if (has_next && !stall) {
        // This window writes slot m, which last held window m-slots of the
        // receiver.
        const uint32_t need = (m + 1 > sslots) ? static_cast<uint32_t>(m + 1 - sslots) : 0u;
        if (cons_seen < need) {
          uint32_t v = need;
          if (lane == 31) v = ld_count(sscope, s_cons, sg ? sg + 1 : nullptr);
          cons_seen = __shfl_sync(kFull, v, 31);
          if (cons_seen < need) {
            if (!count_wait(sscope, s_cons, sg ? sg + 1 : nullptr, need, abort, limit)) return false;
            cons_seen = need;
          }
        }
      }
      if (recv_left) {
        // Shared-memory slot of window m (the per-frame reads use it; grid
        // teams copy their global words there), R slots.
        const uint32_t raddr = r_data + static_cast<uint32_t>((m & (R - 1)) * kWin * 8 + lane * 8);
        // Lane pairs read one 16-byte pair of words; lane i keeps word i.
        // (Ring slots: rslots in global memory for grid teams, R in shared
        // memory otherwise; rslots == R for shared-memory links.)
        auto load_pair = [&](int mm, uint64_t& w0, uint64_t& w1) {
          const int sl = mm & (rslots - 1);
          const uint64_t* rp = rg_data ? rg_data + sl * kWin + (lane & ~1) : nullptr;
          ld_words(rscope, (r_data + static_cast<uint32_t>(sl * kWin * 8 + lane * 8)) & ~15u, rp, w0, w1);
        };
        auto tag_ok = [&](int mm, int nfm, uint64_t w0, uint64_t w1) -> bool {
          const uint64_t w = (lane & 1) ? w1 : w0;
          const uint32_t e = static_cast<uint32_t>(t_begin + kWin * mm + 1 + lane) << 8;
          return (lane >= nfm) | (static_cast<uint32_t>(w >> 32) - e < 256u);
        };
        auto wait_slot = [&](int mm, int nfm, uint64_t& w0, uint64_t& w1) -> bool {
          load_pair(mm, w0, w1);  // usually there already: no timer read
          if (__all_sync(kFull, tag_ok(mm, nfm, w0, w1))) return true;
          const uint64_t t0 = gtimer();
          for (;;) {
            load_pair(mm, w0, w1);
            if (__all_sync(kFull, tag_ok(mm, nfm, w0, w1))) return true;
            if (__any_sync(kFull, (*abort != 0) | (gtimer() - t0 > limit))) {
              if (lane == 0) *abort = 1;
              return false;
            }
          }
        };
        if (rscope != kLinkGpu) {
          uint64_t w0, w1;
          if (!wait_slot(m, nf, w0, w1)) return false;
        } else {
          // Grid teams: the words come from global memory. This warp runs two
          // windows behind its sender and loads window m+1's words at the
          // start of window m, so the L2 round trip overlaps the window's
          // frames; at the next window start the tags say whether the
          // prefetched copy is complete (else it is read again). The
          // window's words are kept in this warp's own (otherwise unused)
          // shared ring slot for the per-frame reads.
          uint64_t w0 = pf0, w1 = pf1;
          if (!(pf_m == m && __all_sync(kFull, tag_ok(m, nf, w0, w1))))
            if (!wait_slot(m, nf, w0, w1)) return false;
          st_words(kLinkCta, raddr & ~15u, nullptr, w0, w1);
          __syncwarp();
          if (m + 1 < nwin_all) {
            const int nf1 = (m + 1 < nwin_full) ? kWin : rem;
            if (m == 0) {  // establish the lag of two windows
              if (!wait_slot(1, nf1, pf0, pf1)) return false;
            } else {
              load_pair(m + 1, pf0, pf1);
            }
            pf_m = m + 1;
          }
        }
      }
      return true;
    };
    auto window_end_recv = [&](const int m) {
      if (recv_left && is_l0) st_count(rscope, r_cons, rg ? rg + 1 : nullptr, static_cast<uint32_t>(m + 1));
    };

    uint32_t pk_lo0 = 0u, pk_hi0 = 0u, pk_lo1 = 0u, pk_hi1 = 0u;  // the left neighbour's words of a frame pair
    // Frame i of window m (frame t_begin + 32m + 1 + i).
    const int Cr = kC != 0 ? kC : C;  // row stride of a stage (a compile-time 32 when kC is)
    auto do_frame = [&](const int m, const int i, const float* rowp, const uint32_t rslot_addr) {
      const uint32_t bit = 1u << i;
      const float eb = rowp[i * Cr + blank];
      float el[K / 2];
#pragma unroll
      for (int q = 0; q < K / 2; ++q) el[q] = rowp[i * Cr + col[q]];
      // The left neighbour's word of this frame (read in pairs, at even frames).
      if ((i & 1) == 0)
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(pk_lo0), "=r"(pk_hi0), "=r"(pk_lo1), "=r"(pk_hi1)
                     : "r"(rslot_addr + static_cast<uint32_t>(i * 8))
                     : "memory");
      const uint64_t pw = (i & 1) ? ((static_cast<uint64_t>(pk_hi1) << 32) | pk_lo1)
                                  : ((static_cast<uint64_t>(pk_hi0) << 32) | pk_lo0);
      const float shf = __shfl_up_sync(kFull, a[K - 1], 1);
      const float left = is_l0 ? __uint_as_float(static_cast<uint32_t>(pw)) : shf;
      int Aleft;
      if (i == 0) {
        Aleft = s0 - 1;  // window start: the left neighbour's anchor is itself
      } else {
        const int shA = __shfl_up_sync(kFull, A[K - 1], 1);
        const uint32_t e = (static_cast<uint32_t>(t_begin + kWin * m + 1 + i) << 8);
        Aleft = is_l0 ? (s0 - 1 - static_cast<int>(static_cast<uint32_t>(pw >> 32) - e)) : shA;
      }
      step_pairs(left, Aleft, eb, el, bits, bit);
      // The word of this frame for the right neighbour is word i+1 of slot m
      // (word 0 of slot m+1 for the window's last frame); even frames store
      // it with the previous frame's word.
      const uint32_t hb = (static_cast<uint32_t>(t_begin + kWin * m + 1) << 8) + static_cast<uint32_t>(s_last);
      const uint64_t w = (static_cast<uint64_t>(hb + (static_cast<uint32_t>(i + 1) << 8) - static_cast<uint32_t>(A[K - 1])) << 32) |
                         __float_as_uint(a[K - 1]);
      if ((i & 1) == 0)
        send_pair(m, i, prev_w, w);
      else
        prev_w = w;
    };

    for (int m = 0; m < nwin_full && !dead; ++m) {
      if (!window_begin(m, kWin)) {
        dead = true;
        break;
      }
      const float* rowp = stage_f + c_stage * stage_floats;
      const uint32_t rslot_addr = r_data + static_cast<uint32_t>((m & (R - 1)) * kWin * 8);
#pragma unroll
      for (int i = 0; i < kWin; ++i) do_frame(m, i, rowp, rslot_addr);
      window_end_recv(m);
      end_window(m, t_begin + (m + 1) * kWin);
      if (__any_sync(kFull, *abort != 0)) dead = true;
    }
    if (!dead && rem > 0) {
      const int m = nwin_full;
      if (!window_begin(m, rem)) {
        dead = true;
      } else {
        const float* rowp = stage_f + c_stage * stage_floats;
        const uint32_t rslot_addr = r_data + static_cast<uint32_t>((m & (R - 1)) * kWin * 8);
        // The same straight-line frames as a full window, each behind a
        // warp-uniform guard: a loop over a runtime frame index runs about
        // three times slower per frame, and every warp of the pipeline waits
        // for its sender to finish this window, so a slow last window costs
        // its time once per warp boundary.
#pragma unroll
        for (int i = 0; i < kWin - 1; ++i)
          if (i < rem) do_frame(m, i, rowp, rslot_addr);
        window_end_recv(m);
        end_window(m, t_end - 1);
      }
    }
    // Release the stage of the last window (a persistent CTA's next job
    // continues the ring).
    if (!dead && nwin_all > 0) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&head->empty[c_stage]);
      if (++c_stage == P.stages) {
        c_stage = 0;
        ++c_round;
      }
    }
  } else {
  float carry_a = a[K - 1];  // alpha of the last state at the first frame of the next package
  int carry_A = A[K - 1];
  uint32_t bits[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) bits[w] = 0u;
  auto end_window = [&](const int m, const int t_last) { end_window_bits(bits, m, t_last); };
  int& c_stage = ring.c_stage;
  uint32_t& c_round = ring.c_round;
  int chunk = -1;  // chunk of this job whose stage is in use
  const float* stage_f = reinterpret_cast<const float*>(stages);
  const int stage_floats = P.stage_bytes / 4;

  // One block: frames t_begin+1+32m+iw0 .. +n-1 (iw0 a multiple of kB). `full`
  // is a compile-time true for blocks of kB frames (every block but possibly
  // the last of a pass); then no frame is guarded. Returns false when a
  // bounded wait ran out.
  auto run_block = [&](auto full, const int m, const int iw0, const int n) -> bool {
    constexpr bool kFullBlk = decltype(full)::value;
    const int ft0 = m * kWin + iw0;  // frames computed before this block
    // Emission chunk of this block: release the previous stage, wait for the
    // rows.
    if ((ft0 & (F - 1)) == 0) {
      if (chunk >= 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&head->empty[c_stage]);
        if (++c_stage == P.stages) {
          c_stage = 0;
          ++c_round;
        }
      }
      ++chunk;
      if (!warp_wait_phase(&head->full[c_stage], c_round & 1u, abort, limit, lane)) return false;
    }
    // Emission rows of the block (in the stage even past n).
    const float* pb = stage_f + c_stage * stage_floats + (ft0 & (F - 1)) * C + blank;
    const float* pl[K / 2];
#pragma unroll
    for (int q = 0; q < K / 2; ++q) pl[q] = pb - blank + col[q];
    float eb[kB];
    float el[kB][K / 2];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      eb[i] = pb[i * C];
#pragma unroll
      for (int q = 0; q < K / 2; ++q) el[i][q] = pl[q][i * C];
    }
    // Package pk from the left neighbour: alpha / anchor offset of its last
    // state at frames t_begin+32m+iw0 .. +kB-1 (lane 0 reads and checks it).
    float pa[kB];
    uint32_t poff[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      pa[i] = -INFINITY;
      poff[i] = 0u;
    }
    if (recv_left) {
      const int slot = static_cast<int>(pk) & (rslots - 1);
      const uint32_t e0 = static_cast<uint32_t>(t_begin + kB * static_cast<int>(pk) + 1) << 8;
      const uint32_t raddr = r_data + slot * kB * 8;
      const uint64_t* rp = rg_data ? rg_data + slot * kB : nullptr;
      bool ok = true;
      if (is_l0) ok = read_package<kB>(rscope, raddr, rp, e0, kFullBlk ? kB : n, pa, poff);
      if (__any_sync(kFull, !ok)) {
        if (!package_wait<kB>(rscope, raddr, rp, e0, kFullBlk ? kB : n, abort, limit)) return false;
        if (is_l0) (void)read_package<kB>(rscope, raddr, rp, e0, kFullBlk ? kB : n, pa, poff);
      }
      // Consumed: the sender may reuse the slot.
      if (is_l0) st_count(rscope, r_cons, rg ? rg + 1 : nullptr, pk + 1);
    }
    // Package for the right neighbour: [0] carried from the previous block,
    // [i + 1] after frame i.
    float sa[kB];
    int sA[kB];
    sa[0] = carry_a;
    sA[0] = carry_A;
    uint32_t bb[NW];  // this block's backpointer bits (bit i = frame iw0 + i)
#pragma unroll
    for (int w = 0; w < NW; ++w) bb[w] = 0u;
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      if (kFullBlk || i < n) {
        const float shf = __shfl_up_sync(kFull, a[K - 1], 1);
        const int shA = __shfl_up_sync(kFull, A[K - 1], 1);
        const float left = is_l0 ? pa[i] : shf;  // alpha_{t-1}(s0 - 1)
        int Aleft = is_l0 ? (s0 - 1 - static_cast<int>(poff[i])) : shA;
        // At a window's first frame the left neighbour's anchor is itself
        // (anchors are reset at window ends).
        if (i == 0 && iw0 == 0) Aleft = s0 - 1;
        const uint32_t bit = 1u << i;
        step_pairs(left, Aleft, eb[i], el[i], bb, bit);
        if (i + 1 < kB) {
          sa[i + 1] = a[K - 1];
          sA[i + 1] = A[K - 1];
        } else {
          carry_a = a[K - 1];
          carry_A = A[K - 1];
        }
      }
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) bits[w] |= bb[w] << iw0;
    if (has_next && !stall) {
      // The slot of package pk last held package pk - slots.
      const uint32_t need = (pk + 1 > static_cast<uint32_t>(sslots)) ? pk + 1 - sslots : 0u;
      if (cons_seen < need) {
        uint32_t v = need;
        if (lane == 31) v = ld_count(sscope, s_cons, sg ? sg + 1 : nullptr);
        cons_seen = __shfl_sync(kFull, v, 31);
        if (cons_seen < need) {
          if (!count_wait(sscope, s_cons, sg ? sg + 1 : nullptr, need, abort, limit)) return false;
          cons_seen = need;
        }
      }
      if (lane == 31) {
        const int slot = static_cast<int>(pk) & (sslots - 1);
        // High word: tag (frame + 1) << 8 plus the anchor offset s_last - A.
        const uint32_t hb = (static_cast<uint32_t>(t_begin + kB * static_cast<int>(pk) + 1) << 8) +
                            static_cast<uint32_t>(s_last);
        uint64_t w[kB];
#pragma unroll
        for (int i = 0; i < kB; ++i)
          w[i] = (static_cast<uint64_t>(hb + (static_cast<uint32_t>(i) << 8) - static_cast<uint32_t>(sA[i])) << 32) |
                 __float_as_uint(sa[i]);
        const uint32_t saddr = s_link + 16 + slot * kB * 8;
        uint64_t* sp = sg_data ? sg_data + slot * kB : nullptr;
#pragma unroll
        for (int q = 0; q < kB / 2; ++q) st_words(sscope, saddr + q * 16, sp ? sp + 2 * q : nullptr, w[2 * q], w[2 * q + 1]);
      }
    }
    ++pk;
    return true;
  };

  const std::true_type kFullBlock{};
  const std::false_type kPartBlock{};
  for (int m = 0; m < nwin_full && !dead; ++m) {
    for (int iw0 = 0; iw0 < kWin; iw0 += kB) {
      if (!run_block(kFullBlock, m, iw0, kB)) {
        dead = true;
        break;
      }
    }
    if (dead) break;
    end_window(m, t_begin + (m + 1) * kWin);
    if (__any_sync(kFull, *abort != 0)) dead = true;
  }
  if (!dead && rem > 0) {
    int iw0 = 0;
    for (; iw0 + kB <= rem && !dead; iw0 += kB) dead = !run_block(kFullBlock, nwin_full, iw0, kB);
    if (!dead && iw0 < rem) dead = !run_block(kPartBlock, nwin_full, iw0, rem - iw0);
    if (!dead) end_window(nwin_full, t_end - 1);
  }
  if (!dead && chunk >= 0) {  // release the last chunk's stage
    __syncwarp();
    if (lane == 0) mbar_arrive(&head->empty[c_stage]);
    if (++c_stage == P.stages) {
      c_stage = 0;
      ++c_round;
    }
  }
  }
  // ---- alpha_{T-1} of the two final states, to where tail 1 reads them:
  // CTA 0's shared memory (over DSMEM from another CTA of a cluster), or the
  // team block of a grid team (device memory) ----
  if (!dead && *abort == 0 && t_end == J.T && (J.flags & kJobWriteFinal)) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (s0 + j == S - 2 || s0 + j == S - 1) {
        const int k = s0 + j - (S - 2);
        if (xteam) {
          reinterpret_cast<float*>(xbar)[2 + k] = a[j];
        } else if (ncta > 1) {
          st_remote_u32(mapa_rank(smem_addr(&head->fin[k]), 0), __float_as_uint(a[j]));
        } else {
          head->fin[k] = a[j];
        }
      }
    }
  }

  }  // compute warps
  fence_proxy_async_smem();
  // Team barrier between the phases, and one decision for the whole team:
  // carry on unless a CTA's bounded wait ran out. A CTA whose wait ran out
  // marks the request timed out (the result block may be in host memory:
  // written, never read back here) and, before the barrier, raises the
  // team's flag in device-side memory: the team block of a grid team, or the
  // flag word in every CTA's shared memory in a cluster (pushed over DSMEM
  // while every CTA still waits at the barrier; after it a CTA reads only its
  // own shared memory, since another CTA may already have exited). The
  // cluster barrier orders memory at cluster scope and the grid barrier
  // fences at GPU scope, so no thread fences on its own.
  auto team_sync_ok = [&]() -> bool {
    __syncthreads();
    const bool mine = *abort != 0;  // no warp of this CTA writes it during the barrier
    if (threadIdx.x == 0 && mine) {
      atomicExch(J.status, kStTimeout);
      if (xteam) atomicExch(xbar + 4, 1u);
      if (!kGrid && ncta > 1)
        for (uint32_t r = 0; r < ncta; ++r) st_remote_u32(mapa_rank(smem_addr(&head->team_bad), r), 1u);
    }
    bool bad = mine;
    if (ncta > 1) {
      if constexpr (kGrid) {
        team_barrier(xbar, ncta, abort, limit);
        if (*abort != 0) {
          if (threadIdx.x == 0) atomicExch(J.status, kStTimeout);
          return false;
        }
        bad = threadIdx.x == 0 && __ldcg(xbar + 4) != 0u;
      } else {
        cluster_sync();
        bad = *reinterpret_cast<volatile uint32_t*>(&head->team_bad) != 0u;
      }
    }
    return __syncthreads_or(bad) == 0;
  };
  if (!team_sync_ok()) return;

  // ---- tail 1 (warp 0 of CTA 0): final state, total, hops back through the anchor rows ----
  // (The barrier before it also ordered every warp's shared-memory accesses
  // to links and stages before the bulk copies that reuse them: each thread
  // fenced them to the asynchronous proxy first.)
  const bool chase = (J.flags & kJobChase) != 0;
  int32_t final_code = kStPending;  // set by the thread that chooses the final state
  unsigned char* tail = smem + P.off_ring;  // links and stages are free now (hop buffer)
  if (crank == 0 && warp == 0) {
    int s_cur;
    if (J.flags & kJobWriteFinal) {
      const float* fin = xteam ? reinterpret_cast<const float*>(xbar) + 2 : head->fin;
      const float f_blank = xteam ? __ldcg(fin + 1) : fin[1];
      const float f_lab = (S > 1) ? (xteam ? __ldcg(fin + 0) : fin[0]) : -INFINITY;
      s_cur = (S > 1 && f_lab > f_blank) ? S - 2 : S - 1;
      const float tot = (S > 1 && f_lab > f_blank) ? f_lab : f_blank;
      final_code = (tot == -INFINITY) ? kStNoPath : kStOk;
      if (lane == 0) {
        if (J.total && !kNorm) *J.total = tot;  // logits: the score pass writes the total
        if (!chase) *J.state_io = s_cur;
      }
    } else {
      s_cur = __ldcg(J.state_io);
    }
    if (chase) {
      if (lane == 0) path[t_end - 1] = s_cur;
      // Batches of kHopBatch rows: lane r copies the slice [lo, hi) of row
      // m - r (16-byte aligned: rows are 16-byte multiples) with one bulk copy
      // on the tail barrier, then lane 0 hops through them in shared memory;
      // a hop that leaves the slice (below lo) reads its byte from global
      // memory in a loop of its own.
      uint8_t* zb = tail;  // [kHopBatch][kHopRowBytes]
      uint64_t* tbar = &head->tailbar;
      uint32_t& t_round = ring.t_round;
      for (int m = nwin - 1; m >= 0; m -= kHopBatch) {
        const int nb = min(kHopBatch, m + 1);
        const int lo = max(0, s_cur - kHopSpan) & ~15;
        const int hi = min(zstride, (s_cur + 16) & ~15);
        const uint32_t bytes = static_cast<uint32_t>(hi - lo);
        fence_proxy_async_smem();  // this warp's earlier reads of the buffer before the copies' writes
        __syncwarp();
        if (lane == 0) mbar_arrive_expect_tx(tbar, bytes * static_cast<uint32_t>(nb));
        __syncwarp();
        if (lane < nb) bulk_g2s(zb + lane * kHopRowBytes, ztab + static_cast<size_t>(m - lane) * zstride + lo, bytes, tbar);
        bool landed = true;
        if (lane == 0) {
          landed = wait_phase(tbar, t_round & 1u, abort, limit, false);
          if (!landed) (void)wait_phase(tbar, t_round & 1u, abort, limit, false);  // copies still in flight land first
        }
        ++t_round;
        if (lane == 0 && landed) {
          int r = 0;
          for (; r < nb; ++r) {
            const int off = s_cur - lo;
            if (off < 0) break;
            s_cur -= static_cast<int>(zb[r * kHopRowBytes + off]);
            path[t_begin + (m - r) * kAnchorD] = s_cur;
          }
          for (; r < nb; ++r) {
            s_cur -= static_cast<int>(__ldcg(ztab + static_cast<size_t>(m - r) * zstride + s_cur));
            path[t_begin + (m - r) * kAnchorD] = s_cur;
          }
        }
        s_cur = __shfl_sync(kFull, s_cur, 0);
        if (__shfl_sync(kFull, landed ? 1 : 0, 0) == 0) break;  // the abort flag is raised
      }
      if (lane == 0) *J.state_io = s_cur;
    }
  }
  // The request's result code, once its job is done (the last write of the
  // job to its result block).
  auto finish = [&]() {
    if (crank == 0 && threadIdx.x == 0 && final_code != kStPending) atomicCAS(J.status, kStPending, final_code);
  };
  if (!chase) {
    finish();
    return;
  }
  if (!team_sync_ok()) return;

  // ---- tail 2 (every lane of the team): walk the windows in parallel ----
  // Window m covers frames (b, e], b = t_begin + 32m, e = min(b + 32, t_end - 1);
  // its top state is path[e]. The words of a state hold all 32 frames of the
  // window, and the K + 1 words of a lane hold its K states, so a walk loads a
  // lane's words together (independent loads, one round trip). The path only
  // moves down, at most 2 <= K states a frame, so the lane it enters next is
  // the one below: its words are loaded while the walk is in the current
  // lane's states.
  constexpr int kWords = K + 1;
  const int nwalk = max(nwin, 1);
  for (int m = g * 32 + lane; !producer && m < nwalk; m += G * 32) {
    const int b = t_begin + m * kAnchorD;
    const int e = (nwin == 0) ? t_begin : min(b + kAnchorD, t_end - 1);
    const uint32_t* wbase = bp + static_cast<size_t>(m) * G * NW * 32;
    auto lane_words = [&](const int lg, uint32_t (&dst)[kWords]) {
      if (lg >= 0) {
        const uint32_t* w = wbase + static_cast<size_t>(lg >> 5) * NW * 32 + (lg & 31);
#pragma unroll
        for (int q = 0; q < kWords; ++q) dst[q] = w[q * 32];
      } else {
#pragma unroll
        for (int q = 0; q < kWords; ++q) dst[q] = 0u;
      }
    };
    int sc = path[e];
    int cur = sc / K;  // lane (over the team) whose words are in wv; wn: the lane below
    {
      // The walk stays in the lanes between its bottom state (path[b], from
      // tail 1) and its top state; word q of 32 consecutive lanes is one
      // 128-byte line, so the lines of up to two warps of lanes are pulled
      // into L1 with independent loads and one wait. (Otherwise a lane
      // switching to new words waits an L2 round trip, and the warp's
      // scoreboard makes every lane wait for every other lane's loads.)
      const int hi_g = cur >> 5, lo_g = min((max(path[b], 0) / K) >> 5, hi_g);
      const uint32_t* l0 = wbase + static_cast<size_t>(lo_g) * NW * 32;
      const uint32_t* l1 = wbase + static_cast<size_t>(min(lo_g + 1, hi_g)) * NW * 32;
      uint32_t v[2 * kWords];
#pragma unroll
      for (int q = 0; q < kWords; ++q) {
        v[q] = __ldca(l0 + q * 32);
        v[kWords + q] = __ldca(l1 + q * 32);
      }
      uint32_t acc = 0u;
#pragma unroll
      for (int q = 0; q < 2 * kWords; ++q) acc ^= v[q];
      asm volatile("" ::"r"(acc));
    }
    uint32_t wv[kWords], wn[kWords];
    lane_words(cur, wv);
    lane_words(cur - 1, wn);
    for (int f = e; f > b; --f) {
      path[f] = sc;
      const int lg = sc / K;
      if (lg != cur) {
        cur = lg;
#pragma unroll
        for (int q = 0; q < kWords; ++q) wv[q] = wn[q];
        lane_words(lg - 1, wn);
      }
      const int j = sc - lg * K;
      uint32_t mw = wv[0], bw = 0u;  // the state's word; for a label state, the blank state's below it
#pragma unroll
      for (int q = 1; q < K; ++q) mw = (j == q) ? wv[q] : mw;
#pragma unroll
      for (int q = 0; q < K / 2; ++q) bw = (j == 2 * q + 1) ? wv[2 * q] : bw;
      const int i = f - b - 1;
      int step = static_cast<int>((mw >> i) & 1u);
      if (step && (j & 1) && ((bw >> i) & 1u) && ((wv[K] >> (j >> 1)) & 1u)) step = 2;
      sc -= step;
    }
    if (m == 0) path[b] = sc;
  }
  if (!team_sync_ok()) return;

  // ---- tail 3 (every thread of the team): states -> tokens, states, scores ----
  constexpr int kT3 = 8;
  const int tid = g * 32 + lane;
  const int nthr = G * 32;
  float part = 0.0f;  // logits: this thread's sum of scores (its frames in order)
  for (int f0 = t_begin + tid; !producer && f0 < t_end; f0 += kT3 * nthr) {
    int st[kT3], tok[kT3];
    float sv[kT3];
#pragma unroll
    for (int k = 0; k < kT3; ++k) {
      const int f = f0 + k * nthr;
      st[k] = (f < t_end) ? path[f] : 0;
    }
#pragma unroll
    for (int k = 0; k < kT3; ++k) tok[k] = (st[k] & 1) ? __ldg(tgt + (st[k] >> 1)) : blank;
#pragma unroll
    for (int k = 0; k < kT3; ++k) {
      const int f = f0 + k * nthr;
      sv[k] = (f < t_end) ? __ldg(lp + static_cast<size_t>(f) * C + tok[k]) : 0.0f;
      if constexpr (kNorm) {
        if (f < t_end) sv[k] -= row_lse(lp + static_cast<size_t>(f) * C, C, (J.flags & kJobBulkRows) != 0);
      }
    }
#pragma unroll
    for (int k = 0; k < kT3; ++k) {
      const int f = f0 + k * nthr;
      if (f < t_end) {
        path[f] = tok[k];
        if (states_out) states_out[f] = st[k];
        scores_out[f] = sv[k];
        if constexpr (kNorm) part += sv[k];
      }
    }
  }
  if constexpr (kNorm) {
    // Total = sum of the scores in a fixed order: per thread, a butterfly over
    // the warp (every lane ends with the same bits), warps in team order.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (lane == 0 && !producer) J.lse[g] = part;
    if (!team_sync_ok()) return;
    if (crank == 0 && warp == 0 && lane == 0 && (J.flags & kJobWriteFinal) && J.total) {
      float tot = 0.0f;
      for (int w = 0; w < G; ++w) tot += __ldcg(J.lse + w);
      *J.total = tot;
    }
  }
  finish();
}

// Stage barriers of the emission ring: `full` completes when a stage's rows
// have landed (one arrival with the byte count for bulk copies, 32 for the
// per-float fallback), `empty` when every compute warp released it.
__device__ __forceinline__ void init_stage_barriers(const FwdParams& P, bool bulk) {
  SmemHead* head = reinterpret_cast<SmemHead*>(fast_smem());
  if (threadIdx.x == 0) {
    for (int st = 0; st < P.stages; ++st) {
      mbar_init(&head->full[st], bulk ? 1u : 32u);
      mbar_init(&head->empty[st], static_cast<uint32_t>((blockDim.x >> 5) - 1));
    }
    mbar_init(&head->tailbar, 1u);
    fence_barrier_init();
  }
  __syncthreads();
}

// One team per job: a thread-block cluster (or one CTA), or a grid team of
// P.grid_ctas consecutive CTAs of a cooperative launch.
template <int K, int kB, bool kGrid, bool kNorm, int kC>
__global__ void __launch_bounds__(512, 1) trellis_fast_kernel(const FwdJob* __restrict__ jobs, const FwdParams P) {
  const uint32_t ncta = kGrid ? static_cast<uint32_t>(max(P.grid_ctas, 1)) : cluster_nctarank();
  const uint32_t crank = kGrid ? blockIdx.x % ncta : cluster_ctarank();
  // The descriptor is read once into shared memory (it may live in pinned
  // host memory, where every field access would cross the chip link).
  FwdJob& sjob = reinterpret_cast<SmemHead*>(fast_smem())->job;
  static_assert(sizeof(FwdJob) % 16 == 0, "descriptor copied in 16-byte words");
  {
    const uint4* src = reinterpret_cast<const uint4*>(jobs + blockIdx.x / ncta);
    uint4* dst = reinterpret_cast<uint4*>(&sjob);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(FwdJob) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  init_stage_barriers(P, (sjob.flags & kJobBulkRows) != 0);
  StageRing ring;
  team_job<K, kB, kGrid, kNorm, kC>(sjob, P, ncta, crank, ring);
}

// Persistent launch: every CTA of a cooperative launch (all resident) takes
// seats from a counter in order. Seat x belongs to job seat_job[x] (jobs
// ordered longest first, each with team_ctas consecutive seats from
// first_seat); a job of several CTAs links them through global memory as a
// grid team does. Seats are handed out in order and every CTA is resident,
// so each team fills: the CTAs of earlier jobs finish and take later seats.
template <int K, int kB, bool kNorm, int kC>
__global__ void __launch_bounds__(512, 1) trellis_persist_kernel(const FwdJob* __restrict__ jobs, const FwdParams P,
                                                                 const int32_t* __restrict__ seat_job,
                                                                 int32_t total_seats, int32_t* counter) {
  SmemHead* head = reinterpret_cast<SmemHead*>(fast_smem());
  init_stage_barriers(P, true);  // every job of a persistent launch has 16-byte rows
  StageRing ring;
  for (;;) {
    if (threadIdx.x == 0) head->unused = static_cast<uint32_t>(atomicAdd(counter, 1));
    __syncthreads();
    const int seat = static_cast<int>(head->unused);
    if (seat >= total_seats) break;  // the same seat in every thread
    // The seat's descriptor into shared memory (the table and descriptors may
    // live in pinned host memory).
    {
      const uint4* src = reinterpret_cast<const uint4*>(jobs + seat_job[seat]);
      uint4* dst = reinterpret_cast<uint4*>(&head->job);
      for (int i = threadIdx.x; i < static_cast<int>(sizeof(FwdJob) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const FwdJob& J = head->job;
    team_job<K, kB, true, kNorm, kC>(J, P, static_cast<uint32_t>(J.team_ctas), static_cast<uint32_t>(seat - J.first_seat),
                                 ring);
    // The backtrack used the links and stages as scratch: the next job's
    // bulk copies write there.
    fence_proxy_async_smem();
    __syncthreads();
    if (*reinterpret_cast<volatile int32_t*>(&head->abort) != 0) break;  // the ring's phases are not trusted after a wait ran out
  }
}

template <int K, int kB, bool kGrid, bool kNorm, int kC>
cudaError_t launch_fast_k(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                          cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int smem_max = max_smem_optin(dev);
  int smem = smem_bytes(shape, p);
  if (kGrid) {
    smem = std::max(smem, smem_max);  // one CTA per SM (see the generic launcher)
    if (njobs != 1) return cudaErrorInvalidValue;
  }
  auto fn = trellis_fast_kernel<K, kB, kGrid, kNorm, kC>;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  if (smem > smem_max) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(njobs * shape.ncta), 1, 1);
  cfg.blockDim = dim3(static_cast<unsigned>((shape.warps + 1) * 32), 1, 1);  // + the producer warp
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  if (kGrid) {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  } else if (shape.ncta > 1) {
    if (shape.ncta > 8) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(shape.ncta);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, fn, d_jobs, p);
}

template <int K, int kB, int kC>
cudaError_t launch_fast_kc(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                           cudaStream_t s) {
  if (shape.grid) {
    if (shape.norm) return launch_fast_k<K, kB, true, true, kC>(shape, p, d_jobs, njobs, s);
    return launch_fast_k<K, kB, true, false, kC>(shape, p, d_jobs, njobs, s);
  }
  if (shape.norm) return launch_fast_k<K, kB, false, true, kC>(shape, p, d_jobs, njobs, s);
  return launch_fast_k<K, kB, false, false, kC>(shape, p, d_jobs, njobs, s);
}

template <int K, int kB>
cudaError_t launch_fast_kb(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                           cudaStream_t s) {
  if constexpr (kB == kAnchorD) {
    if (p.row_c == 32) return launch_fast_kc<K, kB, 32>(shape, p, d_jobs, njobs, s);
  }
  return launch_fast_kc<K, kB, 0>(shape, p, d_jobs, njobs, s);
}

template <int K, int kB>
cudaError_t persist_fn(const FwdParams& p, void (**fn)(const FwdJob*, FwdParams, const int32_t*, int32_t, int32_t*)) {
  if constexpr (kB == kAnchorD) {
    if (p.row_c == 32) {
      *fn = trellis_persist_kernel<K, kB, false, 32>;
      return cudaSuccess;
    }
  }
  *fn = trellis_persist_kernel<K, kB, false, 0>;
  return cudaSuccess;
}

cudaError_t persist_kernel_of(const LaunchShape& shape, const FwdParams& p,
                              void (**fn)(const FwdJob*, FwdParams, const int32_t*, int32_t, int32_t*)) {
  if (shape.norm || shape.sum) return cudaErrorInvalidValue;  // persistent launches align log-probabilities
  if (shape.K == 2 && p.kb == kAnchorD) return persist_fn<2, kAnchorD>(p, fn);
  if (shape.K == 2 && p.kb == 4) return persist_fn<2, 4>(p, fn);
  if (shape.K == 4 && p.kb == kAnchorD) return persist_fn<4, kAnchorD>(p, fn);
  if (shape.K == 4 && p.kb == 4) return persist_fn<4, 4>(p, fn);
  return cudaErrorInvalidValue;
}

}  // namespace

int persist_max_ctas(const LaunchShape& shape, const FwdParams& p, int device, int* ctas) {
  void (*fn)(const FwdJob*, FwdParams, const int32_t*, int32_t, int32_t*) = nullptr;
  cudaError_t e = persist_kernel_of(shape, p, &fn);
  if (e != cudaSuccess) return e;
  const int smem_max = max_smem_optin(device);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (shape.warps + 1) * 32,
                                                    static_cast<size_t>(smem_bytes(shape, p)));
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  *ctas = per_sm * sms;
  return cudaSuccess;
}

int launch_trellis_persist(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs,
                           const int32_t* d_seat_job, int32_t total_seats, int32_t* d_counter, int ctas,
                           void* stream) {
  if (total_seats <= 0) return cudaSuccess;
  void (*fn)(const FwdJob*, FwdParams, const int32_t*, int32_t, int32_t*) = nullptr;
  cudaError_t e = persist_kernel_of(shape, p, &fn);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int smem_max = max_smem_optin(dev);
  const int smem = smem_bytes(shape, p);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  if (smem > smem_max || ctas < 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(std::min(ctas, static_cast<int>(total_seats))), 1, 1);
  cfg.blockDim = dim3(static_cast<unsigned>((shape.warps + 1) * 32), 1, 1);  // + the producer warp
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = static_cast<cudaStream_t>(stream);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: teams fill (see the kernel)
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, d_jobs, p, d_seat_job, total_seats, d_counter);
}

int launch_trellis_fast(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                        void* stream) {
  if (njobs <= 0) return cudaSuccess;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (shape.sum) return cudaErrorInvalidValue;  // the sum-product runs on the generic kernel
  if (shape.K == 2 && p.kb == kAnchorD) return launch_fast_kb<2, kAnchorD>(shape, p, d_jobs, njobs, s);
  if (shape.K == 2 && p.kb == 4) return launch_fast_kb<2, 4>(shape, p, d_jobs, njobs, s);
  if (shape.K == 4 && p.kb == kAnchorD) return launch_fast_kb<4, kAnchorD>(shape, p, d_jobs, njobs, s);
  if (shape.K == 4 && p.kb == 4) return launch_fast_kb<4, 4>(shape, p, d_jobs, njobs, s);
  return cudaErrorInvalidValue;
}

}  // namespace gb300_align
