// Trellis kernels for CTC forced alignment on sm_103a.
//
// One kernel does the whole hot path of one alignment: Viterbi forward over
// the CTC trellis (max-plus recursion, the method of the TorchAudio 2.1 paper
// Sec. 4 "CTC-based forced alignment" on the trellis of the cited CTC work),
// 2-bit backpointers packed by warp ballots, the final-state choice and the
// windowed backtrack that writes path / scores / total.
//
//   alpha_t(s) = max(alpha_{t-1}(s), alpha_{t-1}(s-1), alpha_{t-1}(s-2)) + lp[t][ext[s]]
//   (s-2 only into a label state whose label differs from state s-2's;
//    ties keep the earlier candidate in the order s, s-1, s-2)
//
// Bit-exactness: every cell is one FP32 add after an exact max, with the same
// strict comparisons and candidate order as the definition, so the result
// does not depend on how the states are spread over lanes, warps or CTAs.
// Built without fast-math and without flush-to-zero.
//
// Parallel structure (see trellis.cuh): a team of warps chained along s runs
// as a skewed pipeline. Emission rows are staged per CTA in a 4-stage shared
// ring filled by cp.async.bulk (TMA bulk copies) completing on mbarriers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cfloat>
#include <cstdint>

#include "trellis.cuh"
#include "trellis_common.cuh"

namespace gb300_align {
namespace {

template <int K>
__device__ __forceinline__ void store_bp_words(uint32_t* dst, const uint32_t (&adv)[K], const uint32_t (&skp)[K / 2]) {
  constexpr int NW = bp_words(K);
  uint32_t w[NW];
#pragma unroll
  for (int j = 0; j < K; ++j) w[j] = adv[j];
#pragma unroll
  for (int i = 0; i < K / 2; ++i) w[K + i] = skp[i];
  if constexpr (NW % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NW; i += 4)
      *reinterpret_cast<uint4*>(dst + i) = make_uint4(w[i], w[i + 1], w[i + 2], w[i + 3]);
  } else if constexpr (NW % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NW; i += 2) *reinterpret_cast<uint2*>(dst + i) = make_uint2(w[i], w[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i) dst[i] = w[i];
  }
}

// Slow path of a block read: lane i waits (bounded) until its slot carries
// the tag of frame t0 + i; returns the value bits. Uniform across the warp.
__device__ __noinline__ uint64_t ring_block_spin(const volatile uint64_t* ring, int t0, int nb, int rb_mask,
                                                 int lane, volatile int32_t* abort, uint64_t limit) {
  const uint64_t t_start = gtimer();
  const int f = t0 + (lane < nb ? lane : 0);
  const uint32_t want = (static_cast<uint32_t>(f) + 1u) & ((1u << kTagBits) - 1u);
  const volatile uint64_t* p = ring + (f & rb_mask);
  for (;;) {
    const uint64_t v = *p;
    const bool mine = static_cast<uint32_t>(v >> 40) == want;  // tag field of the ring word
    if (__all_sync(kFull, mine)) return v;
    const bool give_up = (*abort != 0) || (gtimer() - t_start > limit);
    if (__any_sync(kFull, give_up)) {
      if (lane == 0) *abort = 1;
      return static_cast<uint64_t>(__float_as_uint(-INFINITY));
    }
  }
}

// All backpointer words of one warp and frame, stored by lane 0 under a single
// predicate (one setp per frame).
template <int K>
__device__ __forceinline__ void store_bp_words_if(uint32_t* dst, const uint32_t (&adv)[K],
                                                  const uint32_t (&skp)[K / 2], bool pred) {
  const uint32_t pr = static_cast<uint32_t>(pred);
  if constexpr (K == 2) {  // 3 words: 4-byte aligned only
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t"
        "@q st.global.u32 [%0], %1;\n\t@q st.global.u32 [%0+4], %2;\n\t@q st.global.u32 [%0+8], %3;\n\t}" ::"l"(dst),
        "r"(adv[0]), "r"(adv[1]), "r"(skp[0]), "r"(pr)
        : "memory");
  } else if constexpr (K == 4) {  // 6 words: 8-byte aligned
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %7, 0;\n\t"
        "@q st.global.v2.u32 [%0], {%1, %2};\n\t@q st.global.v2.u32 [%0+8], {%3, %4};\n\t"
        "@q st.global.v2.u32 [%0+16], {%5, %6};\n\t}" ::"l"(dst),
        "r"(adv[0]), "r"(adv[1]), "r"(adv[2]), "r"(adv[3]), "r"(skp[0]), "r"(skp[1]), "r"(pr)
        : "memory");
  } else if constexpr (K == 8) {  // 12 words: 16-byte aligned
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %13, 0;\n\t"
        "@q st.global.v4.u32 [%0], {%1, %2, %3, %4};\n\t@q st.global.v4.u32 [%0+16], {%5, %6, %7, %8};\n\t"
        "@q st.global.v4.u32 [%0+32], {%9, %10, %11, %12};\n\t}" ::"l"(dst),
        "r"(adv[0]), "r"(adv[1]), "r"(adv[2]), "r"(adv[3]), "r"(adv[4]), "r"(adv[5]), "r"(adv[6]), "r"(adv[7]),
        "r"(skp[0]), "r"(skp[1]), "r"(skp[2]), "r"(skp[3]), "r"(pr)
        : "memory");
  } else {  // K == 16: 24 words
    constexpr int NW = bp_words(K);
    uint32_t w[NW];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = adv[j];
#pragma unroll
    for (int i = 0; i < K / 2; ++i) w[K + i] = skp[i];
#pragma unroll
    for (int i = 0; i < NW; i += 4) st_global_v4_if(dst + i, w[i], w[i + 1], w[i + 2], w[i + 3], pred);
  }
}

// Sum-product in base 2: values are log2 of probabilities, so the log-add
// needs only the hardware 2^x and log2(x) (PTX ex2.approx / lg2.approx, no
// flush to zero). The largest term is factored out; clamping it to -FLT_MAX
// and using 1 for the largest term (0 when every term is -inf) avoids both a
// branch and one exponential.
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// The largest term contributes 2^0 = 1 (0 when every term is -inf), so only
// the others need an exponential.
__device__ __forceinline__ float log2_add2(float x, float y) {
  const float mr = fmaxf(x, y);
  const float m = fmaxf(mr, -FLT_MAX);
  const float one = (mr == -INFINITY) ? 0.0f : 1.0f;
  return m + lg2_approx(one + ex2_approx(fminf(x, y) - m));
}
__device__ __forceinline__ float log2_add3(float x, float y, float z) {
  const float lo = fminf(x, y), hi = fmaxf(x, y);
  const float mr = fmaxf(hi, z);
  const float mid = fminf(hi, z);  // with lo, the two terms below the largest
  const float m = fmaxf(mr, -FLT_MAX);
  const float one = (mr == -INFINITY) ? 0.0f : 1.0f;
  return m + lg2_approx(one + ex2_approx(lo - m) + ex2_approx(mid - m));
}
constexpr float kLog2e = 1.4426950408889634f;  // log2(e): natural-log emissions to base 2
constexpr float kLn2 = 0.6931471805599453f;    // ln(2): the base-2 total back to natural log

// One backpointer row (NW = 3 or 6 words) stored by the lane that buffered it.
template <int K, int NWB>
__device__ __forceinline__ void store_bp_row(uint32_t* dst, const uint32_t (&w)[NWB]) {
  if constexpr (NWB == 3) {  // 12-byte rows: 4-byte aligned
    dst[0] = w[0];
    dst[1] = w[1];
    dst[2] = w[2];
  } else if constexpr (NWB == 6) {  // 24-byte rows: 8-byte aligned
    *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
    *reinterpret_cast<uint2*>(dst + 2) = make_uint2(w[2], w[3]);
    *reinterpret_cast<uint2*>(dst + 4) = make_uint2(w[4], w[5]);
  }
}

// ------------------------------------------------------------------ kernel --
// kOcc: the register budget of K <= 4 is capped at 64 per thread (two
// 512-thread CTAs per SM), trading per-warp latency for resident warps.
//
// kGrid: the team is P.grid_ctas consecutive CTAs of a cooperative launch
// (one per SM) instead of a thread-block cluster; the links between CTAs (the
// boundary rings, progress words, barrier) are in global memory.
//
// kNorm: log_probs hold raw logits; the per-frame log_softmax shifts come
// from lse_prepass_kernel and are subtracted as the emissions are used (a
// separate instantiation so the log-probability path keeps its own code).
//
// kSum: the sum-product variant: log-add in place of the max (no
// backpointers, anchors or backtrack), in base 2 (log2 of probabilities);
// the job's total is the log-add of the two final states, back in natural log.
template <int K, bool kOcc, bool kGrid, bool kNorm, bool kSum>
__global__ void __launch_bounds__(512, (kOcc && K <= 4) ? 2 : 1)
    trellis_kernel(const FwdJob* __restrict__ jobs, const FwdParams P) {
  static_assert(K % 2 == 0 && K >= 2 && K <= 16, "K must be even, 2..16");
  constexpr int NW = bp_words(K);
  constexpr int GS = 32 * K;  // states per warp
  extern __shared__ __align__(128) unsigned char smem[];
  SmemHead* head = reinterpret_cast<SmemHead*>(smem);
  uint64_t* ring = reinterpret_cast<uint64_t*>(smem + P.off_ring);
  unsigned char* stages = smem + P.off_stage;
  volatile int32_t* abort = &head->abort;

  const uint32_t ncta = kGrid ? static_cast<uint32_t>(max(P.grid_ctas, 1)) : cluster_nctarank();
  const uint32_t crank = kGrid ? blockIdx.x % ncta : cluster_ctarank();
  // Logits mode (kNorm): the per-frame log_softmax shifts come from the lse
  // pre-pass (J.lse, written by lse_prepass_kernel before this launch); the
  // warps subtract them from the staged raw logits as they use them.
  const int W = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const FwdJob& J = jobs[blockIdx.x / ncta];
  const int g = static_cast<int>(crank) * W + warp;  // warp index in the team
  const int S = J.S, C = J.C, blank = J.blank;
  const int t_begin = J.t_begin, t_end = J.t_end;
  const int s0 = (g * 32 + lane) * K;               // first state of this lane
  const int F = P.frames_per_stage;
  const int rb_mask = P.rb - 1;
  const int nchunks = (t_end - 1 - t_begin + F - 1) / F;  // chunks of frames t_begin+1 .. t_end-1
  const bool bulk = (J.flags & kJobBulkRows) != 0;
  const uint64_t limit = P.wait_limit_ns;
  const float* __restrict__ lp = J.lp;
  uint32_t* __restrict__ bp = J.bp;
  const int bp_rows = J.bp_rows;
  float* __restrict__ ckpt = J.ckpt;
  const int ck_every = J.ck_every;
  const int ck_stride = J.ck_stride;
  // Output pointers in registers: stores through them could alias the
  // descriptor, and re-reading it from global memory after every store put a
  // memory round trip on each step of the backtrack.
  int32_t* const path = J.path;
  float* const scores_out = J.scores;
  int32_t* const states_out = J.states;
  const int32_t* const tgt = J.tgt;
  float* const lse_g = J.lse;  // logits mode: per-frame log_softmax shift

  // Launch parameters must fit the job: a stage holds F rows of C floats and
  // the team holds every state. The check is uniform over the cluster (same
  // job, same parameters), so every CTA leaves before any cluster barrier.
  // F and the receive block are powers of two dividing kAnchorD, and checkpoint
  // frames fall on window ends.
  const bool pow2_ok = F >= 1 && F <= kAnchorD && (F & (F - 1)) == 0 && P.block >= 1 && P.block <= kAnchorD &&
                       (P.block & (P.block - 1)) == 0;
  const bool ck_ok = ckpt == nullptr || (ck_every > 0 && ck_every % kAnchorD == 0 && t_begin % ck_every == 0);
  if (F * C * 4 > P.stage_bytes || static_cast<int64_t>(ncta) * W * 32 * K < S || P.stages < kLead ||
      P.stages > kMaxStages || !pow2_ok || !ck_ok || (kGrid && (P.grid_ctas < 1 || J.xlink == nullptr ||
                                                                  P.rb > kMaxRing))) {
    if (threadIdx.x == 0 && crank == 0) atomicExch(J.status, kStBadLaunch);
    return;
  }

  // ---- shared state: rings zeroed, barriers initialised ----
  for (int i = threadIdx.x; i < W * P.rb; i += blockDim.x) ring[i] = 0ull;
  if (threadIdx.x == 0) {
    for (int st = 0; st < P.stages; ++st) {
      mbar_init(&head->full[st], bulk ? 1u : 32u);
      mbar_init(&head->empty[st], static_cast<uint32_t>(W));
    }
    head->abort = 0;
    fence_barrier_init();
  }
  __syncthreads();
  // Neighbours' rings exist and are zero before any remote store (grid teams:
  // the global links were zeroed before the launch).
  if (!kGrid && ncta > 1) cluster_sync();

  // ---- per-lane constants: label columns and skip caps of the label states ----
  int col[K / 2];
  // Skip into label state i of this lane allowed: as a predicate (K <= 4), or
  // as masks that turn alpha(s-2) into -inf when it is not (K >= 8, where
  // predicate registers run out). Either way a forbidden skip never wins and
  // an allowed one compares alpha(s-2) itself, as in the definition.
  bool skok[K / 2];
  uint32_t skeep[K / 2], sfill[K / 2];
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
    skeep[i] = skip ? 0xffffffffu : 0u;
    sfill[i] = skip ? 0u : 0xff800000u;  // -inf
  }

  // ---- emission staging (warp 0 of each CTA is the producer) ----
  // Chunk c holds the rows of frames t_begin+1+c*F .. t_begin+(c+1)*F and goes
  // to stage c mod stages (round c / stages). F is a power of two dividing
  // kAnchorD, so chunks tile the anchor windows. The row of frame t_begin is
  // read directly by the lanes that need it.
  int issued = 0;         // chunks issued (producer)
  int p_stage = 0;        // stage of chunk `issued`
  uint32_t p_round = 0;   // round of chunk `issued`
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
  if (warp == 0) {
    const int first = min(kLead, nchunks);
    for (int c = 0; c < first; ++c) issue_next();
  }

  // ---- frame t_begin: initialisation ----
  float a[K];
  int A[K];  // anchors: state at the last anchor frame on the best path to each state
  if (J.alpha_in == nullptr) {
    // alpha_0: paths start in the blank (state 0) or the first label (state 1).
    const float* row = lp + static_cast<size_t>(t_begin) * C;
    float lse0 = 0.0f;
    if constexpr (kNorm) lse0 = __ldg(lse_g + t_begin);  // logits mode: this row's shift
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int s = s0 + j;
      if constexpr (kNorm)
        a[j] = (s == 0) ? __ldg(row + blank) - lse0 : ((s == 1 && S > 1) ? __ldg(row + col[0]) - lse0 : -INFINITY);
      else
        a[j] = (s == 0) ? __ldg(row + blank) : ((s == 1 && S > 1) ? __ldg(row + col[0]) : -INFINITY);
      if constexpr (kSum) a[j] *= kLog2e;  // the sum-product runs in base 2
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int s = s0 + j;
      a[j] = (s < S) ? __ldg(J.alpha_in + s) : -INFINITY;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) A[j] = s0 + j;

  // Ring endpoints. Each warp receives alpha(first state - 1) of frame t-1
  // from its own ring (written by the previous warp of the team, in this CTA
  // or over DSMEM from the previous CTA) and sends alpha(last state) of
  // frame t to the next warp's ring; the last warp of the team writes a sink.
  // Frames are processed in blocks of up to P.block frames: a receiver waits
  // once per block (lane i holds the word of frame t-1+i), publishes its
  // progress once per block, and a sender checks that progress once per block
  // before reusing ring slots. Lane 0 / lane 31 stores are predicated PTX, so
  // inside a block the only branch is the loop's own.
  uint32_t* prog_w = reinterpret_cast<uint32_t*>(smem + sizeof(SmemHead));  // [32]: progress of my consumer
  const bool recv_left = (g > 0);
  const bool send_local = warp < W - 1;
  const bool send_remote = (warp == W - 1) && (crank + 1 < ncta);
  const bool has_next = send_local || send_remote;
  if (threadIdx.x < 32) prog_w[threadIdx.x] = static_cast<uint32_t>(t_begin);
  __syncthreads();
  if (!kGrid && ncta > 1) cluster_sync();  // progress words initialised before any remote publish
  // Grid teams: ring b (CTA b's last warp -> CTA b+1) at xlink + b * kMaxRing,
  // then prog[b] (how far CTA b+1 has read ring b), then the team barrier.
  uint64_t* const xring = kGrid ? J.xlink : nullptr;
  uint32_t* const xprog = kGrid ? reinterpret_cast<uint32_t*>(J.xlink + static_cast<size_t>(ncta - 1) * kMaxRing) : nullptr;
  uint32_t* const xbar = kGrid ? xprog + ((ncta + 3u) & ~3u) : nullptr;
  // Team barrier with a uniform give-up decision (see the tails below).
  auto team_sync_ok = [&]() -> bool {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && *abort != 0) atomicExch(J.status, kStTimeout);
    if constexpr (kGrid) {
      team_barrier(xbar, ncta, abort, limit);  // ends with __syncthreads
      if (*abort != 0) {                       // this CTA's barrier wait ran out
        if (threadIdx.x == 0) atomicExch(J.status, kStTimeout);
        return false;
      }
    } else if (ncta > 1) {
      cluster_sync();
    } else {
      __syncthreads();
    }
    return *reinterpret_cast<const volatile int32_t*>(J.status) != kStTimeout;
  };
  const uint32_t send_base = kGrid ? 0u
                             : send_local  ? smem_addr(ring + (warp + 1) * P.rb)
                             : send_remote ? mapa_rank(smem_addr(ring), crank + 1)
                                           : smem_addr(&head->sink);
  uint64_t* const send_ptr = !kGrid ? nullptr
                             : send_local  ? ring + (warp + 1) * P.rb
                             : send_remote ? xring + static_cast<size_t>(crank) * kMaxRing
                                           : &head->sink;
  const uint32_t send_mask = has_next ? static_cast<uint32_t>(rb_mask) : 0u;
  // Where this warp publishes how far it has read its ring (its producer's prog_w slot).
  const uint32_t prog_dst = (kGrid || !recv_left) ? 0u
                            : (warp > 0) ? smem_addr(prog_w + (warp - 1))
                                         : mapa_rank(smem_addr(prog_w + (W - 1)), crank - 1);
  uint32_t* const prog_dst_g = (!kGrid || !recv_left) ? nullptr
                               : (warp > 0) ? prog_w + (warp - 1)
                                            : xprog + (crank - 1);
  // Progress of the warp this one sends to.
  const volatile uint32_t* my_prog = (kGrid && send_remote) ? xprog + crank : prog_w + warp;
  int prog_seen = t_begin;                           // consumer has read every frame < prog_seen
  const bool is_l0 = (lane == 0);
  const bool is_l31 = (lane == 31) && !((J.flags & kJobTestStall) && g == 0);
  const uint64_t* my_ring = (kGrid && warp == 0 && crank > 0) ? xring + static_cast<size_t>(crank - 1) * kMaxRing
                                                               : ring + warp * P.rb;
  constexpr uint32_t kTagMask = (1u << kTagBits) - 1u;
  const int s_last = s0 + K - 1;

  auto store_ckpt = [&](int t) {
    float* dst = ckpt + static_cast<size_t>(t / ck_every) * ck_stride;
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (s0 + j < S) dst[s0 + j] = a[j];
  };
  auto send_one = [&](int t, float v, int anc) {
    // High word: tag (t+1 mod 2^24) << 8 | anchor offset; low word: alpha bits.
    // One 64-bit store: a reader that sees the tag also sees the value.
    const uint32_t hi = ((static_cast<uint32_t>(t) + 1u) << 8) + (static_cast<uint32_t>(s_last - anc) & 0xffu);
    const uint64_t word = (static_cast<uint64_t>(hi) << 32) | __float_as_uint(v);
    if constexpr (kGrid)
      st_gpu_u64_if(send_ptr + (static_cast<uint32_t>(t) & send_mask), word, is_l31);
    else
      st_cluster_u64_if(send_base + (static_cast<uint32_t>(t) & send_mask) * 8u, word, is_l31);
  };
  // Anchor row of window m: s - anchor(s) of this lane's states, one store.
  uint8_t* const ztab = J.ztab;
  const int zstride = J.zstride;
  auto store_anchor_row = [&](int m) {
    if (ztab == nullptr || s0 >= zstride) return;
    uint8_t* dst = ztab + static_cast<size_t>(m) * zstride + s0;
    uint32_t packed[(K + 3) / 4];
#pragma unroll
    for (int q = 0; q < (K + 3) / 4; ++q) packed[q] = 0u;
#pragma unroll
    for (int j = 0; j < K; ++j)
      packed[j / 4] |= (static_cast<uint32_t>(s0 + j - A[j]) & 0xffu) << (8 * (j % 4));
    if constexpr (K == 2) {
      *reinterpret_cast<uint16_t*>(dst) = static_cast<uint16_t>(packed[0]);
    } else if constexpr (K == 4) {
      *reinterpret_cast<uint32_t*>(dst) = packed[0];
    } else if constexpr (K == 8) {
      *reinterpret_cast<uint2*>(dst) = make_uint2(packed[0], packed[1]);
    } else {
      *reinterpret_cast<uint4*>(dst) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
  };
  if (ckpt != nullptr && (t_begin % ck_every) == 0) store_ckpt(t_begin);
  send_one(t_begin, a[K - 1], A[K - 1]);  // slot of t_begin is fresh: no flow check needed

  // ---- frames t_begin+1 .. t_end-1 ----
  // Frames run in anchor windows of kAnchorD (an anchor row after each),
  // windows in receive blocks of B = P.block frames (one ring wait each) and
  // in emission chunks of F frames. B and F are powers of two dividing
  // kAnchorD, so a sub-run of min(B, F) frames crosses none of these
  // boundaries and the bookkeeping is incremental (no division in the loop).
  // Checkpoint frames are multiples of ck_every, itself a multiple of
  // kAnchorD, so they fall on window ends.
  int next_ck = (ckpt != nullptr) ? (t_begin / ck_every + 1) * ck_every : (1 << 30);
  const int B = P.block;
  const int R = min(B, F);
  uint32_t* bpw = bp + static_cast<size_t>(g) * bp_rows * NW;  // row 0 of this warp (unused if bp == nullptr)
  const bool write_bp = (bp != nullptr) && is_l0;
  const float* stage_f = reinterpret_cast<const float*>(stages);
  const int stage_floats = P.stage_bytes / 4;
  // Logits mode: lane i holds the shift of frame (window start + i) of the
  // current anchor window (lse_win) and of the next one (lse_next), read from
  // the pre-pass's J.lse one window ahead; a sub-run never crosses a window.
  float lse_win = 0.0f, lse_next = 0.0f;
  if constexpr (kNorm) {
    const int fa = t_begin + 1 + lane, fb = t_begin + 1 + kAnchorD + lane;
    lse_win = (fa < t_end) ? __ldg(lse_g + fa) : 0.0f;
    lse_next = (fb < t_end) ? __ldg(lse_g + fb) : 0.0f;
  }
  constexpr bool kBufBp = NW <= 6;  // K = 2, 4: a window's backpointer rows buffered in registers
  uint32_t wb[kBufBp ? NW : 1];
#pragma unroll
  for (int j = 0; j < (kBufBp ? NW : 1); ++j) wb[j] = 0u;
  int c_stage = 0;        // stage of the current chunk
  uint32_t c_round = 0;   // its round
  int ridx = 0;           // row of frame t in the stage ring (floats)
  float rv = -INFINITY;   // block receive: lane i holds the word of frame (block start - 1 + i)
  int roff = 0;
  int bi = 0;             // frame index within the current block
  int t = t_begin + 1;
  while (t < t_end) {
    const int ft = t - t_begin - 1;  // frames computed so far
    if ((ft & (F - 1)) == 0) {       // first frame of a chunk
      if (ft != 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&head->empty[c_stage]);
        if (++c_stage == P.stages) {
          c_stage = 0;
          ++c_round;
        }
        if (warp == 0 && issued < nchunks) {
          // Refill kLead - 1 chunks ahead, into the stage of chunk
          // issued - stages once every warp has released it.
          if (p_round > 0 && !warp_wait_phase(&head->empty[p_stage], (p_round - 1) & 1u, abort, limit, lane)) break;
          issue_next();
        }
      }
      if (__any_sync(kFull, *abort != 0)) break;
      if (!warp_wait_phase(&head->full[c_stage], c_round & 1u, abort, limit, lane))
        break;
      ridx = c_stage * stage_floats;
    }
    if ((ft & (B - 1)) == 0) {  // first frame of a receive block
      const int nb = min(B, t_end - t);
      // Block receive: lane i takes the word of frame t-1+i (i < nb).
      if (recv_left) {
        const int f = t - 1 + (lane < nb ? lane : 0);
        const uint64_t v = *reinterpret_cast<const volatile uint64_t*>(my_ring + (f & rb_mask));
        const bool mine = static_cast<uint32_t>(v >> 40) == ((static_cast<uint32_t>(f) + 1u) & kTagMask);
        uint64_t vv = v;
        if (!__all_sync(kFull, mine)) vv = ring_block_spin(my_ring, t - 1, nb, rb_mask, lane, abort, limit);
        rv = __uint_as_float(static_cast<uint32_t>(vv));
        roff = static_cast<int>((vv >> 32) & 0xffu);
        // Frames < t + nb - 1 are read after this block: tell the producer.
        if (is_l0) {
          if constexpr (kGrid)
            st_gpu_u32(prog_dst_g, static_cast<uint32_t>(t + nb - 1));
          else
            st_remote_u32(prog_dst, static_cast<uint32_t>(t + nb - 1));
        }
      }
      // Frame t-1 ends a window when this block starts one: its sender reset
      // its anchors after sending it.
      if (is_l0 && (ft & (kAnchorD - 1)) == 0) roff = 0;
      // Block send: slots t .. t+nb-1 reuse those of frames t-rb .. t+nb-1-rb.
      if (has_next && t + nb - 1 - P.rb >= prog_seen) {
        prog_seen = static_cast<int>(prog_spin(my_prog, t + nb - 1 - P.rb, abort, limit));
      }
      bi = 0;
    }
    const int n = min(R, t_end - t);

    // Emissions of this lane's states (blank column shared by the even states),
    // loaded one frame ahead of their use. The ring has one spare row after
    // its last stage, so the look-ahead past a chunk's end stays in bounds.
    float eb_n = stage_f[ridx + blank];
    float el_n[K / 2];
#pragma unroll
    for (int q = 0; q < K / 2; ++q) el_n[q] = stage_f[ridx + col[q]];
    // Backpointer words. NW <= 6: lane i keeps the words of the window's
    // frame i in registers and the warp stores a whole window at once (one
    // row per lane). Wider rows: lane 0 stores the words of the previous
    // frame one frame late, after this frame's loads and shuffles are issued.
    uint32_t padv[K];
    uint32_t pskp[K / 2];
#pragma unroll
    for (int j = 0; j < K; ++j) padv[j] = 0u;
#pragma unroll
    for (int j = 0; j < K / 2; ++j) pskp[j] = 0u;
    bool pend = false;
    const int fi0 = ft & (kAnchorD - 1);  // frame index of t within its window
    if constexpr (kNorm) {
      if (fi0 == 0 && ft != 0) {  // frame t starts a window: its shifts were read one window ago
        lse_win = lse_next;
        const int fn = t + kAnchorD + lane;
        lse_next = (fn < t_end) ? __ldg(lse_g + fn) : 0.0f;
      }
    }
#pragma unroll(K == 2 ? 4 : 1)
    for (int i = 0; i < n; ++i, ++t) {
      float eb = eb_n;
      float el[K / 2];
#pragma unroll
      for (int q = 0; q < K / 2; ++q) el[q] = el_n[q];
      if constexpr (kNorm) {  // log-probability = logit - the frame's shift
        const float sh = __shfl_sync(kFull, lse_win, fi0 + i);
        eb -= sh;
#pragma unroll
        for (int q = 0; q < K / 2; ++q) el[q] -= sh;
      }
      ridx += C;
      eb_n = stage_f[ridx + blank];
#pragma unroll
      for (int q = 0; q < K / 2; ++q) el_n[q] = stage_f[ridx + col[q]];

      // alpha_{t-1}(s0 - 1) and its anchor: lane below by shuffle, lane 0 from the block.
      const float shf = __shfl_up_sync(kFull, a[K - 1], 1);
      const float blk = __shfl_sync(kFull, rv, bi + i);
      const float left = is_l0 ? blk : shf;
      if constexpr (kSum) {  // sum-product: log-add of the allowed predecessors
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {  // descending: a[j-1], a[j-2] still hold frame t-1
          const float p1 = (j == 0) ? left : a[j - 1];
          if ((j & 1) == 0) {
            a[j] = log2_add2(a[j], p1) + eb * kLog2e;
          } else {
            const float p2raw = (j == 1) ? left : a[j - 2];
            const float p2 = __uint_as_float((__float_as_uint(p2raw) & skeep[j >> 1]) | sfill[j >> 1]);
            a[j] = log2_add3(a[j], p1, p2) + el[j >> 1] * kLog2e;
          }
        }
        send_one(t, a[K - 1], s_last);
        continue;
      }
      const int shA = __shfl_up_sync(kFull, A[K - 1], 1);
      const int blko = __shfl_sync(kFull, roff, bi + i);
      const int Aleft = is_l0 ? (s0 - 1 - blko) : shA;
      if constexpr (!kBufBp) store_bp_words_if<K>(bpw - NW, padv, pskp, write_bp && pend);

      uint32_t adv[K];
      uint32_t skp[K / 2];
#pragma unroll
      for (int j = K - 1; j >= 0; --j) {  // descending: a[j-1], a[j-2] still hold frame t-1
        const float p1 = (j == 0) ? left : a[j - 1];
        const int q1 = (j == 0) ? Aleft : A[j - 1];
        if ((j & 1) == 0) {  // blank state: stay or advance
          const bool b1 = p1 > a[j];
          const float m = b1 ? p1 : a[j];
          A[j] = b1 ? q1 : A[j];
          adv[j] = __ballot_sync(kFull, b1);
          a[j] = m + eb;
        } else {  // label state: stay, advance, or skip when allowed
          const float p2raw = (j == 1) ? left : a[j - 2];
          const float p2 = (K <= 4) ? p2raw
                                    : __uint_as_float((__float_as_uint(p2raw) & skeep[j >> 1]) | sfill[j >> 1]);
          const int q2 = (j == 1) ? Aleft : A[j - 2];
          const bool b1 = p1 > a[j];
          float m = b1 ? p1 : a[j];
          int an = b1 ? q1 : A[j];
          const bool b2 = ((K <= 4) ? skok[j >> 1] : true) && (p2 > m);
          m = b2 ? p2 : m;
          A[j] = b2 ? q2 : an;
          adv[j] = __ballot_sync(kFull, b1);
          skp[j >> 1] = __ballot_sync(kFull, b2);
          a[j] = m + el[j >> 1];
        }
      }
      if constexpr (kBufBp) {
        const bool mine = (lane == fi0 + i);
#pragma unroll
        for (int j = 0; j < K; ++j) wb[j] = mine ? adv[j] : wb[j];
#pragma unroll
        for (int j = 0; j < K / 2; ++j) wb[K + j] = mine ? skp[j] : wb[K + j];
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) padv[j] = adv[j];
#pragma unroll
        for (int j = 0; j < K / 2; ++j) pskp[j] = skp[j];
        pend = true;
        bpw += NW;
      }
      send_one(t, a[K - 1], A[K - 1]);
    }
    if constexpr (!kBufBp) store_bp_words_if<K>(bpw - NW, padv, pskp, write_bp && pend);
    bi += n;
    const int done = t - 1 - t_begin;  // frames computed after this sub-run
    if constexpr (kBufBp) {
      if (((done & (kAnchorD - 1)) == 0 || t == t_end) && bp != nullptr) {
        // Rows row0 .. done-1 of this window: row r holds frame t_begin + 1 + r.
        const int row0 = (done - 1) & ~(kAnchorD - 1);
        if (lane < done - row0) store_bp_row<K>(bp + (static_cast<size_t>(g) * bp_rows + row0 + lane) * NW, wb);
      }
    }
    if ((done & (kAnchorD - 1)) == 0) {  // window end: frame t-1 is an anchor frame
      if (t - 1 == next_ck) {
        store_ckpt(next_ck);
        next_ck += ck_every;
      }
      store_anchor_row(done / kAnchorD - 1);
#pragma unroll
      for (int j = 0; j < K; ++j) A[j] = s0 + j;
    }
  }
  // Last, partial window.
  const int nwin = (t_end - 1 - t_begin + kAnchorD - 1) / kAnchorD;  // anchor rows of this pass
  if (*abort == 0 && t_end - 1 > t_begin && ((t_end - 1 - t_begin) % kAnchorD) != 0)
    store_anchor_row(nwin - 1);

  // ---- alpha_{T-1} of the two final states ----
  const bool aborted_here = (*abort != 0);
  if (!aborted_here && t_end == J.T && J.final2 != nullptr) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (s0 + j == S - 1) J.final2[1] = a[j];
      if (s0 + j == S - 2) J.final2[0] = a[j];
    }
  }

  // ---- drain: no copy may still target this CTA's shared memory ----
  // Each stage has at most one chunk in flight; waiting for the latest chunk
  // issued on every stage covers all of them (a completed phase returns at once).
  if (warp == 0 && lane == 0) {
    for (int c = max(0, issued - P.stages); c < issued; ++c)
      (void)wait_phase(&head->full[c % P.stages], (c / P.stages) & 1, abort, limit, false);
  }
  // All backpointers / anchor rows / final values written. A CTA whose wait
  // ran out marks the request timed out before the team barrier; after it
  // every CTA of the team reads the same status and leaves together.
  if (!team_sync_ok()) return;

  // ---- tail 1 (warp 0 of CTA 0): final state, total, hops back through the anchor rows ----
  // Boundary states go to path[t_begin + m*D] (m < nwin) and path[t_end - 1];
  // the window walks below read them before overwriting path with tokens.
  const bool chase = (J.flags & kJobChase) != 0;
  unsigned char* tail = smem + P.off_ring;  // the rings and stages are free now (hop buffer)
  if (crank == 0 && warp == 0) {
    int s_cur;
    if (J.flags & kJobWriteFinal) {
      const float f_blank = __ldcg(J.final2 + 1);
      const float f_lab = (S > 1) ? __ldcg(J.final2 + 0) : -INFINITY;
      s_cur = (S > 1 && f_lab > f_blank) ? S - 2 : S - 1;
      const float tot = kSum ? log2_add2(f_lab, f_blank) * kLn2 : ((S > 1 && f_lab > f_blank) ? f_lab : f_blank);
      if (lane == 0) {
        if (J.total) *J.total = tot;
        atomicCAS(J.status, kStPending, tot == -INFINITY ? kStNoPath : kStOk);
        if (!chase) *J.state_io = s_cur;
      }
    } else {
      s_cur = __ldcg(J.state_io);
    }
    if (chase) {
      if (lane == 0) path[t_end - 1] = s_cur;
      // Batches of kHopBatch rows: lane q copies bytes [lo + 16c, lo + 16c + 16)
      // for c = q, q + 32, ... of every row into shared memory (asynchronous copies, one wait), the
      // range [s - kHopSpan, s] around the current state; then lane 0 hops.
      // A path moves at most 64 states per window but far fewer in practice;
      // a hop below the staged range reads its byte from global memory.
      uint8_t* zb = tail;  // [kHopBatch][kHopRowBytes]
      for (int m = nwin - 1; m >= 0; m -= kHopBatch) {
        const int nb = min(kHopBatch, m + 1);
        const int lo = max(0, s_cur - kHopSpan) & ~15;
        const int hi = min(zstride, (s_cur + 16) & ~15);  // exclusive, 16-aligned
        const int nchunk = (hi - lo) / 16;                // <= kHopRowBytes / 16
        for (int c = lane; c < nchunk; c += 32) {  // lane c copies bytes [lo + 16c, lo + 16c + 16) of each row
          for (int r = 0; r < nb; ++r)
            cp_async16(zb + r * kHopRowBytes + c * 16, ztab + static_cast<size_t>(m - r) * zstride + lo + c * 16);
        }
        cp_async_wait_all();
        __syncwarp();
        if (lane == 0) {
          for (int r = 0; r < nb; ++r) {
            const int off = s_cur - lo;
            const int d = (off >= 0) ? static_cast<int>(zb[r * kHopRowBytes + off])
                                     : static_cast<int>(__ldcg(ztab + static_cast<size_t>(m - r) * zstride + s_cur));
            s_cur -= d;
            path[t_begin + (m - r) * kAnchorD] = s_cur;
          }
        }
        s_cur = __shfl_sync(kFull, s_cur, 0);
        __syncwarp();
      }
      if (lane == 0) *J.state_io = s_cur;  // state at t_begin
    }
  }
  if (!chase) return;
  if (!team_sync_ok()) return;  // boundary states visible to every warp of the team

  // ---- tail 2 (every lane of the team): walk the windows in parallel ----
  // Window m covers frames (t_begin + m*D, e] with e = min(t_begin + (m+1)*D,
  // t_end - 1); its top state is path[e]. One lane walks one window and stores
  // the state of every frame into path[] (window 0 also frame t_begin); lanes
  // of a warp walk 32 windows at once. The backpointer words are read with
  // plain (L1-cached) loads: they were written before the team barrier, whose
  // acquire makes them visible, and consecutive frames of a warp group share
  // cache lines.
  const int G = static_cast<int>(ncta) * W;
  const int nwalk = max(nwin, 1);
  for (int m = g * 32 + lane; m < nwalk; m += G * 32) {
    const int b = t_begin + m * kAnchorD;
    const int e = (nwin == 0) ? t_begin : min(b + kAnchorD, t_end - 1);
    int sc = path[e];
    for (int f = e; f > b; --f) {
      path[f] = sc;
      const int gs = sc / GS;
      const int r = sc % GS;
      const int ln = r / K;
      const int j = r % K;
      const uint32_t* wd = bp + (static_cast<size_t>(gs) * bp_rows + (f - t_begin - 1)) * NW;
      const uint32_t av = (wd[j] >> ln) & 1u;
      const uint32_t sk = (wd[K + (j >> 1)] >> ln) & static_cast<uint32_t>(j) & 1u;
      sc -= sk ? 2 : static_cast<int>(av);
    }
    if (m == 0) path[b] = sc;
  }
  if (!team_sync_ok()) return;  // every frame's state is in path[]

  // ---- tail 3 (every thread of the team): states -> tokens, states, scores ----
  // Each thread takes kT3 frames per round, loading all their states, then
  // all their tokens, then all their emission values: three memory round
  // trips per round instead of three per frame.
  {
    constexpr int kT3 = 8;
    const int tid = g * 32 + lane;
    const int nthr = G * 32;
    for (int f0 = t_begin + tid; f0 < t_end; f0 += kT3 * nthr) {
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
        if constexpr (kNorm)
          sv[k] = (f < t_end) ? __ldg(lp + static_cast<size_t>(f) * C + tok[k]) - lse_g[f] : 0.0f;
        else
          sv[k] = (f < t_end) ? __ldg(lp + static_cast<size_t>(f) * C + tok[k]) : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < kT3; ++k) {
        const int f = f0 + k * nthr;
        if (f < t_end) {
          path[f] = tok[k];
          if (states_out) states_out[f] = st[k];
          scores_out[f] = sv[k];
        }
      }
    }
  }
}

// ------------------------------------------------------- frame-latency probe --
// Per-frame synchronisation bound of the roofline: the irreducible dependent
// chain of one frame of the recursion at warp scope, with null work around it.
// Every lane holds one state; per frame it reads its emission from shared
// memory, takes its left neighbour's previous value by shuffle, and does one
// max and one add. Between warps and CTAs the trellis kernel exchanges values
// once per block of frames, which adds pipeline fill but no per-frame cost, so
// this chain bounds the time per frame of any team shape. Warp 0 of CTA 0
// measures the time per frame with %globaltimer; other warps run the same loop.
__global__ void __launch_bounds__(1024) frame_probe_kernel(int frames, uint64_t limit_ns, uint64_t* out) {
  __shared__ float rows[64 * 32];
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) rows[i] = -0.001f * static_cast<float>(i % 97);
  __syncthreads();
  float a = (lane == 0) ? 0.0f : -INFINITY;
  const uint64_t t0 = gtimer();
  for (int t = 0; t < frames; ++t) {
    const float e = rows[(t & 63) * 32 + lane];
    const float left = __shfl_up_sync(kFull, a, 1);
    a = fmaxf(a, lane == 0 ? -INFINITY : left) + e;
  }
  const uint64_t t1 = gtimer();
  (void)limit_ns;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = t1 - t0;
    out[1] = 0ull;
    out[2] = __float_as_uint(a);
  }
}

// Logits mode: lse[t] = log(sum_c exp(logits[t][c])) of every frame of every
// job, one warp per frame (the maximum factored out, fast exponential,
// accurate logarithm), before the trellis launch reads them.
__global__ void __launch_bounds__(256) lse_prepass_kernel(const FwdJob* __restrict__ jobs) {
  const FwdJob& J = jobs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int C = J.C;
  const int64_t step = static_cast<int64_t>(gridDim.x) * 8;
  for (int64_t t = J.t_begin + static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); t < J.t_end; t += step) {
    const float* row = J.lp + t * C;
    float m = -INFINITY;
    for (int c = lane; c < C; c += 32) m = fmaxf(m, __ldg(row + c));
    for (int k = 16; k > 0; k >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, k));
    float sum = 0.0f;
    for (int c = lane; c < C; c += 32) sum += __expf(__ldg(row + c) - m);
    for (int k = 16; k > 0; k >>= 1) sum += __shfl_xor_sync(kFull, sum, k);
    if (lane == 0) J.lse[t] = m + logf(sum);
  }
}

template <int K, bool kOcc, bool kGrid, bool kNorm, bool kSum = false>
cudaError_t launch_k(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                     cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int smem_max = max_smem_optin(dev);
  int smem = smem_bytes(shape, p);
  if (kGrid) {
    // One CTA per SM: all of the opt-in shared memory, so that no other CTA
    // shares the SM and the cooperative launch can place the whole team.
    smem = std::max(smem, smem_max);
    if (njobs != 1) return cudaErrorInvalidValue;  // one team per cooperative launch
  }
  auto fn = trellis_kernel<K, kOcc, kGrid, kNorm, kSum>;
  if constexpr (kNorm) {  // the per-frame shifts first, on the same stream
    lse_prepass_kernel<<<dim3(128, static_cast<unsigned>(njobs), 1), 256, 0, stream>>>(d_jobs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // The allowed maximum is always the device's opt-in limit, never the size
  // of the launch at hand: launches of one kernel captured into a graph ask
  // for different sizes, and none may see a limit lowered by another.
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  if (smem > smem_max) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(njobs * shape.ncta), 1, 1);
  cfg.blockDim = dim3(static_cast<unsigned>(shape.warps * 32), 1, 1);
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

// The instantiation of a launch shape: latency or occupancy build (K <= 4),
// cluster or grid team, log-probabilities or logits.
template <int K>
cudaError_t launch_shape(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                         cudaStream_t s) {
  if (shape.sum) {
    if (shape.norm) return cudaErrorInvalidValue;  // not built: sum-product takes log-probabilities
    if (shape.grid) return launch_k<K, false, true, false, true>(shape, p, d_jobs, njobs, s);
    return launch_k<K, false, false, false, true>(shape, p, d_jobs, njobs, s);
  }
  if (shape.norm) {
    if (shape.grid) return launch_k<K, false, true, true>(shape, p, d_jobs, njobs, s);
    return launch_k<K, false, false, true>(shape, p, d_jobs, njobs, s);
  }
  if (shape.grid) return launch_k<K, false, true, false>(shape, p, d_jobs, njobs, s);
  if (K <= 4 && shape.occ) return launch_k<K, (K <= 4), false, false>(shape, p, d_jobs, njobs, s);
  return launch_k<K, false, false, false>(shape, p, d_jobs, njobs, s);
}

}  // namespace

FwdParams plan_params(const LaunchShape& shape, int C, int frames_per_stage, uint64_t wait_limit_ns) {
  FwdParams p{};
  const int F = frames_per_stage < 1 ? 1 : frames_per_stage;
  p.grid_ctas = shape.grid ? shape.ncta : 0;
  p.norm = shape.norm ? 1 : 0;
  p.frames_per_stage = F;
  p.stage_bytes = ((F * C * 4) + 15) & ~15;
  p.wait_limit_ns = wait_limit_ns;
  if (shape.fast) {
    // Fast kernel: per-warp links after the head (16-byte counters + package
    // slots), then the emission stages. Warps of a CTA lag each other by about
    // two packages per hop; the stage ring is sized to that lag.
    // Whole 32-frame windows per hand-off when a stage holds a window's rows
    // (C <= 64), else packages of 4 frames.
    p.kb = (F == kAnchorD) ? kAnchorD : 4;
    p.pkgs = (p.kb == kAnchorD) ? kFastWinPkgs : kFastPkgs;
    p.gpkgs = (p.kb == kAnchorD) ? kFastWinGridPkgs : kFastGridPkgs;
    p.link_off = static_cast<int>(sizeof(SmemHead));
    p.link_stride = 16 + p.pkgs * p.kb * 8;
    p.row_c = (p.kb == kAnchorD && C == 32) ? 32 : 0;
    const int hops = std::max(0, shape.warps - 1);
    // Throughput-planned batches with wide rows (packages of 4 frames, stages
    // of 8 KB) keep two stages ahead of the first warp instead of kLead, so
    // that three CTAs of four warps share an SM instead of two.
    const int lead = (p.kb == 4 && shape.occ) ? 2 : kLead;
    p.stages = std::min(kMaxStages, std::max(kLead, lead + (hops * 2 * p.kb + F - 1) / F));
    p.block = p.kb;
    p.rb = 0;
    p.off_ring = p.link_off;  // the backtrack's hop buffer reuses links and stages
    p.off_stage = (p.link_off + shape.warps * p.link_stride + 127) & ~127;
    p.off_lse = p.off_stage + p.stages * p.stage_bytes;
    p.off_bt = (p.off_lse + 127) & ~127;
    return p;
  }
  // Block of frames per ring wait: the warps of a CTA lag each other by up to
  // one block per hop, and the emission ring tolerates (stages - kLead) * F
  // frames of lag between its first and last warp before the producer (warp 0)
  // waits for a stage to be released. Stages beyond that only cost shared
  // memory, i.e. resident CTAs per SM, so the ring is sized to the lag: kLead
  // stages for a one-warp CTA (warp 0 releases a stage itself just before it
  // refills it), up to kMaxStages for wide CTAs.
  // The block is a power of two dividing kAnchorD (as F is).
  const int lag_room = (kMaxStages - kLead) * F;
  const int hops = std::max(0, shape.warps - 1);
  const int room = std::max(1, std::min(kAnchorD, lag_room / std::max(1, hops)));
  p.block = 1;
  while (p.block * 2 <= room) p.block *= 2;
  p.stages = kLead + (hops * p.block + F - 1) / F;
  int rb = 8;
  while (rb < 2 * p.block + 2) rb <<= 1;
  p.rb = rb;
  p.off_ring = static_cast<int>(sizeof(SmemHead)) + 32 * 4;
  p.off_stage = (p.off_ring + shape.warps * rb * 8 + 127) & ~127;
  // One spare row after the last stage: the emission look-ahead of a chunk's
  // last frame reads (and discards) the row after it.
  p.off_lse = (p.off_stage + p.stages * p.stage_bytes + C * 4 + 15) & ~15;
  p.off_bt = (p.off_lse + 127) & ~127;  // end of the forward region
  return p;
}

int smem_bytes(const LaunchShape& shape, const FwdParams& p) {
  // The backtrack reuses the ring / stage region for the hop buffer of
  // kHopBatch anchor-row slices.
  (void)shape;
  return std::max(p.off_bt, p.off_ring + kHopBatch * kHopRowBytes);
}

int launch_trellis(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                   void* stream) {
  if (njobs <= 0) return cudaSuccess;
  if (shape.fast) return launch_trellis_fast(shape, p, d_jobs, njobs, stream);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (shape.K) {
    case 2: return launch_shape<2>(shape, p, d_jobs, njobs, s);
    case 4: return launch_shape<4>(shape, p, d_jobs, njobs, s);
    case 8: return launch_shape<8>(shape, p, d_jobs, njobs, s);
    case 16: return launch_shape<16>(shape, p, d_jobs, njobs, s);
    default: return cudaErrorInvalidValue;
  }
}

int launch_frame_probe(int warps, int ncta, int frames, uint64_t limit_ns, uint64_t* d_out, void* stream) {
  frame_probe_kernel<<<ncta, warps * 32, 0, static_cast<cudaStream_t>(stream)>>>(frames, limit_ns, d_out);
  return cudaGetLastError();
}

int max_smem_optin(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return v;
}

}  // namespace gb300_align
