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

#include <cmath>
#include <cstdint>

#include "trellis.cuh"

namespace gb300_align {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_remote_u64(uint32_t addr, uint64_t v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void st_remote_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// ------------------------------------------------------- shared-memory head --
struct SmemHead {
  uint64_t full[kStages];   // emission stage filled
  uint64_t empty[kStages];  // emission stage released by every warp
  int32_t abort;            // set by any thread of this CTA whose wait hit the limit
  uint32_t prog;            // boundary frames consumed by the next CTA of the cluster (remote writes)
  int32_t pad[14];
};
static_assert(sizeof(SmemHead) == 128, "head size");

// Bounded wait on an mbarrier phase, done by one lane. Returns false on
// timeout (and raises the CTA abort flag) or when another warp aborted.
__device__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int32_t* abort, uint64_t limit,
                           bool honour_abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (honour_abort && *abort) return false;
    if (gtimer() - t0 > limit) {
      *abort = 1;
      return false;
    }
  }
}

// Warp-uniform bounded wait: lane 0 spins, every lane then observes the
// completed phase itself (acquire) before reading the staged data.
__device__ __forceinline__ bool warp_wait_phase(uint64_t* bar, uint32_t parity, volatile int32_t* abort,
                                                uint64_t limit, int lane) {
  int ok = 1;
  if (lane == 0) ok = wait_phase(bar, parity, abort, limit, true);
  ok = __shfl_sync(kFull, ok, 0);
  if (ok) (void)mbar_try_wait(bar, parity);
  return ok != 0;
}

// Receive alpha_{t}(first state - 1) of this warp from its left neighbour's
// tagged ring slot (tag = frame + 1, value = FP32 bits). One lane.
__device__ __forceinline__ float ring_recv(const uint64_t* ring, int t, int rb_mask, volatile int32_t* abort,
                                           uint64_t limit, bool& ok) {
  const volatile uint64_t* p = ring + (t & rb_mask);
  const uint32_t want = static_cast<uint32_t>(t + 1);
  uint64_t v = *p;
  if (static_cast<uint32_t>(v >> 32) != want) {
    const uint64_t t0 = gtimer();
    for (;;) {
      v = *p;
      if (static_cast<uint32_t>(v >> 32) == want) break;
      if (*abort || gtimer() - t0 > limit) {
        *abort = 1;
        ok = false;
        return -INFINITY;
      }
    }
  }
  return __uint_as_float(static_cast<uint32_t>(v));
}

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

// ------------------------------------------------------------------ kernel --
template <int K>
__global__ void __launch_bounds__(K <= 8 ? 1024 : 512)
    trellis_kernel(const FwdJob* __restrict__ jobs, const FwdParams P) {
  static_assert(K % 2 == 0 && K >= 2 && K <= 16, "K must be even, 2..16");
  constexpr int NW = bp_words(K);
  extern __shared__ __align__(128) unsigned char smem[];
  SmemHead* head = reinterpret_cast<SmemHead*>(smem);
  uint64_t* ring = reinterpret_cast<uint64_t*>(smem + P.off_ring);
  unsigned char* stages = smem + P.off_stage;
  volatile int32_t* abort = &head->abort;

  const uint32_t ncta = cluster_nctarank();
  const uint32_t crank = cluster_ctarank();
  const int W = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const FwdJob& J = jobs[blockIdx.x / ncta];
  const int g = static_cast<int>(crank) * W + warp;   // warp index in the team
  const int S = J.S, C = J.C, blank = J.blank;
  const int t_begin = J.t_begin, t_end = J.t_end;
  const int s0 = (g * 32 + lane) * K;               // first state of this lane
  const int F = P.frames_per_stage;
  const int rb_mask = P.rb - 1;
  const int nchunks = (t_end - t_begin + F - 1) / F;
  const bool bulk = (J.flags & kJobBulkRows) != 0;
  const uint64_t limit = P.wait_limit_ns;
  const float* __restrict__ lp = J.lp;
  uint32_t* __restrict__ bp = J.bp;
  const int bp_rows = J.bp_rows;
  float* __restrict__ ckpt = J.ckpt;
  const int ck_every = J.ck_every;
  const int ck_stride = J.ck_stride;

  // ---- shared state: rings zeroed, barriers initialised ----
  for (int i = threadIdx.x; i < W * P.rb; i += blockDim.x) ring[i] = 0ull;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&head->full[st], bulk ? 1u : 32u);
      mbar_init(&head->empty[st], static_cast<uint32_t>(W));
    }
    head->abort = 0;
    head->prog = static_cast<uint32_t>(t_begin);  // no slot holds a frame before t_begin
    fence_barrier_init();
  }
  __syncthreads();
  if (ncta > 1) cluster_sync();  // neighbours' rings exist and are zero before any remote store

  // ---- per-lane constants: label columns and skip caps of the label states ----
  int col[K / 2];
  float cap[K / 2];
#pragma unroll
  for (int i = 0; i < K / 2; ++i) {
    const int s = s0 + 2 * i + 1;
    int lab = 0;
    bool skip = false;
    if (s < S) {
      lab = J.tgt[(s - 1) >> 1];
      skip = (s >= 3) && (lab != J.tgt[(s - 3) >> 1]);
    }
    col[i] = lab;
    cap[i] = skip ? INFINITY : -INFINITY;  // min(alpha(s-2), cap) masks a forbidden skip to -inf
  }

  // ---- emission staging (warp 0 of each CTA is the producer) ----
  int issued = 0;
  auto issue_chunk = [&](int c) {
    const int st = c % kStages;
    const int f0 = t_begin + c * F;
    const int nf = min(F, t_end - f0);
    const float* src = lp + static_cast<size_t>(f0) * C;
    float* dst = reinterpret_cast<float*>(stages + st * P.stage_bytes);
    if (bulk) {
      if (lane == 0) {
        const uint32_t bytes = static_cast<uint32_t>(nf * C * 4);
        mbar_arrive_expect_tx(&head->full[st], bytes);
        bulk_g2s(dst, src, bytes, &head->full[st]);
      }
    } else {
      const int n = nf * C;
      for (int i = lane; i < n; i += 32) cp_async4(dst + i, src + i);
      cp_async_mbar_arrive(&head->full[st]);
    }
  };
  if (warp == 0) {
    for (int c = 0; c < min(kStages - 1, nchunks); ++c) issue_chunk(c);
    issued = min(kStages - 1, nchunks);
  }

  // ---- frame t_begin: initialisation ----
  float a[K];
  int chunk = 0;
  bool ok = warp_wait_phase(&head->full[0], 0, abort, limit, lane);
  const float* row = reinterpret_cast<const float*>(stages);
  if (ok) {
    if (J.alpha_in == nullptr) {
      const float eb = row[blank];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int s = s0 + j;
        a[j] = (s == 0) ? eb : ((s == 1 && S > 1) ? row[col[0]] : -INFINITY);
      }
    } else {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int s = s0 + j;
        a[j] = (s < S) ? __ldg(J.alpha_in + s) : -INFINITY;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) a[j] = -INFINITY;
  }

  const bool recv_left = (g > 0);
  const bool send_local = warp < W - 1;
  const bool send_remote = (warp == W - 1) && (crank + 1 < ncta);
  const uint64_t* my_ring = ring + warp * P.rb;
  uint64_t* next_ring = ring + (warp + 1) * P.rb;
  const uint32_t remote_ring = send_remote ? mapa_rank(smem_addr(ring), crank + 1) : 0u;
  const bool publish_prog = (warp == 0 && crank > 0);
  const uint32_t remote_prog = publish_prog ? mapa_rank(smem_addr(&head->prog), crank - 1) : 0u;
  uint32_t cached_prog = static_cast<uint32_t>(t_begin);

  auto send = [&](int t, float v) {  // lane 31 only
    const uint64_t word = (static_cast<uint64_t>(static_cast<uint32_t>(t + 1)) << 32) | __float_as_uint(v);
    if (send_local) {
      *reinterpret_cast<volatile uint64_t*>(next_ring + (t & rb_mask)) = word;
    } else if (send_remote) {
      // The next CTA must have consumed frame t - rb before its slot is reused.
      if (t - P.rb >= static_cast<int>(cached_prog)) {
        const uint64_t t0 = gtimer();
        for (;;) {
          cached_prog = *reinterpret_cast<volatile uint32_t*>(&head->prog);
          if (t - P.rb < static_cast<int>(cached_prog)) break;
          if (*abort || gtimer() - t0 > limit) {
            *abort = 1;
            return;
          }
        }
      }
      st_remote_u64(remote_ring + static_cast<uint32_t>(t & rb_mask) * 8u, word);
    }
  };
  auto store_ckpt = [&](int t) {
    if (ckpt != nullptr && (t % ck_every) == 0) {
      float* dst = ckpt + static_cast<size_t>(t / ck_every) * ck_stride;
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (s0 + j < S) dst[s0 + j] = a[j];
    }
  };
  if (ok) {
    store_ckpt(t_begin);
    if (lane == 31) send(t_begin, a[K - 1]);
  }

  // ---- frames t_begin+1 .. t_end-1 ----
  for (int t = t_begin + 1; t < t_end; ++t) {
    const int ft = t - t_begin;
    if (ft % F == 0) {  // entering the next stage of emission rows
      __syncwarp();
      if (lane == 0) mbar_arrive(&head->empty[chunk % kStages]);
      ++chunk;
      if (__any_sync(kFull, *abort != 0)) break;
      if (warp == 0 && chunk + 2 < nchunks) {
        // Refill the stage that held chunk - 2 once every warp has released it.
        const int old = chunk - 2;
        bool free_ok = true;
        if (old >= 0)
          free_ok = warp_wait_phase(&head->empty[old % kStages], (old / kStages) & 1, abort, limit, lane);
        if (!free_ok) break;
        issue_chunk(chunk + 2);
        issued = chunk + 3;
      }
      if (!warp_wait_phase(&head->full[chunk % kStages], (chunk / kStages) & 1, abort, limit, lane)) break;
      if (lane == 0 && publish_prog) st_remote_u32(remote_prog, static_cast<uint32_t>(t - 1));
      row = reinterpret_cast<const float*>(stages + (chunk % kStages) * P.stage_bytes);
    } else {
      row += C;
    }

    // Emissions of this lane's states (blank column shared by the even states).
    const float eb = row[blank];
    float el[K / 2];
#pragma unroll
    for (int i = 0; i < K / 2; ++i) el[i] = row[col[i]];

    // alpha_{t-1}(s0 - 1): from the lane below, or from the previous warp's ring.
    float left = __shfl_up_sync(kFull, a[K - 1], 1);
    if (lane == 0) {
      if (recv_left) {
        bool rok = true;
        left = ring_recv(my_ring, t - 1, rb_mask, abort, limit, rok);
      } else {
        left = -INFINITY;
      }
    }

    uint32_t adv[K];
    uint32_t skp[K / 2];
#pragma unroll
    for (int j = K - 1; j >= 0; --j) {  // descending: a[j-1], a[j-2] still hold frame t-1
      const float p1 = (j == 0) ? left : a[j - 1];
      if ((j & 1) == 0) {  // blank state: stay or advance
        const bool b1 = p1 > a[j];
        const float m = b1 ? p1 : a[j];
        adv[j] = __ballot_sync(kFull, b1);
        a[j] = m + eb;
      } else {  // label state: stay, advance, or skip when allowed
        const float p2 = fminf((j == 1) ? left : a[j - 2], cap[j >> 1]);
        const bool b1 = p1 > a[j];
        float m = b1 ? p1 : a[j];
        const bool b2 = p2 > m;
        m = b2 ? p2 : m;
        adv[j] = __ballot_sync(kFull, b1);
        skp[j >> 1] = __ballot_sync(kFull, b2);
        a[j] = m + el[j >> 1];
      }
    }
    if (bp != nullptr && lane == 0)
      store_bp_words<K>(bp + (static_cast<size_t>(g) * bp_rows + (ft - 1)) * NW, adv, skp);
    if (lane == 31) send(t, a[K - 1]);
    store_ckpt(t);
  }

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
    for (int c = max(0, issued - kStages); c < issued; ++c)
      (void)wait_phase(&head->full[c % kStages], (c / kStages) & 1, abort, limit, false);
  }
  __threadfence();
  __syncthreads();
  if (ncta > 1) cluster_sync();  // all backpointers / final values written; no remote access follows
  const bool aborted = (*abort != 0);
  if (aborted && threadIdx.x == 0) atomicExch(J.status, kStTimeout);

  // ---- tail: final state, total, and the backtrack (warp 0 of CTA 0) ----
  if (crank != 0 || warp != 0 || aborted) return;
  int s_cur;
  if (J.flags & kJobWriteFinal) {
    const float f_blank = __ldcg(J.final2 + 1);
    const float f_lab = (S > 1) ? __ldcg(J.final2 + 0) : -INFINITY;
    s_cur = (S > 1 && f_lab > f_blank) ? S - 2 : S - 1;
    const float tot = (S > 1 && f_lab > f_blank) ? f_lab : f_blank;
    if (lane == 0) {
      if (J.total) *J.total = tot;
      atomicCAS(J.status, kStPending, tot == -INFINITY ? kStNoPath : kStOk);
      if (!(J.flags & kJobChase)) *J.state_io = s_cur;
    }
  } else {
    s_cur = __ldcg(J.state_io);
  }
  if (!(J.flags & kJobChase)) return;

  // Windowed walk back: per window of 32 frames the states stay within
  // [s - 62, s], i.e. inside at most two warp groups of 32K >= 64 states.
  // Lanes fetch those backpointer words for one frame each, then lane 0
  // follows the codes in shared memory and all lanes write the outputs.
  constexpr int GS = 32 * K;
  uint32_t* wbuf = reinterpret_cast<uint32_t*>(smem + P.off_bt);          // [32][2][NW]
  int32_t* sbuf = reinterpret_cast<int32_t*>(smem + P.off_bt + kBtWindow * 2 * NW * 4);  // [32]
  const int t_lo = t_begin;
  for (int top = t_end - 1; top >= t_lo; top -= kBtWindow) {
    const int n = min(kBtWindow, top - t_lo + 1);
    const int g_hi = s_cur / GS;
    const int g_lo = max(0, s_cur - 2 * (n - 1)) / GS;
    if (lane < n) {
      const int f = top - lane;
      if (f > t_lo) {
        for (int gi = 0; gi <= g_hi - g_lo; ++gi) {
          const uint32_t* src = bp + (static_cast<size_t>(g_lo + gi) * bp_rows + (f - t_begin - 1)) * NW;
          uint32_t* dst = wbuf + (lane * 2 + gi) * NW;
#pragma unroll
          for (int w = 0; w < NW; ++w) dst[w] = __ldcg(src + w);
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      for (int i = 0; i < n; ++i) {
        const int f = top - i;
        sbuf[i] = s_cur;
        if (f > t_lo) {
          const int gi = s_cur / GS - g_lo;
          const int r = s_cur % GS;
          const int ln = r / K;
          const int j = r % K;
          const uint32_t* wd = wbuf + (i * 2 + gi) * NW;
          const uint32_t av = (wd[j] >> ln) & 1u;
          const uint32_t sk = (j & 1) ? ((wd[K + (j >> 1)] >> ln) & 1u) : 0u;
          s_cur -= sk ? 2 : static_cast<int>(av);
        }
      }
    }
    __syncwarp();
    s_cur = __shfl_sync(kFull, s_cur, 0);
    if (lane < n) {
      const int f = top - lane;
      const int st = sbuf[lane];
      const int tok = (st & 1) ? J.tgt[st >> 1] : blank;
      J.path[f] = tok;
      J.scores[f] = __ldg(lp + static_cast<size_t>(f) * C + tok);
      if (J.states) J.states[f] = st;
    }
    __syncwarp();
  }
  if (lane == 0) *J.state_io = s_cur;
}

template <int K>
cudaError_t launch_k(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                     cudaStream_t stream) {
  const int smem = smem_bytes(shape, p);
  auto fn = trellis_kernel<K>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(njobs * shape.ncta), 1, 1);
  cfg.blockDim = dim3(static_cast<unsigned>(shape.warps * 32), 1, 1);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  if (shape.ncta > 1) {
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

}  // namespace

FwdParams plan_params(const LaunchShape& shape, int C, int frames_per_stage, uint64_t wait_limit_ns) {
  FwdParams p{};
  const int F = frames_per_stage < 1 ? 1 : frames_per_stage;
  int rb = 8;
  while (rb < 4 * F + 2) rb <<= 1;
  p.rb = rb;
  p.frames_per_stage = F;
  p.stage_bytes = ((F * C * 4) + 15) & ~15;
  p.off_ring = static_cast<int>(sizeof(SmemHead));
  p.off_stage = (p.off_ring + shape.warps * rb * 8 + 127) & ~127;
  p.off_bt = (p.off_stage + kStages * p.stage_bytes + 127) & ~127;
  p.wait_limit_ns = wait_limit_ns;
  return p;
}

int smem_bytes(const LaunchShape& shape, const FwdParams& p) {
  return p.off_bt + kBtWindow * 2 * bp_words(shape.K) * 4 + kBtWindow * 4;
}

int launch_trellis(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                   void* stream) {
  if (njobs <= 0) return cudaSuccess;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (shape.K) {
    case 2: return launch_k<2>(shape, p, d_jobs, njobs, s);
    case 4: return launch_k<4>(shape, p, d_jobs, njobs, s);
    case 8: return launch_k<8>(shape, p, d_jobs, njobs, s);
    case 16: return launch_k<16>(shape, p, d_jobs, njobs, s);
    default: return cudaErrorInvalidValue;
  }
}

int max_smem_optin(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return v;
}

}  // namespace gb300_align
