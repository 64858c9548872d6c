// Device helpers shared by the trellis kernels (generic and fast paths):
// inline-PTX wrappers (cluster ranks, DSMEM stores, release / acquire,
// mbarriers, bulk and asynchronous copies), bounded waits, the shared-memory
// head and the grid-team barrier.
#pragma once
#include <cuda_runtime.h>

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
__device__ __forceinline__ void st_remote_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_gpu_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_gpu_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy (bulk copy) writes to the same addresses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Non-blocking test of an mbarrier phase (polling; never suspends the thread).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Potentially blocking test: the thread may be suspended until the phase
// completes or about `ns` nanoseconds pass (then false), so a waiting warp
// leaves its scheduler's issue slots to the others.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
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
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// ------------------------------------------------------- shared-memory head --
struct SmemHead {
  uint64_t full[kMaxStages];   // emission stage filled
  uint64_t empty[kMaxStages];  // emission stage released by every warp
  int32_t abort;            // set by any thread of this CTA whose wait hit the limit
  uint32_t unused;
  uint64_t sink;            // scratch slot written by the last warp of the team
  uint64_t tailbar;         // fast kernel: completion of the anchor-row copies of the backtrack
  uint64_t pad2;
  float fin[2];             // fast kernel, CTA 0 of a cluster team: alpha_{T-1} of states S-2, S-1
  uint32_t team_bad;        // fast kernel, cluster teams: set in every CTA by a CTA whose wait ran out
  uint32_t pad;
  FwdJob job;               // fast kernel: this CTA's copy of its job descriptor
};
static_assert(sizeof(SmemHead) % 16 == 0, "head size: what follows it is 16-byte aligned");

// Bounded wait on an mbarrier phase, done by one lane. Returns false on
// timeout (and raises the CTA abort flag) or when another warp aborted.
__device__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int32_t* abort, uint64_t limit,
                           bool honour_abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    if (mbar_try_wait_suspend(bar, parity, 10000u)) return true;
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


// Slow path of the cross-CTA flow control: wait until the next CTA has
// consumed frame `need` (its published progress exceeds it).
__device__ __noinline__ uint32_t prog_spin(const volatile uint32_t* prog, int need, volatile int32_t* abort,
                                           uint64_t limit) {
  const uint64_t t0 = gtimer();
  for (;;) {
    const uint32_t v = *prog;
    if (static_cast<int>(v) > need) return v;
    if (*abort || gtimer() - t0 > limit) {
      *abort = 1;
      return v;
    }
  }
}

// Stores executed by one lane, written as predicated PTX so the frame loop has
// no lane-dependent branch.
__device__ __forceinline__ void st_global_v4_if(uint32_t* p, uint32_t x, uint32_t y, uint32_t z, uint32_t w,
                                                bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t@q st.global.v4.u32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
      "r"(x), "r"(y), "r"(z), "r"(w), "r"(static_cast<uint32_t>(pred))
      : "memory");
}
__device__ __forceinline__ void st_cluster_u64_if(uint32_t addr, uint64_t v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.relaxed.cluster.shared::cluster.u64 [%0], %1;\n\t}" ::"r"(
          addr),
      "l"(v), "r"(static_cast<uint32_t>(pred))
      : "memory");
}
__device__ __forceinline__ void st_gpu_u64_if(uint64_t* p, uint64_t v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.relaxed.gpu.u64 [%0], %1;\n\t}" ::"l"(p), "l"(v),
      "r"(static_cast<uint32_t>(pred))
      : "memory");
}

// Barrier of the CTAs of a grid team (co-resident: cooperative launch, one
// CTA per SM). bar[0] counts arrivals, bar[1] is the generation. Bounded: on
// timeout the CTA raises its abort flag and continues.
__device__ void team_barrier(uint32_t* bar, uint32_t ncta, volatile int32_t* abort, uint64_t limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t gen = ld_acquire_gpu_u32(bar + 1);
    if (atomicAdd(bar, 1u) == ncta - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      st_release_gpu_u32(bar + 1, gen + 1u);
    } else {
      const uint64_t t0 = gtimer();
      while (ld_acquire_gpu_u32(bar + 1) == gen) {
        if (gtimer() - t0 > limit) {
          *abort = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

}  // namespace
}  // namespace gb300_align
