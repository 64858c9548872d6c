// CTC prefix beam search with blank collapse (paper Sec. 5, "CUDA CTC
// decoder": beam search parallel over batch, hypotheses and vocabulary, after
// the blank collapse of the cited work with frame-skip threshold a).
//
// Two kernels.
//
// rank_kernel (one warp per frame, every frame of the batch at once): the B
// most probable non-blank labels of the frame (B rounds of a warp maximum
// over per-lane heads). They only serve to bound the selection below, so
// equal probabilities may come in any order. This work does not depend on
// the beam and is taken off the serial frame loop.
//
// beam_kernel (one CTA of 512 threads per utterance):
// Prologue (blank collapse): frame t is a blank frame when P[t, blank] > a;
// a blank frame that follows a blank frame is dropped (every run of blank
// frames shrinks to its first frame). A block-wide ballot scan writes the
// kept frame indices to the workspace.
// Per kept frame (the row and its ranked labels staged in shared memory with
// cp.async by warp 1, two frames ahead, a ring of four):
//   S1 (warp 0): every hypothesis' stay (blank: (pb + pnb) * y[blank];
//      repeat of its last label z: pnb * y[z]; plus the growth of the
//      hypothesis whose prefix is this one's minus its last label), and
//      theta = the B-th largest key among the stays and the growths of the
//      best hypothesis by the ranked labels: all actual candidates, so theta
//      is at most the B-th best key of the frame.
//   S2 (all threads): every growth (i, c): ((c == z_i) ? pb_i : pb_i + pnb_i)
//      * y[c]; keys >= theta go to a survivor list in shared memory (about B
//      of them).
//   S3 (warp 0): the top B survivors (rank of each key among the others, or
//      B rounds of warp arg-max when there are more than 32), the new beam
//      (new prefix-tree nodes for growths in the workspace), the power-of-two
//      rescale, and for the next frame the growth (i, c) equal to each
//      hypothesis j (64-bit prefix hashes as a filter, confirmed by walking
//      both prefixes in the tree).
// Keys are (value bits << 32) | (~candidate index): values are non-negative
// binary32, so key order is value order, then the smaller index (stays i
// < B, growths B + i * V + c). Every product and sum is one binary32
// operation in the same order as the definition (no FMA contraction, no
// flush to zero), so the result is the same bit for bit as a plain binary32
// evaluation in that order.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "align.h"

namespace gb300_align {
namespace {

constexpr int kThreads = 512;   // 16 warps: the growth test is latency-bound, more warps hide it
constexpr int kRankThreads = 256;
constexpr int kMaxBeam = 16;   // hypotheses per utterance at most (one lane per stay / growth)
constexpr int kRowRing = 4;    // staged rows
constexpr int kAhead = 2;      // rows in flight ahead of the one in use
constexpr int kSurvCap = 2048; // survivor keys per frame before the exact fallback
constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kHashEmpty = 0x6a09e667f3bcc908ull;

struct BeamArgs {
  const float* probs;        // [total_frames][V]
  const int64_t* foff;       // [n + 1]
  int32_t n, V, blank, B;
  float a;
  int32_t* kept_ws;          // [total_frames] kept frame indices
  const int32_t* topl;       // [total_frames][B] ranked labels of every frame (-1: none)
  int32_t* nparent;          // prefix-tree nodes: utterance u owns [foff[u] * B + u, + T_u * B + 1)
  int32_t* nlabel;
  int32_t* nframe;
  int32_t* tokens;           // hypothesis b of utterance u: [foff[u] * B + b * T_u, + T_u)
  int32_t* times;
  int32_t* lengths;          // [n * B]
  float* totals;             // [n * B]
  int32_t* scale_exp;        // [n]
  float* scores;             // [n * B]
  int32_t* nkept;            // [n]
};

// Hash of a prefix grown by label c (the splitmix64 finaliser over the parent
// hash and the label): only a filter, equality is confirmed on the tree.
__device__ __forceinline__ uint64_t grow_hash(uint64_t h, int c) {
  uint64_t x = h ^ (static_cast<uint64_t>(c + 1) * 0x9e3779b97f4a7c15ull);
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

__device__ __forceinline__ uint64_t make_key(float v, uint32_t idx) {
  return (static_cast<uint64_t>(__float_as_uint(v)) << 32) | static_cast<uint64_t>(0xffffffffu - idx);
}
__device__ __forceinline__ uint32_t key_index(uint64_t k) { return 0xffffffffu - static_cast<uint32_t>(k); }
__device__ __forceinline__ float key_value(uint64_t k) { return __uint_as_float(static_cast<uint32_t>(k >> 32)); }

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m) {
  const uint32_t lo = __shfl_xor_sync(kFull, static_cast<uint32_t>(v), m);
  const uint32_t hi = __shfl_xor_sync(kFull, static_cast<uint32_t>(v >> 32), m);
  return (static_cast<uint64_t>(hi) << 32) | lo;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t k) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    const uint64_t o = shfl_xor_u64(k, m);
    k = k > o ? k : o;
  }
  return k;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16b(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// Named barrier 1 between warp 0 (waits) and warp 1 (arrives after its
// copies completed): orders the staged row before warp 0's reads.
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct BeamState {
  float pb[kMaxBeam], pnb[kMaxBeam];
  int32_t node[kMaxBeam], pnode[kMaxBeam], len[kMaxBeam], last[kMaxBeam];
  uint64_t h[kMaxBeam], hp[kMaxBeam];
};

struct BeamShared {
  BeamState st[2];
  float s[kMaxBeam];        // pb + pnb of the current beam
  float stay_b[kMaxBeam], stay_nb[kMaxBeam];
  int32_t match[kMaxBeam];  // current beam: the hypothesis i whose growth by last[j] is j, or -1
  int32_t mword[kMaxBeam];  // merge bit set for j (word index into mbits, or -1)
  uint64_t theta;
  uint64_t kbuf[32];
  uint64_t sel[kMaxBeam];
  int32_t nsurv;
  int32_t overflow;
  int32_t nlive;
  int32_t warp_tot[kThreads / 32];
};

// The B largest non-blank labels of every frame (by probability; equal
// probabilities in any order), one warp per frame.
__global__ void __launch_bounds__(kRankThreads) rank_kernel(const float* __restrict__ probs, int64_t total_frames,
                                                        int V, int blank, int B, int32_t* __restrict__ topl) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * (kRankThreads / 32);
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * (kRankThreads / 32) + (threadIdx.x >> 5); g < total_frames;
       g += wstride) {
    const float* y = probs + g * V;
    // Lane head: its largest (value, ~label) key below the last one it gave.
    auto head_below = [&](uint64_t lim) {
      uint64_t h = 0;
      for (int c = lane; c < V; c += 32) {
        if (c == blank) continue;
        const uint64_t kc = make_key(__ldg(y + c), static_cast<uint32_t>(c));
        if (kc < lim && kc > h) h = kc;
      }
      return h;
    };
    uint64_t head = head_below(~0ull);
    for (int r = 0; r < B; ++r) {
      const unsigned hv = head ? static_cast<unsigned>(head >> 32) : 0u;
      const unsigned m = __reduce_max_sync(kFull, hv);
      const unsigned who = __ballot_sync(kFull, head != 0 && hv == m);
      int c = -1;
      if (who) {
        const int owner = __ffs(who) - 1;
        c = __shfl_sync(kFull, static_cast<int>(key_index(head)), owner);
        if (lane == owner) head = head_below(head);
      }
      if (lane == 0) topl[g * B + r] = c;
    }
  }
}

__global__ void __launch_bounds__(kThreads) beam_kernel(const BeamArgs A) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ BeamShared S;
  const int u = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int V = A.V, B = A.B, blank = A.blank;
  const int64_t f0 = A.foff[u];
  const int T = static_cast<int>(A.foff[u + 1] - f0);
  const int Vp = (V + 3) & ~3;
  const int Vq = Vp + kMaxBeam + 4;  // a ring slot: the row, its ranked labels, its frame index
  const int W = (V + 31) >> 5;
  float* rows = reinterpret_cast<float*>(dsm);                                      // [kRowRing][Vq]
  uint64_t* surv = reinterpret_cast<uint64_t*>(dsm + sizeof(float) * kRowRing * Vq);  // [kSurvCap]
  uint32_t* mbits = reinterpret_cast<uint32_t*>(surv + kSurvCap);                    // [B][W]
  const float* P = A.probs + f0 * V;
  int32_t* kept = A.kept_ws + f0;
  const int64_t nbase = f0 * B + u;  // root node of this utterance

  for (int w = tid; w < B * W; w += kThreads) mbits[w] = 0u;

  // ---- blank collapse: kept frame indices (ballot scan) ----
  int K = 0;
  for (int base = 0; base < T; base += kThreads) {
    const int t = base + tid;
    bool keep = false;
    if (t < T) {
      const bool bt = P[static_cast<int64_t>(t) * V + blank] > A.a;
      const bool bp = t > 0 && P[static_cast<int64_t>(t - 1) * V + blank] > A.a;
      keep = !(bt && bp);
    }
    const unsigned bal = __ballot_sync(kFull, keep);
    if (lane == 0) S.warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = K;
    int chunk = 0;
    for (int w2 = 0; w2 < kThreads / 32; ++w2) {
      const int c = S.warp_tot[w2];
      if (w2 < warp) before += c;
      chunk += c;
    }
    if (keep) kept[before + __popc(bal & ((1u << lane) - 1u))] = t;
    K += chunk;
    __syncthreads();
  }
  __syncthreads();  // kept[] visible to every thread (global writes of this block)

  const bool vec = (V & 3) == 0 && (reinterpret_cast<uintptr_t>(A.probs) & 15) == 0;
  // Rows are staged by warp 1 alone (its own cp.async groups) while warp 0
  // selects; a named barrier hands each staged row to warp 0 without a
  // block barrier.
  auto issue_row = [&](int k, int t) {
    if (k < K) {
      const float* src = P + static_cast<int64_t>(t) * V;
      float* dst = rows + (k % kRowRing) * Vq;
      if (vec) {
        for (int q = lane; q < (V >> 2); q += 32) cp_async16b(dst + 4 * q, src + 4 * q);
      } else {
        for (int q = lane; q < V; q += 32) cp_async4(dst + q, src + q);
      }
      if (lane < B) cp_async4(dst + Vp + lane, A.topl + (f0 + t) * B + lane);
      if (lane == 0) reinterpret_cast<int32_t*>(dst)[Vp + kMaxBeam] = t;
    }
    cp_commit();
  };

  // S1 for kept frame k over beam buffer c with nl live hypotheses (warp 0):
  // stays, merged growths, theta and the stays above it.
  auto stage1 = [&](int k, int c, int nl) {
    const float* y = rows + (k % kRowRing) * Vq;
    const int32_t* ranked = reinterpret_cast<const int32_t*>(y + Vp);
    const BeamState& ob = S.st[c];
    const int j = lane & 15;
    uint64_t key = 0;
    if (lane < 16) {
      if (j < nl) {  // stay of hypothesis j
        const float sj = ob.pb[j] + ob.pnb[j];
        const float sb = sj * y[blank];
        float snb = ob.len[j] > 0 ? ob.pnb[j] * y[ob.last[j]] : 0.0f;
        const int i = S.match[j];
        if (i >= 0) {
          const int cj = ob.last[j];
          const float si = ob.pb[i] + ob.pnb[i];
          const float base = (ob.last[i] == cj) ? ob.pb[i] : si;
          snb = snb + base * y[cj];
        }
        S.s[j] = sj;
        S.stay_b[j] = sb;
        S.stay_nb[j] = snb;
        key = make_key(sb + snb, static_cast<uint32_t>(j));
      }
    } else if (j < B) {  // growth of hypothesis 0 by its j-th ranked label, when not merged
      const int cr = ranked[j];
      if (cr >= 0 && !((mbits[cr >> 5] >> (cr & 31)) & 1u)) {
        const float base = (ob.last[0] == cr) ? ob.pb[0] : ob.pb[0] + ob.pnb[0];
        key = make_key(base * y[cr], static_cast<uint32_t>(B + cr));
      }
    }
    // theta: the key of rank B-1 among these actual candidates (0 when fewer than B).
    S.kbuf[lane] = key;
    __syncwarp();
    int rank = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) rank += S.kbuf[q] > key;
    const unsigned at = __ballot_sync(kFull, key != 0 && rank == B - 1);
    const uint64_t theta = at ? S.kbuf[__ffs(at) - 1] : 0ull;
    const bool put = lane < 16 && j < nl && key >= theta;
    const unsigned bal = __ballot_sync(kFull, put);
    if (put) surv[__popc(bal & ((1u << lane) - 1u))] = key;
    if (lane == 0) {
      S.theta = theta;
      S.nsurv = __popc(bal);
      S.overflow = 0;
    }
  };

  int n = 1, cur = 0, E = 0;  // uniform across the block
  int t_pref = 0;             // warp 1: frame index of the next row to stage
  const float invV = 1.0f / static_cast<float>(V);
  if (warp == 0) {
    if (lane == 0) {
      BeamState& b0 = S.st[0];
      b0.pb[0] = 1.0f;
      b0.pnb[0] = 0.0f;
      b0.node[0] = 0;
      b0.pnode[0] = -1;
      b0.len[0] = 0;
      b0.last[0] = -1;
      b0.h[0] = kHashEmpty;
      b0.hp[0] = 0;
      S.nlive = 1;
      A.nparent[nbase] = -1;
      A.nlabel[nbase] = -1;
      A.nframe[nbase] = -1;
    }
    if (lane < kMaxBeam) {
      S.match[lane] = -1;
      S.mword[lane] = -1;
    }
  } else if (warp == 1) {  // rows are staged by warp 1 (its own cp.async groups)
    for (int k = 0; k < kAhead; ++k) issue_row(k, k < K ? kept[k] : 0);
    t_pref = kAhead < K ? kept[kAhead] : 0;
    cp_wait<kAhead - 1>();
  }
  __syncthreads();  // row 0 staged, the initial beam written
  if (warp == 0 && K > 0) stage1(0, 0, 1);
  __syncthreads();

  for (int k = 0; k < K; ++k) {
    const float* y = rows + (k % kRowRing) * Vq;
    const BeamState& ob = S.st[cur];

    // ---- S2 (all threads): growths above theta ----
    {
      const uint64_t theta = S.theta;
      for (int c = tid; c < V; c += kThreads) {
        if (c == blank) continue;
        const float yc = y[c];
        unsigned hit = 0;  // hypotheses whose growth by c reaches theta
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
          const float base = (ob.last[i] == c) ? ob.pb[i] : S.s[i];
          const uint64_t key = make_key(base * yc, static_cast<uint32_t>(B + i * V + c));
          hit |= (key >= theta) ? (1u << i) : 0u;
        }
        while (hit) {  // rare: recompute the key and append it unless merged
          const int i = __ffs(hit) - 1;
          hit &= hit - 1;
          if ((mbits[i * W + (c >> 5)] >> (c & 31)) & 1u) continue;
          const float base = (ob.last[i] == c) ? ob.pb[i] : S.s[i];
          const uint64_t key = make_key(base * yc, static_cast<uint32_t>(B + i * V + c));
          const int slot = atomicAdd(&S.nsurv, 1);
          if (slot < kSurvCap) surv[slot] = key;
          else S.overflow = 1;
        }
      }
    }
    __syncthreads();

    // ---- S3 (warp 0): selection, new beam, rescale, merges; then S1 of the next frame ----
    if (warp == 0) {
      const int ns = min(S.nsurv, kSurvCap);
      uint64_t mine = 0;  // this lane's selected key (0: none) and its place in the new beam
      int slot = lane;
      if (!S.overflow && ns <= 32) {  // rank of each survivor among the others
        mine = lane < ns ? surv[lane] : 0ull;
        int rank = 0;
#pragma unroll 8
        for (int q = 0; q < ns; ++q) rank += surv[q] > mine;
        slot = rank;
      } else {
        // B rounds of warp arg-max below the previous pick: over the survivors,
        // or over every candidate when the survivor list overflowed.
        uint64_t prev = ~0ull;
        for (int b = 0; b < B; ++b) {
          uint64_t best = 0;
          if (!S.overflow) {
            for (int q = lane; q < ns; q += 32) {
              const uint64_t kk = surv[q];
              if (kk < prev && kk > best) best = kk;
            }
          } else {
            for (int i = lane; i < n; i += 32) {
              const uint64_t kk = make_key(S.stay_b[i] + S.stay_nb[i], static_cast<uint32_t>(i));
              if (kk < prev && kk > best) best = kk;
            }
            for (int c = lane; c < V; c += 32) {
              if (c == blank) continue;
              for (int i = 0; i < n; ++i) {
                if ((mbits[i * W + (c >> 5)] >> (c & 31)) & 1u) continue;
                const float base = (ob.last[i] == c) ? ob.pb[i] : S.s[i];
                const uint64_t kk = make_key(base * y[c], static_cast<uint32_t>(B + i * V + c));
                if (kk < prev && kk > best) best = kk;
              }
            }
          }
          best = warp_max_u64(best);
          if (lane == b) mine = best;
          prev = best;
          if (best == 0) break;
        }
      }
      const bool valid = mine != 0 && slot < B;
      const unsigned have = __ballot_sync(kFull, valid);
      const int nb = __popc(have);  // the new beam fills slots 0 .. nb-1
      // The largest total is the value of the slot-0 key (stays: the same
      // sum; growths: 0 + value): the rescale by a power of two that brings
      // it into [0.5, 1) is known before the entries are written.
      const unsigned top = __ballot_sync(kFull, valid && slot == 0);
      const float m = __uint_as_float(__shfl_sync(kFull, static_cast<unsigned>(mine >> 32), __ffs(top) - 1));
      int e = 0;
      float f = 1.0f;
      bool pow2 = true;
      if (m > 0.0f) {
        const uint32_t mb = __float_as_uint(m);
        e = static_cast<int>((mb >> 23) & 0xffu) - 126;  // m = f * 2^e, f in [0.5, 1), m normal
        if (mb >= 0x00800000u && e > -126 && e < 127) {
          f = __uint_as_float(static_cast<uint32_t>(127 - e) << 23);  // 2^-e, a normal float
        } else {
          (void)frexpf(m, &e);
          pow2 = false;
        }
        E += e;
      }
      const int t_k = reinterpret_cast<const int32_t*>(y + Vp)[kMaxBeam];
      BeamState& nbm = S.st[cur ^ 1];
      if (valid) {
        const uint32_t idx = key_index(mine);
        float pbv, pnbv;
        if (idx < static_cast<uint32_t>(B)) {  // a stay
          const int i = static_cast<int>(idx);
          pbv = S.stay_b[i];
          pnbv = S.stay_nb[i];
          nbm.node[slot] = ob.node[i];
          nbm.pnode[slot] = ob.pnode[i];
          nbm.len[slot] = ob.len[i];
          nbm.last[slot] = ob.last[i];
          nbm.h[slot] = ob.h[i];
          nbm.hp[slot] = ob.hp[i];
        } else {  // a growth: a new node of the prefix tree
          const int r = static_cast<int>(idx) - B;  // i * V + c with i < 16: exact in a float
          int i = static_cast<int>(static_cast<float>(r) * invV);
          if (i * V > r) --i;
          if ((i + 1) * V <= r) ++i;
          const int c = r - i * V;
          const int id = 1 + k * B + slot;
          A.nparent[nbase + id] = ob.node[i];
          A.nlabel[nbase + id] = c;
          A.nframe[nbase + id] = t_k;
          pbv = 0.0f;
          pnbv = key_value(mine);
          nbm.node[slot] = id;
          nbm.pnode[slot] = ob.node[i];
          nbm.len[slot] = ob.len[i] + 1;
          nbm.last[slot] = c;
          nbm.h[slot] = grow_hash(ob.h[i], c);
          nbm.hp[slot] = ob.h[i];
        }
        if (m > 0.0f) {
          pbv = pow2 ? pbv * f : ldexpf(pbv, -e);
          pnbv = pow2 ? pnbv * f : ldexpf(pnbv, -e);
        }
        nbm.pb[slot] = pbv;
        nbm.pnb[slot] = pnbv;
      }
      // Clear last frame's merge bits; then for each new hypothesis j (lane
      // 16 + j) the hypothesis i (lane i) whose prefix is j's minus its last
      // label: equal (hash, length) keys by a warp match, confirmed by the
      // parent node, or by walking both prefixes when the nodes differ.
      if (lane < kMaxBeam && S.mword[lane] >= 0) {
        mbits[S.mword[lane]] = 0u;
        S.mword[lane] = -1;
      }
      __syncwarp();
      const int e16 = lane & 15;
      const bool as_i = lane < 16 && e16 < nb;
      const bool as_j = lane >= 16 && e16 < nb && nbm.len[e16] > 0;
      uint64_t mk = ~static_cast<uint64_t>(lane);  // matches nothing real in practice; confirmed below anyway
      if (as_i) mk = nbm.h[e16] ^ (static_cast<uint64_t>(nbm.len[e16]) * 0x9e3779b97f4a7c15ull);
      if (as_j) mk = nbm.hp[e16] ^ (static_cast<uint64_t>(nbm.len[e16] - 1) * 0x9e3779b97f4a7c15ull);
      const unsigned imask = __ballot_sync(kFull, as_i);
      unsigned cand = __match_any_sync(kFull, mk) & imask;
      int match = -1;
      if (as_j) {
        const int32_t* par = A.nparent + nbase;
        const int32_t* lab = A.nlabel + nbase;
        while (cand && match < 0) {
          const int i = __ffs(cand) - 1;
          cand &= cand - 1;
          if (nbm.len[i] != nbm.len[e16] - 1) continue;
          int x = nbm.node[i];
          int z = nbm.pnode[e16];
          bool same = true;
          for (int step = 0; step <= nbm.len[i] && x != z; ++step) {  // equal depths: both reach the root
            if (lab[x] != lab[z]) {
              same = false;
              break;
            }
            x = par[x];
            z = par[z];
          }
          if (same && x == z) match = i;
        }
        S.match[e16] = match;
      } else if (lane >= 16) {
        S.match[e16] = -1;
      }
      __syncwarp();
      if (match >= 0) {
        const int c = nbm.last[e16];
        const int w = match * W + (c >> 5);
        atomicOr(&mbits[w], 1u << (c & 31));
        S.mword[e16] = w;
      }
      if (lane == 0) S.nlive = nb;
      // Next frame's S1 once warp 1 has staged its row (named barrier 1).
      named_sync(1, 64);
      if (k + 1 < K) stage1(k + 1, cur ^ 1, nb);
    } else if (warp == 1) {
      // Meanwhile: stage row k + 2, wait for row k + 1, signal warp 0.
      issue_row(k + kAhead, t_pref);
      t_pref = (k + kAhead + 1 < K) ? kept[k + kAhead + 1] : 0;  // used one frame later
      cp_wait<kAhead - 1>();
      named_arrive(1, 64);
    }
    cur ^= 1;
    __syncthreads();  // the new beam, its merges, theta and the next row are visible to every warp
    n = S.nlive;
  }
  cp_wait<0>();

  // ---- outputs (warp 0): hypotheses in beam order ----
  if (warp == 0) {
    const BeamState& fb = S.st[cur];
    const int64_t hbase = static_cast<int64_t>(u) * B;
    if (lane < B) {
      if (lane < n) {
        const float tot = fb.pb[lane] + fb.pnb[lane];
        A.totals[hbase + lane] = tot;
        A.scores[hbase + lane] = tot > 0.0f ? logf(tot) + static_cast<float>(E) * 0.693147180559945f : -INFINITY;
        const int L = fb.len[lane];
        A.lengths[hbase + lane] = L;
        int32_t* tk = A.tokens + f0 * B + static_cast<int64_t>(lane) * T;
        int32_t* tm = A.times + f0 * B + static_cast<int64_t>(lane) * T;
        int x = fb.node[lane];
        for (int p = L - 1; p >= 0; --p) {
          tk[p] = A.nlabel[nbase + x];
          tm[p] = A.nframe[nbase + x];
          x = A.nparent[nbase + x];
        }
      } else {
        A.totals[hbase + lane] = 0.0f;
        A.scores[hbase + lane] = -INFINITY;
        A.lengths[hbase + lane] = -1;
      }
    }
    if (lane == 0) {
      A.scale_exp[u] = E;
      A.nkept[u] = K;
    }
  }
}

}  // namespace
}  // namespace gb300_align

using namespace gb300_align;

extern "C" {

uint64_t align_ctc_beam_workspace_bytes(int32_t n, int64_t total_frames, int32_t beam) {
  if (n < 0 || total_frames < 0 || beam < 1) return 0;
  const uint64_t nodes = static_cast<uint64_t>(total_frames) * beam + n;
  const uint64_t kept = (static_cast<uint64_t>(total_frames) * 4 + 255) & ~255ull;
  const uint64_t arr = (nodes * 4 + 255) & ~255ull;
  const uint64_t ranked = (static_cast<uint64_t>(total_frames) * beam * 4 + 255) & ~255ull;
  return kept + 3 * arr + ranked;
}

int align_ctc_beam_decode(const float* probs, const int64_t* frame_offsets, int32_t n, int64_t total_frames,
                          int32_t V, int32_t blank, int32_t beam, float threshold, void* workspace,
                          uint64_t workspace_bytes, int32_t* tokens, int32_t* timesteps, int32_t* lengths,
                          float* totals, int32_t* scale_exp, float* scores, int32_t* kept, void* cuda_stream) {
  if (n < 0 || total_frames < 0 || V < 2 || blank < 0 || blank >= V || beam < 1 || beam > kMaxBeam ||
      !(threshold >= 0.0f))
    return ALIGN_E_INVAL;
  if (static_cast<int64_t>(beam) * V + beam >= 0x7fffffffll) return ALIGN_E_TOO_LARGE;
  if (n == 0) return ALIGN_OK;
  if (!probs || !frame_offsets || !workspace || !tokens || !timesteps || !lengths || !totals || !scale_exp ||
      !scores || !kept)
    return ALIGN_E_INVAL;
  if (workspace_bytes < align_ctc_beam_workspace_bytes(n, total_frames, beam)) return ALIGN_E_INVAL;
  const uint64_t nodes = static_cast<uint64_t>(total_frames) * beam + n;
  const uint64_t kbytes = (static_cast<uint64_t>(total_frames) * 4 + 255) & ~255ull;
  const uint64_t abytes = (nodes * 4 + 255) & ~255ull;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  BeamArgs a{};
  a.probs = probs;
  a.foff = frame_offsets;
  a.n = n;
  a.V = V;
  a.blank = blank;
  a.B = beam;
  a.a = threshold;
  a.kept_ws = reinterpret_cast<int32_t*>(ws);
  a.nparent = reinterpret_cast<int32_t*>(ws + kbytes);
  a.nlabel = reinterpret_cast<int32_t*>(ws + kbytes + abytes);
  a.nframe = reinterpret_cast<int32_t*>(ws + kbytes + 2 * abytes);
  int32_t* topl = reinterpret_cast<int32_t*>(ws + kbytes + 3 * abytes);
  a.topl = topl;
  a.tokens = tokens;
  a.times = timesteps;
  a.lengths = lengths;
  a.totals = totals;
  a.scale_exp = scale_exp;
  a.scores = scores;
  a.nkept = kept;
  const int Vq = ((V + 3) & ~3) + kMaxBeam + 4;
  const size_t smem = sizeof(float) * kRowRing * Vq + sizeof(uint64_t) * kSurvCap +
                      sizeof(uint32_t) * beam * ((V + 31) / 32);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ALIGN_E_CUDA;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem + sizeof(BeamShared) > static_cast<size_t>(optin)) return ALIGN_E_TOO_LARGE;
  if (cudaFuncSetAttribute(beam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess)
    return ALIGN_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (total_frames > 0) {
    const int64_t blocks = std::min<int64_t>((total_frames + kRankThreads / 32 - 1) / (kRankThreads / 32),
                                             static_cast<int64_t>(std::max(sms, 1)) * 8);
    rank_kernel<<<static_cast<unsigned>(blocks), kRankThreads, 0, st>>>(probs, total_frames, V, blank, beam, topl);
  }
  beam_kernel<<<n, kThreads, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? ALIGN_OK : ALIGN_E_CUDA;
}

}  // extern "C"
