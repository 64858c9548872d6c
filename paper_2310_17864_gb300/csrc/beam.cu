// CTC prefix beam search with blank collapse (paper Sec. 5, "CUDA CTC
// decoder": beam search parallel over batch, hypotheses and vocabulary, after
// the blank collapse of the cited work with frame-skip threshold a).
//
// One CTA per utterance, 256 threads.
//
// Prologue (blank collapse): frame t is a blank frame when P[t, blank] > a;
// a blank frame that follows a blank frame is dropped (every run of blank
// frames shrinks to its first frame). A block-wide ballot scan writes the
// kept frame indices to the workspace.
//
// Per kept frame (rows staged in shared memory with cp.async, two frames
// ahead, a ring of four rows):
//   S1 (warp 0): the two most probable non-blank labels of the frame; every
//      hypothesis' stay (blank: (pb + pnb) * y[blank]; repeat of its last
//      label z: pnb * y[z]; plus the growth of the hypothesis whose prefix is
//      this one's minus its last label); a lower bound theta of the B-th best
//      candidate key from 2n actual candidates (the n stays and each
//      hypothesis' growth by its best non-merged label).
//   S2 (all threads): every growth (i, c): ((c == z_i) ? pb_i : pb_i + pnb_i)
//      * y[c]; keys >= theta go to a survivor list in shared memory.
//   S3 (warp 0): the top B survivors (a 32-lane bitonic sort, or B rounds of
//      warp arg-max), the new beam (new prefix-tree nodes for growths in the
//      workspace), the power-of-two rescale, and for the next frame the
//      growth (i, c) equal to each hypothesis j (64-bit prefix hashes as a
//      filter, confirmed by walking both prefixes in the tree).
// Keys are (value bits << 32) | (~candidate index): values are non-negative
// binary32, so key order is value order, then the smaller index (stays i
// < B, growths B + i * V + c). Every product and sum is one binary32
// operation in the same order as the definition (no FMA contraction, no
// flush to zero), so the result is the same bit for bit as a plain binary32
// evaluation in that order.
#include <cstdint>

#include <cuda_runtime.h>

#include "align.h"

namespace gb300_align {
namespace {

constexpr int kThreads = 256;
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

// Descending bitonic sort of one 64-bit key per lane across the warp.
__device__ __forceinline__ uint64_t warp_sort_desc(uint64_t k, int lane) {
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const uint64_t o = shfl_xor_u64(k, stride);
      const bool up = (lane & size) == 0;        // this block sorts descending when up
      const bool lower = (lane & stride) == 0;   // this lane keeps the larger key when lower == up
      const bool keep_max = (lower == up);
      k = keep_max ? (k > o ? k : o) : (k < o ? k : o);
    }
  }
  return k;
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
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct BeamState {
  float pb[kMaxBeam], pnb[kMaxBeam];
  int32_t node[kMaxBeam], len[kMaxBeam], last[kMaxBeam];
  uint64_t h[kMaxBeam], hp[kMaxBeam];
};

struct BeamShared {
  BeamState st[2];
  float s[kMaxBeam];        // pb + pnb of the current beam
  float stay_b[kMaxBeam], stay_nb[kMaxBeam];
  int32_t match[kMaxBeam];  // current beam: the hypothesis i whose growth by last[j] is j, or -1
  int32_t mword[kMaxBeam];  // merge bit set for j (word index into mbits, or -1)
  uint64_t theta;
  int32_t nsurv;
  int32_t overflow;
  int32_t nlive;
  int32_t warp_tot[kThreads / 32];
};

__global__ void __launch_bounds__(kThreads) beam_kernel(const BeamArgs A) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ BeamShared S;
  const int u = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int V = A.V, B = A.B, blank = A.blank;
  const int64_t f0 = A.foff[u];
  const int T = static_cast<int>(A.foff[u + 1] - f0);
  const int Vp = (V + 3) & ~3;
  const int W = (V + 31) >> 5;
  float* rows = reinterpret_cast<float*>(dsm);                                      // [kRowRing][Vp]
  uint64_t* surv = reinterpret_cast<uint64_t*>(dsm + sizeof(float) * kRowRing * Vp);  // [kSurvCap]
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
  auto issue_row = [&](int k) {
    if (k < K) {
      const float* src = P + static_cast<int64_t>(kept[k]) * V;
      float* dst = rows + (k % kRowRing) * Vp;
      if (vec) {
        for (int q = tid; q < (V >> 2); q += kThreads) cp_async16b(dst + 4 * q, src + 4 * q);
      } else {
        for (int q = tid; q < V; q += kThreads) cp_async4(dst + q, src + q);
      }
    }
    cp_commit();
  };

  if (tid == 0) {
    BeamState& b0 = S.st[0];
    b0.pb[0] = 1.0f;
    b0.pnb[0] = 0.0f;
    b0.node[0] = 0;
    b0.len[0] = 0;
    b0.last[0] = -1;
    b0.h[0] = kHashEmpty;
    b0.hp[0] = 0;
    A.nparent[nbase] = -1;
    A.nlabel[nbase] = -1;
    A.nframe[nbase] = -1;
  }
  if (tid < kMaxBeam) {
    S.match[tid] = -1;
    S.mword[tid] = -1;
  }
  int n = 1, cur = 0, E = 0;  // uniform across the block
  for (int k = 0; k < kAhead; ++k) issue_row(k);
  __syncthreads();

  for (int k = 0; k < K; ++k) {
    issue_row(k + kAhead);
    cp_wait<kAhead>();
    __syncthreads();  // row k staged by every thread
    const float* y = rows + (k % kRowRing) * Vp;
    const BeamState& ob = S.st[cur];

    // ---- S1 (warp 0): stays, merged growths, theta ----
    if (warp == 0) {
      uint64_t k1 = 0, k2 = 0;  // two best non-blank labels: (y bits, ~c)
      for (int c = lane; c < V; c += 32) {
        if (c == blank) continue;
        const uint64_t kc = make_key(y[c], static_cast<uint32_t>(c));
        if (kc > k1) {
          k2 = k1;
          k1 = kc;
        } else if (kc > k2) {
          k2 = kc;
        }
      }
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) {
        const uint64_t o1 = shfl_xor_u64(k1, m), o2 = shfl_xor_u64(k2, m);
        const uint64_t n1 = k1 > o1 ? k1 : o1;
        const uint64_t n2 = k1 > o1 ? (k2 > o1 ? k2 : o1) : (k1 > o2 ? k1 : o2);
        k1 = n1;
        k2 = n2;
      }
      const int c1 = k1 ? static_cast<int>(key_index(k1)) : -1;
      const int c2 = k2 ? static_cast<int>(key_index(k2)) : -1;
      const int j = lane & 15;
      float sj = 0.0f;
      if (j < n) sj = ob.pb[j] + ob.pnb[j];
      uint64_t key = 0;
      if (lane < 16 && j < n) {  // stays
        const float sb = sj * y[blank];
        float snb = ob.len[j] > 0 ? ob.pnb[j] * y[ob.last[j]] : 0.0f;
        const int i = S.match[j];
        if (i >= 0) {
          const int c = ob.last[j];
          const float si = ob.pb[i] + ob.pnb[i];
          const float base = (ob.last[i] == c) ? ob.pb[i] : si;
          snb = snb + base * y[c];
        }
        S.s[j] = sj;
        S.stay_b[j] = sb;
        S.stay_nb[j] = snb;
        key = make_key(sb + snb, static_cast<uint32_t>(j));
      } else if (lane >= 16 && j < n) {  // hypothesis j's growth by its best label that is not merged
        int c = -1;
        if (c1 >= 0 && !((mbits[j * W + (c1 >> 5)] >> (c1 & 31)) & 1u)) c = c1;
        else if (c2 >= 0 && !((mbits[j * W + (c2 >> 5)] >> (c2 & 31)) & 1u)) c = c2;
        if (c >= 0) {
          const float base = (ob.last[j] == c) ? ob.pb[j] : sj;
          key = make_key(base * y[c], static_cast<uint32_t>(B + j * V + c));
        }
      }
      const uint64_t sorted = warp_sort_desc(key, lane);
      const uint64_t th = __shfl_sync(kFull, static_cast<uint32_t>(sorted >> 32), B - 1);
      const uint64_t tl = __shfl_sync(kFull, static_cast<uint32_t>(sorted), B - 1);
      const uint64_t theta = (th << 32) | tl;  // 0 when fewer than B candidates were seen
      const bool put = lane < 16 && j < n && key >= theta;
      const unsigned bal = __ballot_sync(kFull, put);
      if (put) surv[__popc(bal & ((1u << lane) - 1u))] = key;
      if (lane == 0) {
        S.theta = theta;
        S.nsurv = __popc(bal);
        S.overflow = 0;
      }
    }
    __syncthreads();

    // ---- S2 (all threads): growths above theta ----
    {
      const uint64_t theta = S.theta;
      for (int c = tid; c < V; c += kThreads) {
        if (c == blank) continue;
        const float yc = y[c];
        for (int i = 0; i < n; ++i) {
          if ((mbits[i * W + (c >> 5)] >> (c & 31)) & 1u) continue;
          const float base = (ob.last[i] == c) ? ob.pb[i] : S.s[i];
          const uint64_t key = make_key(base * yc, static_cast<uint32_t>(B + i * V + c));
          if (key >= theta) {
            const int slot = atomicAdd(&S.nsurv, 1);
            if (slot < kSurvCap) surv[slot] = key;
            else S.overflow = 1;
          }
        }
      }
    }
    __syncthreads();

    // ---- S3 (warp 0): selection, new beam, rescale, merges of the next frame ----
    if (warp == 0) {
      const int ns = min(S.nsurv, kSurvCap);
      uint64_t mine = 0;  // lane b < B: the b-th selected key (0: none)
      if (!S.overflow && ns <= 32) {
        const uint64_t kk = lane < ns ? surv[lane] : 0ull;
        mine = warp_sort_desc(kk, lane);
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
      const unsigned have = __ballot_sync(kFull, lane < B && mine != 0);
      const int nb = __popc(have);  // selected keys occupy lanes 0 .. nb-1
      BeamState& nbm = S.st[cur ^ 1];
      float tot = 0.0f;
      if (lane < nb) {
        const uint32_t idx = key_index(mine);
        if (idx < static_cast<uint32_t>(B)) {  // a stay
          const int i = static_cast<int>(idx);
          nbm.pb[lane] = S.stay_b[i];
          nbm.pnb[lane] = S.stay_nb[i];
          nbm.node[lane] = ob.node[i];
          nbm.len[lane] = ob.len[i];
          nbm.last[lane] = ob.last[i];
          nbm.h[lane] = ob.h[i];
          nbm.hp[lane] = ob.hp[i];
        } else {  // a growth: a new node of the prefix tree
          const uint32_t r = idx - static_cast<uint32_t>(B);
          const int i = static_cast<int>(r / static_cast<uint32_t>(V));
          const int c = static_cast<int>(r % static_cast<uint32_t>(V));
          const int id = 1 + k * B + lane;
          A.nparent[nbase + id] = ob.node[i];
          A.nlabel[nbase + id] = c;
          A.nframe[nbase + id] = kept[k];
          nbm.pb[lane] = 0.0f;
          nbm.pnb[lane] = key_value(mine);
          nbm.node[lane] = id;
          nbm.len[lane] = ob.len[i] + 1;
          nbm.last[lane] = c;
          nbm.h[lane] = grow_hash(ob.h[i], c);
          nbm.hp[lane] = ob.h[i];
        }
        tot = nbm.pb[lane] + nbm.pnb[lane];
      }
      // Rescale by a power of two: the largest total into [0.5, 1).
      float m = tot;
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, s));
      if (m > 0.0f) {
        int e = 0;
        (void)frexpf(m, &e);
        if (lane < nb) {
          nbm.pb[lane] = ldexpf(nbm.pb[lane], -e);
          nbm.pnb[lane] = ldexpf(nbm.pnb[lane], -e);
        }
        E += e;
      }
      // Clear last frame's merge bits, then find this beam's merges.
      if (lane < kMaxBeam && S.mword[lane] >= 0) {
        mbits[S.mword[lane]] = 0u;
        S.mword[lane] = -1;
      }
      __syncwarp();
      int match = -1;
      if (lane < nb && nbm.len[lane] > 0) {
        const int32_t* par = A.nparent + nbase;
        const int32_t* lab = A.nlabel + nbase;
        for (int i = 0; i < nb && match < 0; ++i) {
          if (nbm.len[i] != nbm.len[lane] - 1 || nbm.h[i] != nbm.hp[lane]) continue;
          int x = nbm.node[i];
          int z = par[nbm.node[lane]];
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
      }
      if (lane < kMaxBeam) S.match[lane] = lane < nb ? match : -1;
      __syncwarp();
      if (match >= 0) {
        const int c = nbm.last[lane];
        const int w = match * W + (c >> 5);
        atomicOr(&mbits[w], 1u << (c & 31));
        S.mword[lane] = w;
      }
      if (lane == 0) S.nlive = nb;
    }
    cur ^= 1;
    __syncthreads();  // the new beam, its merges and its size are visible to every warp
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
  return kept + 3 * arr;
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
  a.tokens = tokens;
  a.times = timesteps;
  a.lengths = lengths;
  a.totals = totals;
  a.scale_exp = scale_exp;
  a.scores = scores;
  a.nkept = kept;
  const int Vp = (V + 3) & ~3;
  const size_t smem = sizeof(float) * kRowRing * Vp + sizeof(uint64_t) * kSurvCap +
                      sizeof(uint32_t) * beam * ((V + 31) / 32);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ALIGN_E_CUDA;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem + sizeof(BeamShared) > static_cast<size_t>(optin)) return ALIGN_E_TOO_LARGE;
  if (cudaFuncSetAttribute(beam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess)
    return ALIGN_E_CUDA;
  beam_kernel<<<n, kThreads, smem, static_cast<cudaStream_t>(cuda_stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? ALIGN_OK : ALIGN_E_CUDA;
}

}  // extern "C"
