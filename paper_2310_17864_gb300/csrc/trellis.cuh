// Device-side descriptors shared by the trellis kernels and the host runtime.
//
// Trellis (CTC, as used by the forced-alignment feature of TorchAudio 2.1,
// paper Sec. 4): S = 2L+1 states; even states are the blank, odd state s
// carries targets[(s-1)/2].
//
// Work decomposition: one alignment ("job") is owned by a team of warps that
// are chained along the state axis. Warp g of the team holds states
// [32*K*g, 32*K*(g+1)); lane l of it holds the K consecutive states starting
// at 32*K*g + K*l, in registers. Information only flows towards larger s
// (alpha_t(s) reads s, s-1, s-2 at t-1), so each warp only needs one value
// per frame from its left neighbour: alpha_{t-1}(first state - 1). Inside a
// warp it comes by shuffle, between warps of a CTA through a tagged ring in
// shared memory, between CTAs of a thread-block cluster through the same
// ring written over distributed shared memory. Warps therefore run as a
// skewed pipeline: no barrier per frame.
//
// Backpointer layout of the generic kernel (2 bits of information per cell,
// packed by warp ballots; the fast kernel's per-window layout is described in
// trellis_fast.cu): for warp g and stored frame row r, NW = 3K/2 32-bit words
//   word j      (0 <= j < K): bit l = "advance won" for state 32Kg + Kl + j
//   word K + i  (0 <= i < K/2): bit l = "skip won" for the label state
//                               32Kg + Kl + 2i + 1
// at bp[(g * bp_rows + r) * NW]. The predecessor is s-2 if the skip bit is
// set, else s-1 if the advance bit is set, else s.
//
// Anchors (for a parallel backtrack): frames t_begin + m*D (D = kAnchorD) are
// anchor frames. Along the forward pass every state also carries anchor(s),
// the state at the last anchor frame on its best path (selected with the same
// predicates as the max). At the end of window m (frame t_begin + (m+1)*D, or
// the last frame) row m of ztab stores s - anchor(s) in [0, 2D] as a byte;
// the anchors are then reset to s. The backtrack hops from window to window
// through these rows, then walks every window's 32 frames in parallel.
//
// Ring word (one per frame and warp boundary): bits 63..40 frame tag
// (t + 1 mod 2^24), bits 39..32 anchor offset of the sent state, bits 31..0
// alpha as FP32 bits.
#pragma once
#include <cstdint>

namespace gb300_align {

constexpr int kMaxStages = 16;        // emission ring stages per CTA, at most (planned per shape)
constexpr int kLead = 4;              // stages in flight ahead of the consumer
constexpr int kBtWindow = 32;         // frames per backtrack window
constexpr int kAnchorD = 32;          // frames between anchor rows (== kBtWindow)
constexpr int kHopBatch = 32;         // anchor rows fetched per batch while hopping back
constexpr int kHopSpan = 640;         // states below the current one staged per anchor row
constexpr int kHopRowBytes = (kHopSpan + 32 + 15) / 16 * 16;  // staged bytes per row (16-aligned range)
constexpr int kTagBits = 24;          // frame tag bits in a ring word

// Job flags.
constexpr uint32_t kJobWriteFinal = 1u;  // pick the final state, write total/status/state_io
constexpr uint32_t kJobChase = 2u;       // walk the backpointers from state_io and write outputs
constexpr uint32_t kJobBulkRows = 4u;    // emission rows may be staged with cp.async.bulk
constexpr uint32_t kJobTestStall = 8u;   // test hook: warp 0 of the team never sends (waits run out)

struct alignas(16) FwdJob {
  const float* lp;         // [T][C] row-major FP32
  const int32_t* tgt;      // [L] device copy of the targets
  uint32_t* bp;            // packed backpointers (nullptr: none stored)
  float* ckpt;             // alpha rows at frames 0, ck_every, 2*ck_every, ... (nullptr: none)
  const float* alpha_in;   // alpha at t_begin (S floats); nullptr: the t = 0 initialisation
  float* final2;           // [2] alpha_{T-1}(S-2), alpha_{T-1}(S-1) (generic kernel; the fast
                           // kernel keeps them in shared memory or the team block)
  int32_t* status;         // request status word (see align.h codes)
  int32_t* state_io;       // chase entry state (in) / state at t_begin (out)
  int32_t* path;           // [T] outputs (nullptr when not chasing)
  float* scores;           // [T]
  float* total;            // [1]
  int32_t* states;         // [T] or nullptr
  int32_t T, C, blank, L;
  int32_t S;
  int32_t t_begin;         // first frame of this pass
  int32_t t_end;           // one past the last frame of this pass
  int32_t bp_rows;         // rows per warp in bp; row r holds frame t_begin + 1 + r
  int32_t ck_every;        // checkpoint interval in frames (0: none)
  int32_t ck_stride;       // floats between checkpoint rows
  uint32_t flags;
  int32_t zstride;         // bytes per anchor row (multiple of 16, >= S)
  uint8_t* ztab;           // anchor rows: row m holds s - anchor(s) at the end of window m
  uint64_t* xlink;         // grid teams: links between consecutive CTAs (zeroed before launch)
  float* lse;              // logits mode: per-frame log_softmax shift [T] (written by the lse pre-pass)
  int32_t team_ctas;       // persistent launches: CTAs of this job's team
  int32_t first_seat;      // persistent launches: the team's first seat (rank 0)
};

struct FwdParams {
  int32_t rb;              // boundary ring slots per warp (power of two, >= 2*block + 2)
  int32_t block;           // frames per ring wait / progress publication (<= 32)
  int32_t frames_per_stage;
  int32_t stage_bytes;     // bytes per emission stage (16-byte multiple)
  int32_t off_ring;        // shared-memory offsets
  int32_t off_stage;
  int32_t off_lse;         // end of the stage ring and its spare row
  int32_t off_bt;
  int32_t stages;          // emission stages in the ring (kLead .. kMaxStages)
  int32_t grid_ctas;       // 0: a team is one thread-block cluster; > 0: CTAs per grid team
  int32_t norm;            // 1: log_probs hold raw logits (shifts from the lse pre-pass in J.lse)
  // Fast kernel (LaunchShape::fast): neighbour hand-off in packages of kb frames.
  int32_t kb;              // frames per package (4 or 8)
  int32_t pkgs;            // package slots per shared-memory link (power of two)
  int32_t gpkgs;           // package slots per global link of a grid team (power of two)
  int32_t link_off;        // shared-memory offset of the per-warp links
  int32_t link_stride;     // bytes per warp link: 16-byte head + pkgs * kb * 8
  int32_t row_c;           // 32: every job of the launch has 32 classes and whole-window
                           // hand-offs (rows at compile-time offsets); else 0
  uint64_t wait_limit_ns;  // limit of every spin wait
};

// Result codes written to FwdJob::status (same values as align.h).
constexpr int32_t kStOk = 0;
constexpr int32_t kStPending = 1;
constexpr int32_t kStNoPath = -6;
constexpr int32_t kStTimeout = -7;
constexpr int32_t kStBadLaunch = -8;  // launch parameters do not fit the job (reported as ALIGN_E_CUDA)

// Host-side launch entry points (defined in trellis_kernels.cu).
struct LaunchShape {
  int K;                   // states per lane
  int warps;               // warps per CTA
  int ncta;                // CTAs per cluster (1: no cluster)
  int occ = 0;             // 1: build with fewer registers per thread (K <= 4) for more
                           // resident warps, for batches that oversubscribe the GPU
  int grid = 0;            // 1: the team is ncta CTAs of one cooperative launch, one per SM,
                           // linked through global memory (transcripts beyond a cluster)
  int norm = 0;            // 1: inputs are raw logits: an lse pre-pass runs before the launch
  int sum = 0;             // 1: sum-product forward score only (log-add in place of max)
  int fast = 0;            // 1: the fast Viterbi kernel (K = 2 or 4, at least 4 frames per stage)
  int persist = 0;         // 1: a job of a persistent launch (teams of any CTAs, global links)
};

// Bytes of the global links of a grid team of ncta CTAs: a ring of kMaxRing
// words per CTA boundary, one progress word per CTA and a 2-word barrier.
constexpr int kMaxRing = 128;  // ring slots per boundary, at least P.rb
inline uint64_t xlink_bytes(int ncta) {
  const uint64_t b = static_cast<uint64_t>(ncta > 1 ? ncta - 1 : 0) * kMaxRing * 8ull +
                     static_cast<uint64_t>((ncta + 3) & ~3) * 4ull + 16ull;
  return (b + 255) & ~255ull;
}

// Fast kernel: package slots per link, and the bytes of a grid team's global
// links (one per CTA boundary: 16-byte head + slots of kb alphas and kb
// anchors) followed by the team block (barrier, final alphas, timeout flag).
constexpr int kFastPkgs = 8;       // packages of 4 frames per shared-memory link
constexpr int kFastGridPkgs = 16;  // packages of 4 frames per global link
constexpr int kFastWinPkgs = 4;    // 32-frame windows per shared-memory link (window mode)
constexpr int kFastWinGridPkgs = 8;  // 32-frame windows per global link (window mode)
inline uint64_t fast_xlink_bytes(int ncta, int kb) {
  const uint64_t slots = (kb == 32) ? kFastWinGridPkgs : kFastGridPkgs;
  const uint64_t gstride = 16ull + slots * kb * 8ull;
  // After the links, the team block: barrier count and generation, the two
  // final alphas, the team's timeout flag.
  const uint64_t b = static_cast<uint64_t>(ncta > 1 ? ncta - 1 : 0) * gstride + 32ull;
  return (b + 255) & ~255ull;
}

// Number of 32-bit backpointer words per warp and frame.
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int bp_words(int K) { return 3 * K / 2; }

// Shared-memory plan for a launch shape and vocabulary size.
FwdParams plan_params(const LaunchShape& shape, int C, int frames_per_stage, uint64_t wait_limit_ns);
int smem_bytes(const LaunchShape& shape, const FwdParams& p);

// Launch the fused forward (+ backtrack) kernel over njobs jobs, one cluster
// (or CTA) per job, on the given stream. Returns a cudaError_t value.
int launch_trellis(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs,
                   void* stream);

// The fast Viterbi kernel (trellis_fast.cu) for shapes with fast = 1.
int launch_trellis_fast(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs, int njobs, void* stream);

// One persistent launch over the jobs of a batch planned with one shape
// (trellis_fast.cu): `ctas` resident CTAs take the `total_seats` seats in
// order from *d_counter (zero before the launch); seat x is job
// d_seat_job[x]. Every job's rows must be 16-byte aligned.
int launch_trellis_persist(const LaunchShape& shape, const FwdParams& p, const FwdJob* d_jobs,
                           const int32_t* d_seat_job, int32_t total_seats, int32_t* d_counter, int ctas,
                           void* stream);
// The most CTAs of that shape that are resident at once on the device.
int persist_max_ctas(const LaunchShape& shape, const FwdParams& p, int device, int* ctas);

// Null-work frame-latency probe (warp-scope chain of one frame); d_out[0] =
// ns for `frames` frames measured by CTA 0, d_out[1] = 0.
int launch_frame_probe(int warps, int ncta, int frames, uint64_t limit_ns, uint64_t* d_out, void* stream);

// Largest dynamic shared memory the kernel for this shape may use.
int max_smem_optin(int device);

// One piece of a batched host <-> device copy (copy_kernels.cu): both
// addresses must be addressable by the device.
struct alignas(16) CopyChunk {
  const void* src;
  void* dst;
  uint64_t bytes;
  uint64_t pad;
};
constexpr uint64_t kCopyChunk = 256ull << 10;  // bytes per chunk at most
int launch_copy_chunks(const CopyChunk* d_chunks, int n, int sm_count, void* stream);
// *d_flag = 1 when one of the n floats at p is NaN or +inf, else 0 (asynchronous).
int launch_scan_nonfinite(const float* p, int64_t n, int32_t* d_flag, int sm_count, void* stream);

}  // namespace gb300_align
