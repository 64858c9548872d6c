// Allocation-free alignment entry point (align_forced_noalloc).
//
// Some callers cannot allocate device memory at the moment they need an
// alignment: a real-time audio thread for which cudaMalloc's possible
// device-wide synchronisation is not acceptable, or a host application that
// hands the library a fixed device-memory budget up front and forbids any
// later growth. For them this entry point runs the same trellis kernel as
// align_submit, but every piece of scratch it needs (job descriptor, status
// words, device copy of the targets, backpointers and anchor rows) lives in
// one file-scope device array of fixed size compiled into the library. The
// caller still provides the inputs and the outputs.
//
// Rules of use:
//   * the library holds kNoAllocScratchBytes (32 MiB) of device memory on
//     every GPU where it is loaded, until the process exits;
//   * the first call on a device looks up the array's device address (once,
//     with that device current). Under CUDA's lazy module loading that first
//     call is also where the library's device code and this array are loaded
//     onto the device, which allocates and may synchronise: make the first call
//     outside the allocation-sensitive path, and before any stream capture on
//     the device;
//   * every call uses the same array, which keeps the previous call's
//     contents: calls that overlap on the GPU (different streams, or several
//     host threads) race and must not be issued; the call synchronises its
//     stream before returning, so back-to-back calls from one thread are safe;
//   * requests whose scratch exceeds the array are rejected with
//     ALIGN_E_TOO_LARGE and a message in align_last_error.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/align.h"
#include "align_internal.h"
#include "trellis.cuh"

namespace gb300_align {
namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

// The scratch area. In host code this name is only a stand-in for the symbol:
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
thread_local char g_msg[256];

int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return ALIGN_E_INVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[device] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // `device` is current here
    if (e != cudaSuccess || p == nullptr) {
      std::snprintf(g_msg, sizeof(g_msg), "align_forced_noalloc: cudaGetSymbolAddress failed: %s",
                    cudaGetErrorString(e));
      return ALIGN_E_CUDA;
    }
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return ALIGN_OK;
}

inline uint64_t up256(uint64_t v) { return (v + 255) / 256 * 256; }

// Per-request metadata block (same layout as the runtime's: status, chase
// state, alpha of the two final states).
struct Meta {
  int32_t status;
  int32_t state_io;
  float final2[2];
};
static_assert(sizeof(Meta) == 16, "metadata block layout");

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

// A device (or managed) buffer on `device`; a host pointer given to the kernel
// would fault on the GPU instead of returning an error.
bool on_device(const void* p, int device) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace
}  // namespace gb300_align

using namespace gb300_align;

extern "C" const char* align_noalloc_last_error(void) { return g_msg; }

extern "C" int align_forced_noalloc(const float* log_probs, int64_t T, int64_t C, const int32_t* targets, int64_t L,
                                    int32_t blank, align_out out, void* cuda_stream, int32_t* request_status) {
  g_msg[0] = '\0';
  if (!log_probs || !out.path || !out.scores || !out.total || (L > 0 && !targets))
    return fail(ALIGN_E_INVAL, "align_forced_noalloc: a required pointer is NULL");
  {
    // The call copies from host memory and synchronises its stream, which a
    // stream capture cannot record: refused before any other CUDA call.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cs) != cudaSuccess) {
      (void)cudaGetLastError();
    } else if (cs != cudaStreamCaptureStatusNone) {
      return fail(ALIGN_E_INVAL, "align_forced_noalloc: the stream is being captured");
    }
  }
  int64_t R = 0;
  int rc = validate_request(targets, L, C, blank, T, &R);
  if (rc != ALIGN_OK)
    return fail(rc, "align_forced_noalloc: request rejected by validation (%s)", align_status_string(rc));
  if (T >= (1ll << kTagBits))
    return fail(ALIGN_E_TOO_LARGE, "align_forced_noalloc: T = %lld frames exceeds 2^%d - 1", static_cast<long long>(T),
                kTagBits);
  Plan p{};
  rc = make_plan(default_tune_table(), T, C, L, ~0ull, false, &p);
  if (rc != ALIGN_OK)
    return fail(rc, "align_forced_noalloc: transcript of %lld targets needs more than one thread-block cluster",
                static_cast<long long>(L));

  // Scratch layout: descriptor | metadata | targets | backpointers + anchor rows.
  const uint64_t off_job = 0;
  const uint64_t off_meta = up256(sizeof(FwdJob));
  const uint64_t off_tgt = off_meta + 256;
  const uint64_t off_bp = off_tgt + up256(static_cast<uint64_t>(L > 0 ? L : 1) * 4);
  const uint64_t need = off_bp + p.bp_bytes;
  if (need > kNoAllocScratchBytes)
    return fail(ALIGN_E_TOO_LARGE, "align_forced_noalloc: request needs %llu bytes of scratch, the fixed area holds %llu",
                static_cast<unsigned long long>(need), static_cast<unsigned long long>(kNoAllocScratchBytes));
  int device = 0;
  cudaError_t ge = cudaGetDevice(&device);
  if (ge != cudaSuccess) return fail(ALIGN_E_CUDA, "align_forced_noalloc: %s", cudaGetErrorString(ge));
  if (!on_device(log_probs, device) || !on_device(out.path, device) || !on_device(out.scores, device) ||
      !on_device(out.total, device) || (out.states && !on_device(out.states, device)))
    return fail(ALIGN_E_INVAL, "align_forced_noalloc: log_probs and outputs must be device memory of device %d",
                device);
  void* base_v = nullptr;
  rc = scratch_address(device, &base_v);
  if (rc != ALIGN_OK) return rc;
  unsigned char* base = static_cast<unsigned char*>(base_v);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  // Host images of the descriptor and the metadata (status must start pending).
  FwdJob j{};
  Meta m{kStPending, 0, {-INFINITY, -INFINITY}};
  Meta* dmeta = reinterpret_cast<Meta*>(base + off_meta);
  j.lp = log_probs;
  j.tgt = reinterpret_cast<const int32_t*>(base + off_tgt);
  j.bp = reinterpret_cast<uint32_t*>(base + off_bp);
  j.ztab = reinterpret_cast<uint8_t*>(base + off_bp + p.z_off);
  j.zstride = p.zstride;
  j.final2 = dmeta->final2;
  j.status = &dmeta->status;
  j.state_io = &dmeta->state_io;
  j.path = out.path;
  j.scores = out.scores;
  j.total = out.total;
  j.states = out.states;
  j.T = static_cast<int32_t>(T);
  j.C = static_cast<int32_t>(C);
  j.blank = blank;
  j.L = static_cast<int32_t>(L);
  j.S = static_cast<int32_t>(2 * L + 1);
  j.t_begin = 0;
  j.t_end = j.T;
  j.bp_rows = j.T - 1;
  j.flags = kJobWriteFinal | kJobChase | (rows_bulk_ok(log_probs, C) ? kJobBulkRows : 0u);

  cudaError_t e = cudaMemcpyAsync(base + off_job, &j, sizeof(j), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dmeta, &m, sizeof(m), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && L > 0)
    e = cudaMemcpyAsync(base + off_tgt, targets, static_cast<size_t>(L) * 4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) {
    const FwdParams prm = plan_params(p.shape, static_cast<int>(C), p.frames_per_stage, 2000000000ull);
    e = static_cast<cudaError_t>(
        launch_trellis(p.shape, prm, reinterpret_cast<const FwdJob*>(base + off_job), 1, stream));
  }
  int32_t st = kStPending;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, &dmeta->status, 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(ALIGN_E_CUDA, "align_forced_noalloc: %s", cudaGetErrorString(e));
  if (request_status) *request_status = (st == kStPending) ? ALIGN_E_TIMEOUT : st;
  return ALIGN_OK;
}
