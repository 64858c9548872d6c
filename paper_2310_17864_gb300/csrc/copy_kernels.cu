// Batched copies between host buffers the GPU can address (pinned and mapped,
// or system memory on a device with host page-table access) and device
// memory: one launch moves every host-buffer request's emissions in, or every
// request's outputs out, instead of one cudaMemcpyAsync per buffer. Each CTA
// takes whole chunks (at most kCopyChunk bytes); 16-byte vectors when source,
// destination and size allow, else 4-byte words, else bytes.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "trellis.cuh"

namespace gb300_align {
namespace {

__global__ void __launch_bounds__(256) copy_chunks_kernel(const CopyChunk* __restrict__ chunks, int n) {
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    const CopyChunk c = chunks[k];
    const uint64_t a = reinterpret_cast<uint64_t>(c.src) | reinterpret_cast<uint64_t>(c.dst) | c.bytes;
    if ((a & 15u) == 0) {
      const uint4* s = reinterpret_cast<const uint4*>(c.src);
      uint4* d = reinterpret_cast<uint4*>(c.dst);
      const uint64_t n16 = c.bytes / 16;
#pragma unroll 4
      for (uint64_t i = threadIdx.x; i < n16; i += blockDim.x) d[i] = s[i];
    } else if ((a & 3u) == 0) {
      const uint32_t* s = reinterpret_cast<const uint32_t*>(c.src);
      uint32_t* d = reinterpret_cast<uint32_t*>(c.dst);
      const uint64_t n4 = c.bytes / 4;
#pragma unroll 4
      for (uint64_t i = threadIdx.x; i < n4; i += blockDim.x) d[i] = s[i];
    } else {
      const unsigned char* s = reinterpret_cast<const unsigned char*>(c.src);
      unsigned char* d = reinterpret_cast<unsigned char*>(c.dst);
      for (uint64_t i = threadIdx.x; i < c.bytes; i += blockDim.x) d[i] = s[i];
    }
  }
}

}  // namespace

// Any NaN or +inf among n floats: *flag becomes 1 (-inf, log 0, is allowed).
__global__ void __launch_bounds__(256) scan_nonfinite_kernel(const float* __restrict__ p, int64_t n,
                                                             int32_t* __restrict__ flag) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float x = p[i];
    bad |= (x != x) || (x == INFINITY);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

int launch_scan_nonfinite(const float* p, int64_t n, int32_t* d_flag, int sm_count, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int32_t), st);
  if (e != cudaSuccess || n <= 0) return e;
  const int64_t want = (n + 255) / 256;
  const int grid = static_cast<int>(want < 4 * sm_count ? want : 4 * sm_count);
  scan_nonfinite_kernel<<<grid, 256, 0, st>>>(p, n, d_flag);
  return cudaGetLastError();
}

int launch_copy_chunks(const CopyChunk* d_chunks, int n, int sm_count, void* stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = n < 4 * sm_count ? n : 4 * sm_count;
  copy_chunks_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_chunks, n);
  return cudaGetLastError();
}

}  // namespace gb300_align
