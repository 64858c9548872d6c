// Token spans of packed alignments. Transcript token i of an utterance
// occupies the frames whose trellis state is 2i + 1 (consecutive on a valid
// CTC path): its span is [first such frame, last + 1) and its score the FP32
// left-fold sum of those frames' scores divided by the span length (paper
// Sec. 4: forced alignment produces the alignment between audio frames and
// transcript tokens; this is that alignment per token).
//
// Pass 1, one thread per frame: a frame whose state differs from its left
// neighbour starts a span, one that differs from its right neighbour ends it.
// Pass 2, one thread per token: the sequential fold over the span's frames
// (spans are a few frames long), then one IEEE division.
#include <cstdint>

#include <cuda_runtime.h>

#include "align.h"
#include "trellis.cuh"

namespace gb300_align {
namespace {

// The segment u with off[u] <= x < off[u + 1] (off[0] = 0; empty segments
// are skipped: the largest such u).
__device__ __forceinline__ int find_segment(const int64_t* __restrict__ off, int n, int64_t x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256) span_bounds_kernel(const int32_t* __restrict__ states,
                                                          const int64_t* __restrict__ foff,
                                                          const int64_t* __restrict__ toff, int n, int64_t total_T,
                                                          int32_t* __restrict__ start, int32_t* __restrict__ end) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total_T; g += stride) {
    const int32_t st = states[g];
    if (!(st & 1)) continue;  // blank states belong to no token
    const int u = find_segment(foff, n, g);
    const int64_t f0 = __ldg(foff + u), f1 = __ldg(foff + u + 1);
    const int64_t tok = __ldg(toff + u) + (st >> 1);
    if (st < 0 || tok >= __ldg(toff + u + 1)) continue;  // not a state of this transcript
    if (g == f0 || states[g - 1] != st) start[tok] = static_cast<int32_t>(g - f0);
    if (g + 1 == f1 || states[g + 1] != st) end[tok] = static_cast<int32_t>(g + 1 - f0);
  }
}

__global__ void __launch_bounds__(256) span_scores_kernel(const float* __restrict__ scores,
                                                          const int64_t* __restrict__ foff,
                                                          const int64_t* __restrict__ toff, int n, int64_t total_L,
                                                          int32_t* __restrict__ start, int32_t* __restrict__ end,
                                                          float* __restrict__ score) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < total_L; k += stride) {
    const int32_t s = start[k], e = end[k];
    if (s < 0 || e <= s) {  // a token without frames (not a valid alignment)
      start[k] = -1;
      end[k] = -1;
      score[k] = 0.0f;
      continue;
    }
    const int u = find_segment(toff, n, k);
    const float* p = scores + __ldg(foff + u);
    float acc = 0.0f;
    for (int32_t t = s; t < e; ++t) acc = __fadd_rn(acc, p[t]);
    score[k] = __fdiv_rn(acc, static_cast<float>(e - s));
  }
}

}  // namespace
}  // namespace gb300_align

using namespace gb300_align;

extern "C" int align_token_spans(const int32_t* states, const float* scores, const int64_t* frame_offsets,
                                 const int64_t* token_offsets, int32_t n, int64_t total_frames, int64_t total_tokens,
                                 int32_t* span_start, int32_t* span_end, float* span_score, void* cuda_stream) {
  if (n < 0 || total_frames < 0 || total_tokens < 0) return ALIGN_E_INVAL;
  if (n == 0 || total_tokens == 0) return ALIGN_OK;
  if (!states || !scores || !frame_offsets || !token_offsets || !span_start || !span_end || !span_score)
    return ALIGN_E_INVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ALIGN_E_CUDA;
  // Tokens without frames keep -1 (all bytes 0xff).
  if (cudaMemsetAsync(span_start, 0xff, static_cast<size_t>(total_tokens) * 4, s) != cudaSuccess ||
      cudaMemsetAsync(span_end, 0xff, static_cast<size_t>(total_tokens) * 4, s) != cudaSuccess)
    return ALIGN_E_CUDA;
  const auto grid = [&](int64_t items) {
    const int64_t b = (items + 255) / 256;
    return static_cast<unsigned>(b < 8ll * sms ? (b > 0 ? b : 1) : 8ll * sms);
  };
  if (total_frames > 0)
    span_bounds_kernel<<<grid(total_frames), 256, 0, s>>>(states, frame_offsets, token_offsets, n, total_frames,
                                                          span_start, span_end);
  span_scores_kernel<<<grid(total_tokens), 256, 0, s>>>(scores, frame_offsets, token_offsets, n, total_tokens,
                                                        span_start, span_end, span_score);
  return cudaGetLastError() == cudaSuccess ? ALIGN_OK : ALIGN_E_CUDA;
}
