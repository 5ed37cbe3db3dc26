// Warp-level building blocks.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

constexpr unsigned kFull = 0xffffffffu;

// End (exclusive) of the segment that contains `lane`, given the warp's
// head mask (bit i set = lane i starts a segment; lane 0 always does).
__device__ __forceinline__ int segment_end(unsigned head_mask, int lane) {
  unsigned above = (lane == 31) ? 0u : (head_mask & (~0u << (lane + 1)));
  return above ? (__ffs(above) - 1) : 32;
}

// Head-segmented warp reduction (Sec. 5.2, HeadSegmentedReduce): after the
// call, every lane holds the sum of its own value and the values of the
// later lanes of its segment, so each head lane holds its segment's total.
// Suffix sums by doubling: with lane + o < seg_end the lane o places to the
// right lies in the same segment and holds a sum that stays inside it.
template <int K>
__device__ __forceinline__ void head_segmented_reduce(double (&v)[K], int lane, int seg_end) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const bool take = lane + o < seg_end;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = __shfl_down_sync(kFull, v[k], o);
      if (take) v[k] += t;
    }
  }
}

// Stored inverse entry -> arithmetic type (FP64, FP32 or BF16 storage).
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

}  // namespace gs
