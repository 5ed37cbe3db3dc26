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

// Conversions between FP64 and FP32 from the bit patterns.  On this part the
// conversion instructions run on the FP64 pipe (2 per clock per SM); these use
// integer instructions only.
// double -> float rounded to nearest (ties away from zero); a value below the
// float normal range becomes a signed zero, one above it infinity.
__device__ __forceinline__ float f64_to_f32_bits(double v) {
  const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
  const unsigned sign = hw & 0x80000000u;
  const int ef = (int)((hw >> 20) & 0x7ffu);
  const int fe = ef - 896;  // float exponent field (biases 1023 and 127)
  if (ef == 0 || fe <= 0) return __uint_as_float(sign);
  if (ef == 0x7ff || fe >= 255) return __uint_as_float(sign | 0x7f800000u | (ef == 0x7ff && ((hw & 0xfffffu) | lw) ? 0x400000u : 0u));
  const unsigned bits = sign | ((unsigned)fe << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
  return __uint_as_float(bits + ((lw >> 28) & 1u));  // a carry into the exponent rounds up exactly
}
// float -> double, exact; a subnormal float (below 2^-126) becomes a signed zero.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned fe = (b >> 23) & 0xffu;
  if (fe == 0) return __hiloint2double((int)(b & 0x80000000u), 0);
  const unsigned de = fe == 0xffu ? 0x7ffu : fe + 896u;
  return __hiloint2double((int)((b & 0x80000000u) | (de << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
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

// Addresses of the multilevel restricted vectors: value v = 3 k + c (RHS k,
// component c) of item `item` of one level.  RHS-major (FP64 apply):
// rl[k * lstride + 3 (off + item) + c]; node-major (FP32 inner solve):
// rl[(off + item) * nv + v].
struct LevelIdxRhsMajor {
  int64_t lstride, off;
  __device__ __forceinline__ int64_t operator()(int64_t item, int v) const {
    return (int64_t)(v / 3) * lstride + 3 * (off + item) + v % 3;
  }
};
struct LevelIdxNodeMajor {
  int64_t off;
  int nv;
  __device__ __forceinline__ int64_t operator()(int64_t item, int v) const { return (off + item) * nv + v; }
};

// Restriction from level l >= 1 to level l + 1 (supplement Eq. 5-6, C_{l+1}
// = C'_l C_l).  A level-(l+1) item is a connected component of one level-l
// domain (items dN .. dN+N-1), so one warp per level-l domain sums the
// values of each parent's items in ascending lane order and stores the total:
// every parent has one writer and a fixed order of addition, so the result
// does not depend on scheduling.  up[a]: the parent of item a (-1: none).
// Lanes own values v = lane, lane + 32, ... < nv; a lane first loads its
// value of all 32 items (independent loads, one round trip), then sums each
// parent's members from registers.  The parents' member masks come from
// __match_any_sync and are shared through shared memory.
template <typename T, typename Idx>
__global__ void __launch_bounds__(128) k_restrict_up(const int32_t* __restrict__ up, int32_t n_dom, int N, int nv,
                                                     Idx src, Idx dst, T* __restrict__ rl,
                                                     const int* __restrict__ skip) {
  if (skip && *skip) return;  // every RHS of the solve has converged
  __shared__ uint32_t gmask[4][32];
  __shared__ int32_t gpar[4][32];
  const int w = threadIdx.x >> 5;
  const int32_t d = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (d >= n_dom) return;  // whole warp
  const int32_t par = lane < N ? up[(int64_t)d * N + lane] : -1;
  const uint32_t realm = __ballot_sync(kFull, par >= 0);
  const uint32_t same = __match_any_sync(kFull, par);
  const bool leader = par >= 0 && lane == __ffs(same) - 1;
  const uint32_t leaders = __ballot_sync(kFull, leader);
  if (leader) {
    const int slot = __popc(leaders & ((1u << lane) - 1u));
    gmask[w][slot] = same;
    gpar[w][slot] = par;
  }
  __syncwarp();
  const int ng = __popc(leaders);
  for (int v = lane; v < nv; v += 32) {
    T val[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) val[j] = ((realm >> j) & 1u) ? rl[src((int64_t)d * N + j, v)] : (T)0;
    for (int g = 0; g < ng; ++g) {
      const uint32_t m = gmask[w][g];
      T sum = (T)0;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if ((m >> j) & 1u) sum += val[j];
      rl[dst(gpar[w][g], v)] = sum;
    }
  }
}

}  // namespace gs
