// Level-0 MAS product of the BF16 form (Eq. 6 at level 0).
//
// The domain inverse is kept as its inverse Cholesky factor W = L^{-1}
// (M_d = L L^T, M_d^{-1} = W^T W), rounded to BF16, and applied as
// z_d = W^T (W r_d) with FP32 accumulation.  Rounding M_d^{-1} itself to
// BF16 (8 significant bits) makes it indefinite once a domain's condition
// number passes ~1e3, which stalls PCG; any rounding of W keeps W^T W
// positive semi-definite.
//
// Tensor-core kernel, one CTA per domain:
//   * one bulk asynchronous copy brings the domain's W (BF16, stored at build
//     time in the K-major operand layout) into shared memory;
//   * r_d is gathered and every FP32 value split into BF16 hi + lo parts
//     (hi = bf16(v), lo = bf16(v - hi): about 16 significant bits), the 16
//     columns of the B operand (8 RHS x {hi, lo});
//   * MMA 1: y = W [r_hi | r_lo], 3N/16 tcgen05.mma (M = 128 with the 3N = 96
//     rows padded, N = 16, K = 16), FP32 accumulation in TMEM columns 0..15;
//   * each warp reads its TMEM lanes, adds the hi and lo columns, splits y
//     again into hi + lo and writes the B operand of MMA 2;
//   * MMA 2: z = W^T [y_hi | y_lo] with the same shared-memory copy of W read
//     as an MN-major operand (the transposed A), TMEM columns 16..31;
//   * epilogue: z = hi + lo columns, plus the prolongated coarse results,
//     summed in FP32 (every level's product is FP32) with the FP64 <-> FP32
//     conversions done on bit patterns: on this part conversion
//     instructions run on the FP64 pipe, which otherwise bounds the kernel.
// All waits are bounded; on a timeout the kernel sets kErrTimeout, skips the
// rest and still frees its TMEM.
//
// FP32-core kernel (nrhs > 8, 3N not a multiple of 16, or chosen by the
// tuner): the same two triangular products from shared memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "primitives.cuh"
#include "umma.cuh"

namespace gs {
namespace bf16f {

constexpr int kM = 128;  // MMA rows: domain rows padded
constexpr int kN = 16;   // MMA columns: high + low parts of 8 RHS
constexpr int kThreads = 128;

struct Levels {
  const int32_t* coarse[8];
  int64_t vec_off[8];
  int L;
};

// Shared-memory bytes the A operand spans: as K-major W (rows padded to
// 128 within each K group) and as MN-major W^T (rows of W^T padded to 128).
__host__ __device__ inline uint32_t a_span(int ld) {
  const uint32_t k_major = (uint32_t)(ld * ld * 2 - ld * 16 + kM * 16);
  const uint32_t mn_major = (uint32_t)(kM / 8) * ld * 16;
  return k_major > mn_major ? k_major : mn_major;
}
__host__ __device__ inline uint32_t b_bytes(int ld) { return (uint32_t)(ld / 8) * 256; }
__host__ __device__ inline uint32_t round128(uint32_t x) { return (x + 127u) & ~127u; }

// B operand element (n, kk), K-major: (kk/8)*256 + (n/8)*128 + (n%8)*16 + (kk%8)*2.
__device__ __forceinline__ void put_hi_lo(unsigned char* sB, int kk, int k, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  unsigned char* col = sB + (kk >> 3) * 256 + (kk & 7) * 2;
  *(__nv_bfloat16*)(col + k * 16) = hi;        // n = k
  *(__nv_bfloat16*)(col + 128 + k * 16) = lo;  // n = 8 + k
}

// Gathered right-hand side value (node-major FP32 or RHS-major FP64).
template <bool kF32>
__device__ __forceinline__ float load_r(const void* rv, int64_t stride, int nrhs, int32_t node, int k, int c) {
  if (kF32) return ((const float*)rv)[((int64_t)node * nrhs + k) * 3 + c];
  return f64_to_f32_bits(((const double*)rv)[k * stride + 3 * (int64_t)node + c]);
}

// z at (node, c) for RHS 0..nrhs-1: level-0 value plus the coarse levels.
template <bool kF32>
__device__ __forceinline__ void store_z(const Levels& al, const void* zlv, int64_t lstride, void* zv, int64_t stride,
                                        int nrhs, int32_t node, int c, const float* v) {
  int64_t citem[8];
#pragma unroll
  for (int l = 1; l < 8; ++l) citem[l] = l < al.L ? al.vec_off[l] + al.coarse[l][node] : 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k >= nrhs) break;
    if (kF32) {
      float w = v[k];
#pragma unroll
      for (int l = 1; l < 8; ++l)
        if (l < al.L) w += ((const float*)zlv)[(citem[l] * nrhs + k) * 3 + c];
      ((float*)zv)[((int64_t)node * nrhs + k) * 3 + c] = w;
    } else {  // the sum in FP32, the precision of every level's product; conversions from bit patterns
      float w = v[k];
#pragma unroll
      for (int l = 1; l < 8; ++l)
        if (l < al.L) w += f64_to_f32_bits(((const double*)zlv)[k * lstride + 3 * citem[l] + c]);
      ((double*)zv)[k * stride + 3 * (int64_t)node + c] = f32_to_f64_bits(w);
    }
  }
}

template <bool kF32>
__global__ void __launch_bounds__(kThreads) k_level0_tc(const __nv_bfloat16* __restrict__ W,
                                                        const int32_t* __restrict__ remap0, int N, int nrhs,
                                                        Levels al, const void* __restrict__ rv, int64_t stride,
                                                        const void* __restrict__ zlv, int64_t lstride,
                                                        void* __restrict__ zv, const int* __restrict__ skip,
                                                        int* __restrict__ flags) {
  using namespace umma;
  if (skip && *skip) return;
  extern __shared__ unsigned char smem_raw[];
  const int ld = 3 * N;
  const uint32_t a_bytes = (uint32_t)ld * ld * 2;
  const uint32_t span = a_span(ld);
  unsigned char* sA = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* sB = sA + round128(span);
  uint64_t* bars = (uint64_t*)(sB + b_bytes(ld));  // [0] copy, [1] MMA 1, [2] MMA 2
  uint32_t* tslot = (uint32_t*)(bars + 3);
  int* sfail = (int*)(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t d = blockIdx.x;
  const uint32_t idesc1 = idesc_bf16_f32(kM, kN);               // A = W, K-major
  const uint32_t idesc2 = idesc_bf16_f32(kM, kN) | (1u << 15);  // A = W^T, MN-major
  const uint32_t lbo_a = (uint32_t)ld * 16;                      // between 8-row groups of W

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    *sfail = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 32);
    tmem_relinquish();
  }
  // the padding rows the M = 128 operand reads past the domain: zero them
  for (uint32_t e = a_bytes + 16u * tid; e < span; e += 16u * kThreads) *(uint4*)(sA + e) = make_uint4(0, 0, 0, 0);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], a_bytes);
    bulk_g2s(sA, W + (int64_t)d * ld * ld, a_bytes, &bars[0]);
  }
  for (int e = tid; e < 8 * ld; e += kThreads) {
    const int k = e / ld, kk = e - k * ld;
    float v = 0.0f;
    if (k < nrhs) {
      const int32_t node = remap0[(int64_t)d * N + kk / 3];
      if (node >= 0) v = load_r<kF32>(rv, stride, nrhs, node, k, kk % 3);
    }
    put_hi_lo(sB, kk, k, v);
  }
  fence_proxy_async();
  __syncthreads();
  const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
  if (tid == 0) {
    if (mbar_wait(&bars[0], 0)) {
      fence_after_sync();
      for (int s = 0; s < ld / 16; ++s)
        mma_bf16(tmem, smem_desc(a0 + 2u * s * lbo_a, lbo_a, 128), smem_desc(b0 + 512u * s, 256, 128), idesc1,
                 s > 0 ? 1u : 0u);
      mma_commit(&bars[1]);
    } else {
      *sfail = 1;
      atomicOr(flags, kErrTimeout);
      mbar_wait(&bars[0], 0);  // let a late copy land before the CTA leaves
      mbar_arrive(&bars[1]);
    }
  }
  __syncwarp();
  bool ok = mbar_wait(&bars[1], 0);
  if (!ok) atomicOr(flags, kErrTimeout);
  ok = __all_sync(0xffffffffu, ok) && !*sfail;
  fence_after_sync();
  // y = hi + lo columns -> split again -> B operand of MMA 2 (the buffer of MMA 1 is free now)
  if (ok && warp * 32 < ld) {
    float acc[16];
    tmem_ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16), acc);
    const int i = warp * 32 + lane;
    if (i < ld) {
#pragma unroll
      for (int k = 0; k < 8; ++k) put_hi_lo(sB, i, k, acc[k] + acc[8 + k]);
    }
  }
  if (!ok) *sfail = 1;
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (tid == 0) {
    if (!*sfail) {
      // W^T as an MN-major operand: 8-element runs along M (columns of W) are
      // contiguous; without swizzling the descriptor's leading offset is the
      // K-direction step between core matrices (128 bytes) and its stride
      // offset the M-direction step (ld*16 bytes), as for K-major operands
      for (int s = 0; s < ld / 16; ++s)
        mma_bf16(tmem + 16, smem_desc(a0 + 256u * s, 128, lbo_a), smem_desc(b0 + 512u * s, 256, 128), idesc2,
                 s > 0 ? 1u : 0u);
      mma_commit(&bars[2]);
    } else {
      mbar_arrive(&bars[2]);
    }
  }
  __syncwarp();
  bool ok2 = mbar_wait(&bars[2], 0);
  if (!ok2) atomicOr(flags, kErrTimeout);
  ok2 = __all_sync(0xffffffffu, ok2) && !*sfail;
  fence_after_sync();
  if (ok2 && warp * 32 < ld) {
    float acc[16];
    tmem_ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16) + 16, acc);
    const int i = warp * 32 + lane;
    const int32_t node = i < ld ? remap0[(int64_t)d * N + i / 3] : -1;
    if (node >= 0) {
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = acc[k] + acc[8 + k];
      store_z<kF32>(al, zlv, lstride, zv, stride, nrhs, node, i % 3, v);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, 32);
  }
}

// FP32-core form: thread (row i, group of 4 RHS); W (row-major BF16) and the
// vectors in shared memory; pass 1 y = W r (row i of W), pass 2 z = W^T y
// (column i of W).  Row stride ld + 2 keeps pass 1 free of bank conflicts.
constexpr int kCoreRpt = 4;

template <bool kF32>
__global__ void __launch_bounds__(768) k_level0_cores(const __nv_bfloat16* __restrict__ W,
                                                      const int32_t* __restrict__ remap0, int N, int nrhs, Levels al,
                                                      const void* __restrict__ rv, int64_t stride,
                                                      const void* __restrict__ zlv, int64_t lstride,
                                                      void* __restrict__ zv, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ unsigned char smem_raw[];
  const int ld = 3 * N, S = ld + 2;
  __nv_bfloat16* sW = (__nv_bfloat16*)smem_raw;
  float* sr = (float*)(smem_raw + ((size_t)ld * S * 2 + 15) / 16 * 16);
  float* sy = sr + ld * nrhs;
  const int32_t d = blockIdx.x;
  const int tid = threadIdx.x;
  const __nv_bfloat16* Wd = W + (int64_t)d * ld * ld;
  for (int e = tid; e < ld * ld; e += blockDim.x) sW[(e / ld) * S + e % ld] = Wd[e];
  for (int e = tid; e < ld * nrhs; e += blockDim.x) {
    const int j = e / nrhs, k = e % nrhs;
    const int32_t node = remap0[(int64_t)d * N + j / 3];
    sr[e] = node >= 0 ? load_r<kF32>(rv, stride, nrhs, node, k, j % 3) : 0.0f;
  }
  __syncthreads();
  const int i = tid % ld, g = tid / ld, k0 = g * kCoreRpt;
  const bool act = k0 < nrhs;
  float acc[kCoreRpt];
  if (act) {
#pragma unroll
    for (int q = 0; q < kCoreRpt; ++q) acc[q] = 0.0f;
    for (int j = 0; j <= i; ++j) {
      const float w = __bfloat162float(sW[i * S + j]);
#pragma unroll
      for (int q = 0; q < kCoreRpt; ++q)
        if (k0 + q < nrhs) acc[q] = fmaf(w, sr[j * nrhs + k0 + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kCoreRpt; ++q)
      if (k0 + q < nrhs) sy[i * nrhs + k0 + q] = acc[q];
  }
  __syncthreads();
  if (!act) return;
#pragma unroll
  for (int q = 0; q < kCoreRpt; ++q) acc[q] = 0.0f;
  for (int j = i; j < ld; ++j) {
    const float w = __bfloat162float(sW[j * S + i]);
#pragma unroll
    for (int q = 0; q < kCoreRpt; ++q)
      if (k0 + q < nrhs) acc[q] = fmaf(w, sy[j * nrhs + k0 + q], acc[q]);
  }
  const int32_t node = remap0[(int64_t)d * N + i / 3];
  if (node < 0) return;
  const int c = i % 3;
#pragma unroll
  for (int q = 0; q < kCoreRpt; ++q) {
    const int k = k0 + q;
    if (k >= nrhs) break;
    if (kF32) {
      float w = acc[q];
      for (int l = 1; l < al.L; ++l)
        w += ((const float*)zlv)[((al.vec_off[l] + al.coarse[l][node]) * nrhs + k) * 3 + c];
      ((float*)zv)[((int64_t)node * nrhs + k) * 3 + c] = w;
    } else {
      float w = acc[q];
      for (int l = 1; l < al.L; ++l)
        w += f64_to_f32_bits(((const double*)zlv)[k * lstride + 3 * (al.vec_off[l] + al.coarse[l][node]) + c]);
      ((double*)zv)[k * stride + 3 * (int64_t)node + c] = f32_to_f64_bits(w);
    }
  }
}

// double -> float -> bfloat16 (both to nearest even) of the row-major FP64
// factor W, written in the K-major operand layout: per domain
// [k/8][i/8][i%8][k%8] with A[i][k] = W[i][k].
__global__ void k_to_bf16_tc(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n_dom, int ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)ld * ld;
  if (e >= n_dom * per) return;
  const int64_t dom = e / per;
  const int rem = (int)(e - dom * per);
  const int k8 = rem & 7, r8 = (rem >> 3) & 7, t = rem >> 6;
  const int groups = ld / 8;
  const int i = (t % groups) * 8 + r8, k = (t / groups) * 8 + k8;
  b[e] = __float2bfloat16_rn((float)a[dom * per + (int64_t)i * ld + k]);
}

}  // namespace bf16f

bool level0_bf16_on_tensor_cores(gs_ctx ctx, gs_mas mas, int nrhs) {
  return mas->precision == GS_PREC_BF16 && mas->inv16_tc != nullptr && nrhs >= 1 && nrhs <= 8 &&
         ctx->tune[GS_TUNE_BF16_TC] != 0;
}

int level0_bf16_prepare(gs_ctx ctx, gs_mas mas, const double* fac0) {
  const int ld = 3 * mas->N;
  if (ld % 16 != 0 || ld > bf16f::kM || mas->inv16_tc) return GS_OK;
  const int64_t cnt = (int64_t)mas->n_domains[0] * ld * ld;
  GS_TRY(ctx->alloc(&mas->inv16_tc, (size_t)std::max<int64_t>(cnt, 1) * 2));
  if (cnt) {
    GS_PROF(ctx, GS_K_MAS_INVERT);
    bf16f::k_to_bf16_tc<<<ceil_div(cnt, 256), 256, 0, ctx->stream>>>(fac0, (__nv_bfloat16*)mas->inv16_tc,
                                                                      mas->n_domains[0], ld);
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

int level0_bf16_launch(gs_ctx ctx, gs_mas mas, bool f32_node_major, int nrhs, const void* r, int64_t stride,
                       const void* zl, int64_t lstride, void* z, const int* skip, int* flags) {
  GS_CHECK(mas->precision == GS_PREC_BF16 && !mas->inv16.empty(), GS_ERR_INVALID, "level-0 BF16 apply: no factors");
  if (mas->n_domains[0] == 0) return GS_OK;
  const int ld = 3 * mas->N;
  bf16f::Levels al{};
  al.L = mas->L;
  for (int l = 0; l < mas->L; ++l) al.coarse[l] = mas->coarse[l], al.vec_off[l] = mas->vec_off[l];
  cudaStream_t st = ctx->stream;
  if (level0_bf16_on_tensor_cores(ctx, mas, nrhs)) {
    const size_t smem = 128 + bf16f::round128(bf16f::a_span(ld)) + bf16f::b_bytes(ld) + 3 * 8 + 8;
    if (f32_node_major)
      bf16f::k_level0_tc<true><<<mas->n_domains[0], bf16f::kThreads, smem, st>>>(
          (const __nv_bfloat16*)mas->inv16_tc, mas->remap0, mas->N, nrhs, al, r, stride, zl, lstride, z, skip, flags);
    else
      bf16f::k_level0_tc<false><<<mas->n_domains[0], bf16f::kThreads, smem, st>>>(
          (const __nv_bfloat16*)mas->inv16_tc, mas->remap0, mas->N, nrhs, al, r, stride, zl, lstride, z, skip, flags);
  } else {
    const int threads = ((ld * ceil_div(nrhs, bf16f::kCoreRpt) + 31) / 32) * 32;
    GS_CHECK(threads <= 768, GS_ERR_UNSUPPORTED, "level-0 BF16 apply: too many right-hand sides (%d)", nrhs);
    const size_t smem = ((size_t)ld * (ld + 2) * 2 + 15) / 16 * 16 + 2 * (size_t)ld * nrhs * 4;
    if (smem > 48 * 1024) {
      GS_CUDA(cudaFuncSetAttribute(bf16f::k_level0_cores<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
      GS_CUDA(cudaFuncSetAttribute(bf16f::k_level0_cores<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    }
    if (f32_node_major)
      bf16f::k_level0_cores<true><<<mas->n_domains[0], threads, smem, st>>>(
          (const __nv_bfloat16*)mas->inv16[0], mas->remap0, mas->N, nrhs, al, r, stride, zl, lstride, z, skip);
    else
      bf16f::k_level0_cores<false><<<mas->n_domains[0], threads, smem, st>>>(
          (const __nv_bfloat16*)mas->inv16[0], mas->remap0, mas->N, nrhs, al, r, stride, zl, lstride, z, skip);
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs
