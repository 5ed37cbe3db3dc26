// Level-0 MAS product on the tensor cores (Eq. 6 at level 0, BF16 inverses).
//
// Per level-0 domain d the product z_d = M_d^{-1} r_d is a dense
// (3N x 3N) . (3N x nrhs) contraction.  One CTA per domain:
//   * one bulk asynchronous copy brings the domain's BF16 inverse, stored at
//     build time in the tensor core's K-major operand layout, into shared
//     memory;
//   * the CTA gathers r_d, splits every FP32 value into a high and a low
//     BF16 part (hi = bf16(v), lo = bf16(v - hi); hi + lo keeps about 16
//     mantissa bits) and writes them as the B operand, columns 0..7 the high
//     parts of RHS 0..7 and columns 8..15 the low parts;
//   * one thread issues 3N/16 tcgen05.mma (M = 128, N = 16, K = 16; the
//     3N = 96 domain rows padded to 128), FP32 accumulation in TMEM;
//   * each warp reads its 32 TMEM lanes (rows), adds the high and low
//     columns, adds the prolongated coarse-level results and writes z.
// Both waits (copy, MMA) are bounded; on a timeout the kernel sets
// kErrTimeout, skips the epilogue and still frees its TMEM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "umma.cuh"

namespace gs {
namespace tc {

constexpr int kM = 128;  // MMA rows: domain rows padded
constexpr int kN = 16;   // MMA columns: high + low parts of 8 RHS
constexpr int kThreads = 128;

struct Levels {
  const int32_t* coarse[8];
  int64_t vec_off[8];
  int L;
};

// Shared-memory bytes the M = 128 A operand spans for a domain of ld rows:
// the domain's ld*ld BF16 values plus the rows 96..127 of the last K group.
__host__ __device__ inline uint32_t a_span(int ld) { return (uint32_t)(ld * ld * 2 - ld * 16 + kM * 16); }
__host__ __device__ inline uint32_t b_bytes(int ld) { return (uint32_t)(ld / 8) * 256; }
__host__ __device__ inline uint32_t round128(uint32_t x) { return (x + 127u) & ~127u; }

// kF32: vectors FP32 node-major [node][R][3] (mixed solve), else FP64
// RHS-major [k][3n] with strides `stride` (fine) and `lstride` (coarse).
template <bool kF32>
__global__ void __launch_bounds__(kThreads) k_level0_tc(const __nv_bfloat16* __restrict__ inv,
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
  uint64_t* bars = (uint64_t*)(sB + b_bytes(ld));  // [0] copy done, [1] MMAs done
  uint32_t* tslot = (uint32_t*)(bars + 2);
  int* sfail = (int*)(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t d = blockIdx.x;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    *sfail = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 32);
    tmem_relinquish();
  }
  // the rows 96..127 of the last K group lie past the domain: zero them
  for (uint32_t e = a_bytes + 16u * tid; e < span; e += 16u * kThreads) *(uint4*)(sA + e) = make_uint4(0, 0, 0, 0);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], a_bytes);
    bulk_g2s(sA, inv + (int64_t)d * ld * ld, a_bytes, &bars[0]);
  }
  // B operand, K-major: element (n, kk) at (kk/8)*256 + (n/8)*128 + (n%8)*16 + (kk%8)*2
  for (int e = tid; e < 8 * ld; e += kThreads) {
    const int k = e / ld, kk = e - k * ld;
    float v = 0.0f;
    if (k < nrhs) {
      const int32_t node = remap0[(int64_t)d * N + kk / 3];
      if (node >= 0) {
        const int c = kk % 3;
        if (kF32)
          v = ((const float*)rv)[((int64_t)node * nrhs + k) * 3 + c];
        else
          v = (float)((const double*)rv)[k * stride + 3 * (int64_t)node + c];
      }
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    unsigned char* col = sB + (kk >> 3) * 256 + (kk & 7) * 2;
    *(__nv_bfloat16*)(col + k * 16) = hi;             // n = k      (core matrix 0 along N)
    *(__nv_bfloat16*)(col + 128 + k * 16) = lo;       // n = 8 + k  (core matrix 1 along N)
  }
  fence_proxy_async();
  __syncthreads();
  if (tid == 0) {
    if (mbar_wait(&bars[0], 0)) {
      fence_after_sync();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      const uint32_t lbo_a = (uint32_t)ld * 16;  // next 8 columns of K: past all ld/8 row groups
      const uint32_t idesc = idesc_bf16_f32(kM, kN);
      for (int s = 0; s < ld / 16; ++s)
        mma_bf16(tmem, smem_desc(a0 + 2u * s * lbo_a, lbo_a, 128), smem_desc(b0 + 512u * s, 256, 128), idesc,
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
  if (ok && warp * 32 < ld) {
    float acc[16];
    tmem_ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16), acc);
    const int i = warp * 32 + lane;
    const int32_t node = i < ld ? remap0[(int64_t)d * N + i / 3] : -1;
    if (node >= 0) {
      const int c = i % 3;
      int64_t citem[8];  // item of this node at every coarse level (static indices: registers)
#pragma unroll
      for (int l = 1; l < 8; ++l) citem[l] = l < al.L ? al.vec_off[l] + al.coarse[l][node] : 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k >= nrhs) break;
        const float v = acc[k] + acc[8 + k];
        if (kF32) {
          float w = v;
#pragma unroll
          for (int l = 1; l < 8; ++l)
            if (l < al.L) w += ((const float*)zlv)[(citem[l] * nrhs + k) * 3 + c];
          ((float*)zv)[((int64_t)node * nrhs + k) * 3 + c] = w;
        } else {
          double w = (double)v;
#pragma unroll
          for (int l = 1; l < 8; ++l)
            if (l < al.L) w += ((const double*)zlv)[k * lstride + 3 * citem[l] + c];
          ((double*)zv)[k * stride + 3 * (int64_t)node + c] = w;
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, 32);
  }
}

// double -> float -> bfloat16 (both to nearest even), written in the
// K-major operand layout: per domain [k/8][i/8][i%8][k%8], A[i][k] = M^{-1}[k][i].
__global__ void k_to_bf16_tc(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n_dom, int ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)ld * ld;
  if (e >= n_dom * per) return;
  const int64_t dom = e / per;
  const int rem = (int)(e - dom * per);
  const int k8 = rem & 7, r8 = (rem >> 3) & 7, t = rem >> 6;
  const int groups = ld / 8;
  const int i = (t % groups) * 8 + r8, k = (t / groups) * 8 + k8;
  b[e] = __float2bfloat16_rn((float)a[dom * per + (int64_t)k * ld + i]);
}

}  // namespace tc

bool level0_tc_usable(gs_ctx ctx, gs_mas mas, int nrhs) {
  return mas->inv16_tc != nullptr && nrhs >= 1 && nrhs <= 8 && ctx->tune[GS_TUNE_BF16_TC] != 0;
}

int level0_tc_prepare(gs_ctx ctx, gs_mas mas) {
  const int ld = 3 * mas->N;
  if (mas->precision != GS_PREC_BF16 || ld % 16 != 0 || ld > tc::kM || mas->inv16_tc) return GS_OK;
  const int64_t cnt = (int64_t)mas->n_domains[0] * ld * ld;
  GS_TRY(ctx->alloc(&mas->inv16_tc, (size_t)std::max<int64_t>(cnt, 1) * 2));
  if (cnt) {
    GS_PROF(ctx, GS_K_MAS_INVERT);
    tc::k_to_bf16_tc<<<ceil_div(cnt, 256), 256, 0, ctx->stream>>>(mas->inv64[0], (__nv_bfloat16*)mas->inv16_tc,
                                                                   mas->n_domains[0], ld);
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

int level0_tc_launch(gs_ctx ctx, gs_mas mas, bool f32_node_major, int nrhs, const void* r, int64_t stride,
                     const void* zl, int64_t lstride, void* z, const int* skip, int* flags) {
  GS_CHECK(level0_tc_usable(ctx, mas, nrhs), GS_ERR_UNSUPPORTED, "tensor-core level-0 apply: not available");
  const int ld = 3 * mas->N;
  tc::Levels al{};
  al.L = mas->L;
  for (int l = 0; l < mas->L; ++l) al.coarse[l] = mas->coarse[l], al.vec_off[l] = mas->vec_off[l];
  const size_t smem = 128 + tc::round128(tc::a_span(ld)) + tc::b_bytes(ld) + 2 * 8 + 8;
  if (mas->n_domains[0] == 0) return GS_OK;
  if (f32_node_major)
    tc::k_level0_tc<true><<<mas->n_domains[0], tc::kThreads, smem, ctx->stream>>>(
        (const __nv_bfloat16*)mas->inv16_tc, mas->remap0, mas->N, nrhs, al, r, stride, zl, lstride, z, skip, flags);
  else
    tc::k_level0_tc<false><<<mas->n_domains[0], tc::kThreads, smem, ctx->stream>>>(
        (const __nv_bfloat16*)mas->inv16_tc, mas->remap0, mas->N, nrhs, al, r, stride, zl, lstride, z, skip, flags);
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs
