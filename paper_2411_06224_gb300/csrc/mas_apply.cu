// MAS preconditioner apply z = sum_l C_l^T M_l^{-1} C_l r (supplement Eq. 4-6).
//
// The coarseners map level 0 directly to every level, so all levels are
// independent once the restricted vectors exist:
//   1. k_restrict: one warp per level-0 domain gathers its nodes' residuals
//      and sums them per level-1 item (an item lies inside one domain, so
//      the warp stores its sums); k_restrict_up then sums each level's items
//      into the next level's, one warp per domain, in a fixed order;
//   2. k_domain_product on the coarse levels: z_l = M_l^{-1} r_l per domain;
//   3. k_domain_product on level 0 fused with the prolongation: each node's
//      z = (M_0^{-1} r)_slot + sum_l z_l[coarse_l(node)], written once.
// The dense products read each inverse once for all right-hand sides: a
// thread owns one row of the 3N x 3N inverse and kRPT right-hand sides;
// the inverse is symmetric, so row i is read as column i (coalesced).
#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "primitives.cuh"
#include "umma.cuh"

namespace gs {

struct ApplyLevels {
  const int32_t* coarse[8];
  int64_t vec_off[8];
  int L;
  int N;
};

// One warp per level-0 domain, four warps per block; lane q < 24 owns value q
// of a node (RHS k0 + q / 3, component q % 3) and sums it over the nodes of
// a group in ascending slot order: about 31 FP64 adds per group, no shuffle
// trees (FP64 adds are scarce on this part).  Groups are the domain's level-1
// items; a level-1 item lies inside one item of every coarser level, so its
// sums serve all levels.  Most domains are one group: then the 32 nodes'
// values are loaded at once and summed in registers.
constexpr int kRestrictWarps = 4;
// Inverse entries a thread of the dense products loads before it uses them.
constexpr int kChunk = 16;

// FP64 <-> arithmetic type; the FP32 conversions go through bit patterns
// (conversion instructions would run on the FP64 pipe).
template <typename Tm>
__device__ __forceinline__ Tm to_tm(double v) {
  return v;
}
template <>
__device__ __forceinline__ float to_tm<float>(double v) {
  return f64_to_f32_bits(v);
}
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64_bits(v); }

__global__ void __launch_bounds__(32 * kRestrictWarps) k_restrict(const double* __restrict__ r, int64_t stride,
                                                                  int nrhs, const int32_t* __restrict__ remap0,
                                                                  int32_t n_dom0, ApplyLevels al,
                                                                  double* __restrict__ rl, int64_t lstride,
                                                                  const int* __restrict__ skip) {
  if (skip && *skip) return;  // every RHS of the solve has converged
  const int wib = threadIdx.x >> 5;
  const int32_t d = (int32_t)(blockIdx.x * kRestrictWarps + wib);
  const int lane = threadIdx.x & 31;
  if (d >= n_dom0) return;  // whole warp
  const int N = al.N;
  const int32_t node = lane < N ? remap0[(int64_t)d * N + lane] : -1;
  const bool real = node >= 0;
  const int32_t c1 = real ? al.coarse[1][node] : -1;
  const uint32_t realm = __ballot_sync(kFull, real);
  if (!realm) return;  // whole warp
  const int lead0 = __ffs(realm) - 1;
  const int32_t c_first = __shfl_sync(kFull, c1, lead0);
  const bool one_group = __all_sync(kFull, !real || c1 == c_first);
  for (int k0 = 0; k0 < nrhs; k0 += 8) {
    const int k = k0 + lane / 3, c = lane % 3;
    const bool act = lane < 24 && k < nrhs;
    const double* rk = r + k * stride + c;
    uint32_t left = realm;
    while (left) {
      int lead;
      int32_t cc;
      uint32_t g;
      double sum = 0.0;
      if (one_group) {  // all real slots: loads first, then the sum in slot order
        lead = lead0, cc = c_first, g = realm;
        double v[32];
#pragma unroll
        for (int s = 0; s < 32; ++s) {
          const int32_t ns = __shfl_sync(kFull, node, s);
          v[s] = (act && ns >= 0) ? rk[3 * (int64_t)ns] : 0.0;
        }
#pragma unroll
        for (int s = 0; s < 32; ++s)
          if ((realm >> s) & 1u) sum += v[s];
      } else {
        lead = __ffs(left) - 1;
        cc = __shfl_sync(kFull, c1, lead);
        g = __ballot_sync(kFull, real && c1 == cc);
        for (uint32_t m = g; m; m &= m - 1) {
          const int32_t ns = __shfl_sync(kFull, node, __ffs(m) - 1);
          if (act) sum += rk[3 * (int64_t)ns];
        }
      }
      left &= ~g;
      // a level-1 item lies inside this domain: this warp is its only writer
      if (act) rl[k * lstride + c + 3 * (al.vec_off[1] + cc)] = sum;
    }
  }
}

// Dense per-domain products.  kMode 0: coarse levels (input rl, output zl);
// kMode 1: level 0 (gather through remap0, prolongate, write z).  Ts is
// the storage type of the inverses, Tm the arithmetic type.
template <typename Ts, typename Tm, int kRPT, int kMode>
__global__ void __launch_bounds__(1024) k_domain_product(
    const Ts* const* __restrict__ inv, const int32_t* __restrict__ job_level, const int32_t* __restrict__ job_dom,
    int N, int nrhs,
    // level-0 inputs / outputs
    const double* __restrict__ r, double* __restrict__ z, int64_t stride, const int32_t* __restrict__ remap0,
    // multilevel vectors
    const double* __restrict__ rl, double* __restrict__ zl, int64_t lstride, ApplyLevels al) {
  extern __shared__ unsigned char smem_raw[];
  Tm* sr = (Tm*)smem_raw;  // [3N][nrhs]
  const int ld = 3 * N;
  const int l = (kMode == 1) ? 0 : job_level[blockIdx.x];
  const int32_t d = (kMode == 1) ? blockIdx.x : job_dom[blockIdx.x];
  const Ts* Mi = inv[l] + (int64_t)d * ld * ld;
  const int tid = threadIdx.x;
  // stage the domain's right-hand sides
  for (int e = tid; e < ld * nrhs; e += blockDim.x) {
    const int j = e / nrhs, k = e % nrhs;
    double v;
    if (kMode == 1) {
      const int32_t node = remap0[(int64_t)d * N + j / 3];
      v = node >= 0 ? r[k * stride + 3 * (int64_t)node + j % 3] : 0.0;
    } else {
      v = rl[k * lstride + 3 * (al.vec_off[l] + (int64_t)d * N) + j];
    }
    sr[j * nrhs + k] = to_tm<Tm>(v);
  }
  __syncthreads();
  const int i = tid % ld;
  const int g = tid / ld;
  const int k0 = g * kRPT;
  if (k0 >= nrhs) return;
  Tm acc[kRPT];
#pragma unroll
  for (int q = 0; q < kRPT; ++q) acc[q] = (Tm)0;
  // the column in chunks of kChunk independent loads, so each thread keeps
  // that many inverse entries in flight; the sums stay in ascending j
  const Ts* col = Mi + i;
  int j = 0;
  for (; j + kChunk <= ld; j += kChunk, col += (int64_t)kChunk * ld) {
    Tm mv[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) mv[u] = (Tm)widen(col[u * ld]);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const Tm* rj = sr + (j + u) * nrhs + k0;
#pragma unroll
      for (int q = 0; q < kRPT; ++q)
        if (k0 + q < nrhs) acc[q] += mv[u] * rj[q];
    }
  }
  for (; j < ld; ++j, col += ld) {
    const Tm m = (Tm)widen(*col);
    const Tm* rj = sr + j * nrhs + k0;
#pragma unroll
    for (int q = 0; q < kRPT; ++q)
      if (k0 + q < nrhs) acc[q] += m * rj[q];
  }
  if (kMode == 0) {
#pragma unroll
    for (int q = 0; q < kRPT; ++q)
      if (k0 + q < nrhs) zl[(k0 + q) * lstride + 3 * (al.vec_off[l] + (int64_t)d * N) + i] = to_f64(acc[q]);
    return;
  }
  const int32_t node = remap0[(int64_t)d * N + i / 3];
  if (node < 0) return;
  const int x = i % 3;
  int32_t citem[8];
  for (int ll = 1; ll < al.L; ++ll) citem[ll] = al.coarse[ll][node];
#pragma unroll
  for (int q = 0; q < kRPT; ++q) {
    const int k = k0 + q;
    if (k >= nrhs) break;
    // summed in the arithmetic type: FP64, or FP32 for the FP32 form (its
    // every level's product is FP32), conversions from bit patterns
    Tm v = acc[q];
    for (int ll = 1; ll < al.L; ++ll) v += to_tm<Tm>(zl[k * lstride + 3 * (al.vec_off[ll] + citem[ll]) + x]);
    z[k * stride + 3 * (int64_t)node + x] = to_f64(v);
  }
}

// FP32 level 0 + prolongation: one CTA of 3N threads per domain, thread i
// owning row i for all (at most 8) right-hand sides.  The domain's inverse is
// stored as its lower triangle packed by rows (18.6 KB at N = 32, half the
// full matrix), so ten CTAs share an SM, and comes into shared memory by one
// bulk asynchronous copy issued first; the right-hand sides are gathered into
// shared memory and the prolongated coarse results (which start the sums)
// are loaded while it lands.  Row i of the symmetric inverse is its packed
// row for j <= i and column i below it (entry (j, i) of row j) for j > i,
// summed in ascending j; four steps' shared-memory loads are issued before
// their FMAs (one step at a time left the warps waiting on each load).  The
// copy wait is bounded: on a timeout the kernel sets kErrTimeout, waits
// (bounded) for the copy to land and writes nothing.
constexpr int kF32Unroll = 4;

__global__ void __launch_bounds__(96) k_level0_f32_cta(const float* __restrict__ invp, int pitch, int N, int nrhs,
                                                        const double* __restrict__ r, double* __restrict__ z,
                                                        int64_t stride, const int32_t* __restrict__ remap0,
                                                        const double* __restrict__ zl, int64_t lstride,
                                                        ApplyLevels al, const int* __restrict__ skip,
                                                        int* __restrict__ flags) {
  using namespace umma;
  if (skip && *skip) return;  // every RHS of the solve has converged
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = 3 * N;
  const int32_t d = blockIdx.x;
  const int tid = threadIdx.x;
  const uint32_t mbytes = (uint32_t)pitch * 4;
  float* sp = (float*)smem_raw;
  float* sr = sp + pitch;  // [ld][8]
  uint64_t* bar = (uint64_t*)(sr + ld * 8);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, mbytes);
    bulk_g2s(sp, invp + (int64_t)d * pitch, mbytes, bar);
  }
  for (int e = tid; e < ld * 8; e += blockDim.x) {  // e = j * 8 + k
    const int j = e >> 3, k = e & 7;
    float v = 0.0f;
    if (k < nrhs) {
      const int32_t node = remap0[(int64_t)d * N + j / 3];
      if (node >= 0) v = f64_to_f32_bits(r[k * stride + 3 * (int64_t)node + j % 3]);
    }
    sr[e] = v;
  }
  const int i = tid;
  const bool act = i < ld;
  const int32_t node = act ? remap0[(int64_t)d * N + i / 3] : -1;
  const int x = i % 3;
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
  if (node >= 0) {
#pragma unroll
    for (int ll = 1; ll < 8; ++ll) {
      if (ll >= al.L) break;
      const int64_t ci = al.vec_off[ll] + al.coarse[ll][node];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < nrhs) acc[k] += f64_to_f32_bits(zl[k * lstride + 3 * ci + x]);
    }
  }
  __shared__ int s_ok;
  if (tid == 0) s_ok = mbar_wait(bar, 0);
  __syncthreads();
  if (!s_ok) {
    if (tid == 0) {
      atomicOr(flags, kErrTimeout);
      mbar_wait(bar, 0);  // let a late copy land before the CTA leaves
    }
    return;
  }
  if (!act) return;
  const int rb = i * (i + 1) / 2;
  int tri = 0;  // j (j + 1) / 2
  int j0 = 0;
  for (; j0 + kF32Unroll <= ld; j0 += kF32Unroll) {
    float m[kF32Unroll];
    float4 ra[kF32Unroll], rc[kF32Unroll];
#pragma unroll
    for (int u = 0; u < kF32Unroll; ++u) {
      const int j = j0 + u;
      m[u] = sp[j <= i ? rb + j : tri + i];
      ra[u] = *reinterpret_cast<const float4*>(sr + j * 8);
      rc[u] = *reinterpret_cast<const float4*>(sr + j * 8 + 4);
      tri += j + 1;
    }
#pragma unroll
    for (int u = 0; u < kF32Unroll; ++u) {
      acc[0] = fmaf(m[u], ra[u].x, acc[0]), acc[1] = fmaf(m[u], ra[u].y, acc[1]);
      acc[2] = fmaf(m[u], ra[u].z, acc[2]), acc[3] = fmaf(m[u], ra[u].w, acc[3]);
      acc[4] = fmaf(m[u], rc[u].x, acc[4]), acc[5] = fmaf(m[u], rc[u].y, acc[5]);
      acc[6] = fmaf(m[u], rc[u].z, acc[6]), acc[7] = fmaf(m[u], rc[u].w, acc[7]);
    }
  }
  for (; j0 < ld; ++j0) {
    const float m = sp[j0 <= i ? rb + j0 : tri + i];
    const float* rj = sr + j0 * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = fmaf(m, rj[k], acc[k]);
    tri += j0 + 1;
  }
  if (node < 0) return;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (k < nrhs) z[k * stride + 3 * (int64_t)node + x] = f32_to_f64_bits(acc[k]);
}

// Floats per domain of the packed level-0 inverses (16-byte multiple).
static int f32_pitch(int N) {
  const int ld = 3 * N;
  return ((ld * (ld + 1) / 2 + 3) / 4) * 4;
}

// Shared memory of k_level0_f32_cta; 0 when it cannot be used (3N <= 96 rows).
static size_t f32_cta_smem(int N) {
  const size_t ld = 3 * (size_t)N;
  if (ld > 96) return 0;
  return (size_t)f32_pitch(N) * 4 + ld * 8 * 4 + 16;
}

bool level0_f32_bulk_usable(gs_mas mas, int nrhs) {
  return mas->precision == GS_PREC_FP32 && mas->inv32p && nrhs <= 8 && f32_cta_smem(mas->N) > 0;
}

// Coarse levels hold few domains, so each output (row i of a domain, RHS k)
// gets its own thread: the 3N-long dot product reads row i of the symmetric
// inverse as column i (coalesced across i) and broadcasts r.
template <typename Ts, typename Tm>
__global__ void __launch_bounds__(256) k_coarse_product(const Ts* const* __restrict__ inv,
                                                        const int32_t* __restrict__ job_level,
                                                        const int32_t* __restrict__ job_dom, int n_jobs, int N,
                                                        int nrhs, const double* __restrict__ rl,
                                                        double* __restrict__ zl, int64_t lstride, ApplyLevels al) {
  const int ld = 3 * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_job = (int64_t)ld * nrhs;
  if (t >= per_job * n_jobs) return;
  const int job = (int)(t / per_job);
  const int rem = (int)(t % per_job);
  const int k = rem / ld, i = rem % ld;
  const int l = job_level[job];
  const int32_t d = job_dom[job];
  const Ts* Mi = inv[l] + (int64_t)d * ld * ld;
  const double* rj = rl + k * lstride + 3 * (al.vec_off[l] + (int64_t)d * N);
  Tm acc = (Tm)0;
  const Ts* col = Mi + i;
  int j = 0;
  for (; j + kChunk <= ld; j += kChunk, col += (int64_t)kChunk * ld) {  // kChunk loads in flight, sums in order
    Tm mv[kChunk], rv[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      mv[u] = (Tm)widen(col[u * ld]);
      rv[u] = to_tm<Tm>(rj[j + u]);
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u) acc += mv[u] * rv[u];
  }
  for (; j < ld; ++j, col += ld) acc += (Tm)widen(*col) * to_tm<Tm>(rj[j]);
  zl[k * lstride + 3 * (al.vec_off[l] + (int64_t)d * N) + i] = to_f64(acc);
}

template <typename Ts, typename Tm>
static int launch_apply(gs_ctx ctx, gs_mas mas, const Ts* const* d_inv, const int32_t* d_jobs, int n_coarse_jobs,
                        const double* r, double* z, int nrhs, double* rl, double* zl, const int* skip) {
  cudaStream_t st = ctx->stream;
  const int N = mas->N, ld = 3 * N;
  const int64_t stride = 3LL * mas->n;
  const int64_t lstride = 3 * std::max<int64_t>(mas->vec_items, 1);
  ApplyLevels al{};
  al.L = mas->L;
  al.N = N;
  for (int l = 0; l < mas->L; ++l) {
    al.coarse[l] = mas->coarse[l];
    al.vec_off[l] = mas->vec_off[l];
  }
  const int kRPT = ctx->tune[GS_TUNE_APPLY_RHS];
  const int groups = ceil_div(nrhs, kRPT);
  const int threads = ((ld * groups + 31) / 32) * 32;
  const size_t smem = (size_t)ld * nrhs * sizeof(Tm);
  GS_CHECK(threads <= 1024, GS_ERR_UNSUPPORTED, "mas apply: too many right-hand sides (%d)", nrhs);
  if (mas->L > 1) {
    GS_CUDA(cudaMemsetAsync(rl, 0, (size_t)nrhs * lstride * sizeof(double), st));
    { GS_PROF(ctx, GS_K_MAS_APPLY_COARSE); k_restrict<<<ceil_div(mas->n_domains[0], kRestrictWarps), 32 * kRestrictWarps, 0, st>>>(r, stride, nrhs, mas->remap0,
                                                                              mas->n_domains[0], al, rl, lstride, skip); }
    for (int l = 1; l + 1 < mas->L; ++l) {  // levels >= 2 from the level below, in a fixed order
      GS_PROF(ctx, GS_K_MAS_APPLY_COARSE);
      k_restrict_up<double, LevelIdxRhsMajor><<<ceil_div((int64_t)mas->n_domains[l] * 32, 128), 128, 0, st>>>(
          mas->up[l], mas->n_domains[l], N, 3 * nrhs, LevelIdxRhsMajor{lstride, mas->vec_off[l]},
          LevelIdxRhsMajor{lstride, mas->vec_off[l + 1]}, rl, skip);
    }
    if (level0_f64tc_usable(ctx, mas, nrhs)) {  // FP64 accuracy on the BF16 tensor cores
      GS_PROF(ctx, GS_K_MAS_APPLY_COARSE);
      GS_TRY(coarse_f64tc_launch(ctx, mas, nrhs, rl, zl, lstride, skip));
    } else if (std::is_same<Ts, float>::value && nrhs <= 8 && n_coarse_jobs > 0) {
      // FP32: one CTA per coarse domain, (row, 4 RHS) per thread, inverse
      // entries loaded 16 ahead (a thread per output re-read the RHS row
      // per output and waited on each inverse entry)
      GS_PROF(ctx, GS_K_MAS_APPLY_COARSE);
      const int thr = ((ld * ceil_div(nrhs, 4) + 31) / 32) * 32;
      k_domain_product<Ts, Tm, 4, 0><<<n_coarse_jobs, thr, (size_t)ld * nrhs * sizeof(Tm), st>>>(
          d_inv, d_jobs, d_jobs + n_coarse_jobs, N, nrhs, nullptr, nullptr, 0, nullptr, rl, zl, lstride, al);
    } else {
      GS_PROF(ctx, GS_K_MAS_APPLY_COARSE);
      const int64_t outs = (int64_t)n_coarse_jobs * ld * nrhs;
      k_coarse_product<Ts, Tm><<<ceil_div(outs, 256), 256, 0, st>>>(d_inv, d_jobs, d_jobs + n_coarse_jobs, n_coarse_jobs,
                                                                N, nrhs, rl, zl, lstride, al);
    }
  }
  if (mas->precision == GS_PREC_BF16) {  // level 0 holds BF16 factors: z = W^T (W r)
    GS_PROF(ctx, GS_K_MAS_APPLY_L0);
    GS_TRY(level0_bf16_launch(ctx, mas, false, nrhs, r, stride, zl, lstride, z, nullptr, ctx->d_flags));
  } else if (std::is_same<Ts, float>::value && level0_f32_bulk_usable(mas, nrhs)) {  // FP32, packed inverses
    GS_PROF(ctx, GS_K_MAS_APPLY_L0);
    k_level0_f32_cta<<<mas->n_domains[0], ((ld + 31) / 32) * 32, f32_cta_smem(N), st>>>(
        mas->inv32p, f32_pitch(N), N, nrhs, r, z, stride, mas->remap0, zl, lstride, al, skip, ctx->d_flags);
  } else if (level0_f64tc_usable(ctx, mas, nrhs)) {  // FP64 accuracy on the BF16 tensor cores
    GS_PROF(ctx, GS_K_MAS_APPLY_L0);
    GS_TRY(level0_f64tc_launch(ctx, mas, nrhs, (const double*)r, stride, (const double*)zl, lstride, (double*)z,
                               skip));
  } else {
    GS_PROF(ctx, GS_K_MAS_APPLY_L0);
#define GS_L0_ARGS d_inv, d_jobs, d_jobs, N, nrhs, r, z, stride, mas->remap0, rl, zl, lstride, al
    if (kRPT == 2)
      k_domain_product<Ts, Tm, 2, 1><<<mas->n_domains[0], threads, smem, st>>>(GS_L0_ARGS);
    else if (kRPT == 8)
      k_domain_product<Ts, Tm, 8, 1><<<mas->n_domains[0], threads, smem, st>>>(GS_L0_ARGS);
    else
      k_domain_product<Ts, Tm, 4, 1><<<mas->n_domains[0], threads, smem, st>>>(GS_L0_ARGS);
#undef GS_L0_ARGS
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

int mas_apply_launch(gs_ctx ctx, gs_mas mas, const double* r, double* z, int nrhs, double* rl, double* zl) {
  return mas_apply_launch_skip(ctx, mas, r, z, nrhs, rl, zl, nullptr);
}

// The same, but the restriction and the digit-split products return at once
// while *skip (device) is set (PCG's all-converged word).
int mas_apply_launch_skip(gs_ctx ctx, gs_mas mas, const double* r, double* z, int nrhs, double* rl, double* zl,
                          const int* skip) {
  // the BF16 form's coarse levels are FP32 inverses
  if (mas->precision == GS_PREC_FP32 || mas->precision == GS_PREC_BF16)
    return launch_apply<float, float>(ctx, mas, (const float* const*)mas->d_inv_tab, mas->d_coarse_jobs,
                                      mas->n_coarse_jobs, r, z, nrhs, rl, zl, skip);
  return launch_apply<double, double>(ctx, mas, (const double* const*)mas->d_inv_tab, mas->d_coarse_jobs,
                                      mas->n_coarse_jobs, r, z, nrhs, rl, zl, skip);
}

int mas_level_vectors(gs_ctx ctx, gs_mas mas, int nrhs, double** rl, double** zl) {
  const size_t per = (size_t)nrhs * 3 * std::max<int64_t>(mas->vec_items, 1);
  double* b = nullptr;
  GS_TRY(ctx->scratch_buf(kSlotMasLevelVec, 2 * per * sizeof(double), (void**)&b));
  *rl = b;
  *zl = b + per;
  return GS_OK;
}

}  // namespace gs

extern "C" int gs_mas_apply(gs_ctx ctx, gs_mas mas, const double* r, double* z, int32_t nrhs) {
  GS_CHECK(ctx && mas && r && z && r != z, GS_ERR_INVALID, "gs_mas_apply: null or aliased argument");
  GS_CHECK(nrhs >= 1, GS_ERR_INVALID, "gs_mas_apply: nrhs %d", nrhs);
  GS_CUDA(cudaSetDevice(ctx->device));
  double *rl, *zl;
  GS_TRY(gs::mas_level_vectors(ctx, mas, nrhs, &rl, &zl));
  GS_TRY(gs::mas_apply_launch(ctx, mas, r, z, nrhs, rl, zl));
  if (gs::level0_bf16_on_tensor_cores(ctx, mas, nrhs) || gs::level0_f64tc_usable(ctx, mas, nrhs) ||
      gs::level0_f32_bulk_usable(mas, nrhs)) {
    // the tensor-core and bulk-copy kernels report bounded-wait timeouts
    int flags = 0;
    GS_TRY(ctx->take_flags(&flags));
    if (flags) return gs::status_from_flags(flags);
  }
  return GS_OK;
}
