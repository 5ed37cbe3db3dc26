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

#include "common.cuh"
#include "primitives.cuh"

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
    sr[j * nrhs + k] = (Tm)v;
  }
  __syncthreads();
  const int i = tid % ld;
  const int g = tid / ld;
  const int k0 = g * kRPT;
  if (k0 >= nrhs) return;
  Tm acc[kRPT];
#pragma unroll
  for (int q = 0; q < kRPT; ++q) acc[q] = (Tm)0;
  for (int j = 0; j < ld; ++j) {
    const Tm m = (Tm)widen(Mi[(int64_t)j * ld + i]);
    const Tm* rj = sr + j * nrhs + k0;
#pragma unroll
    for (int q = 0; q < kRPT; ++q)
      if (k0 + q < nrhs) acc[q] += m * rj[q];
  }
  if (kMode == 0) {
#pragma unroll
    for (int q = 0; q < kRPT; ++q)
      if (k0 + q < nrhs) zl[(k0 + q) * lstride + 3 * (al.vec_off[l] + (int64_t)d * N) + i] = (double)acc[q];
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
    double v = (double)acc[q];
    for (int ll = 1; ll < al.L; ++ll) v += zl[k * lstride + 3 * (al.vec_off[ll] + citem[ll]) + x];
    z[k * stride + 3 * (int64_t)node + x] = v;
  }
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
  for (int j = 0; j < ld; ++j) acc += (Tm)widen(Mi[(int64_t)j * ld + i]) * (Tm)rj[j];
  zl[k * lstride + 3 * (al.vec_off[l] + (int64_t)d * N) + i] = (double)acc;
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
  if (gs::level0_bf16_on_tensor_cores(ctx, mas, nrhs) || gs::level0_f64tc_usable(ctx, mas, nrhs)) {
    // the tensor-core kernels report bounded-wait timeouts
    int flags = 0;
    GS_TRY(ctx->take_flags(&flags));
    if (flags) return gs::status_from_flags(flags);
  }
  return GS_OK;
}
