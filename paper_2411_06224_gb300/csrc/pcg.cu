// Preconditioned conjugate gradients for several right-hand sides (Sec. 3.2).
//
// Per iteration (one SpMV per RHS):
//   Ap = A p                         spmv.cu
//   alpha = rz / (p . Ap)            k_dot (finalised on the device)
//   x += alpha p, r -= alpha Ap      k_update_xr, fused with ||r||^2 and the
//                                    per-RHS convergence test
//   z = M^{-1} r                     mas_apply.cu
//   beta = (r . z) / rz, rz = r . z  k_dot
//   p = z + beta p                   k_update_p
// Every reduction is deterministic: a fixed grid writes per-block partials
// and the last block to finish sums them in block order and updates the
// per-RHS scalars, so no scalar ever travels to the host inside the loop.
// A RHS stops moving once converged (alpha = 0), which keeps each RHS on
// exactly its own single-RHS recurrence.  Kernels return at once after
// every RHS converged; the host only polls that flag every few iterations.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "ff.cuh"
#include "primitives.cuh"

namespace gs {

int spmv_launch(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, int variant);
int mas_apply_launch(gs_ctx ctx, gs_mas mas, const double* r, double* z, int nrhs, double* rl, double* zl);
int mas_level_vectors(gs_ctx ctx, gs_mas mas, int nrhs, double** rl, double** zl);
int ensure_row_order(gs_ctx ctx, gs_mat m);

constexpr int kMaxRhs = 32;
constexpr int kRedThreads = 256;
constexpr int kMaxRedBlocks = 256;  // reduction blocks per right-hand side
constexpr int kUnroll = 4;          // strided elements per thread and pass of k_dot and k_update_p

struct PcgScalars {
  double bnorm2[kMaxRhs];
  double rz[kMaxRhs];
  double alpha[kMaxRhs];
  double beta[kMaxRhs];
  double rr[kMaxRhs];
  int conv[kMaxRhs];
  int iters[kMaxRhs];
  // float-float SpMV operand (GS_SPMV_ROW_FF): |z| < 2^fz, |p| < 2^fp, and
  // the split copy of p holds p 2^(k_node - K - fsplit)
  int fz[kMaxRhs];
  int fp[kMaxRhs];
  int fsplit[kMaxRhs];
  int all_conv;
  unsigned counter;
  int flags;
};

enum DotOp : int { kOpBnorm = 0, kOpRzInit, kOpPAp, kOpRR, kOpRz };

// Grid of the vector kernels: (G, nrhs); block (g, k) covers a contiguous
// chunk of right-hand side k.  G depends only on the vector length, the RHS
// count and the GPU's SM count, so on one GPU the reduction order -- and
// therefore the result -- is fixed.
inline int red_blocks(int64_t len, int nrhs, int sms) {
  // 32 entries per thread: each block's reduction, fence and arrival are
  // fixed costs, so blocks are made long (measured: 8 per thread left k_dot
  // stalled on its block reductions at 21 % of the DRAM peak) -- but no
  // fewer than about two blocks per SM over all RHS while a block still gets
  // 8 entries per thread
  int64_t g = (len + kRedThreads * 32 - 1) / (kRedThreads * 32);
  const int64_t want = (2LL * std::max(sms, 1) + nrhs - 1) / nrhs;
  const int64_t cap8 = (len + kRedThreads * 8 - 1) / (kRedThreads * 8);
  g = std::max(g, std::min(want, cap8));
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxRedBlocks));
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;  // valid in warp 0
}

__device__ __forceinline__ int block_max(int v) {
  __shared__ int red[kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  if (lane == 0) red[w] = v;
  __syncthreads();
  int t = kExpNone;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : kExpNone;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = max(t, __shfl_xor_sync(kFull, t, o));
  }
  __syncthreads();
  return t;  // valid in warp 0
}

__device__ __forceinline__ void chunk_of(int64_t len, int64_t& b, int64_t& e) {
  const int64_t per = (len + gridDim.x - 1) / gridDim.x;
  b = (int64_t)blockIdx.x * per;
  e = b + per < len ? b + per : len;
}

__device__ void apply_op(PcgScalars* s, int k, double sum, int op, double tol2) {
  if (!isfinite(sum)) {
    atomicOr(&s->flags, kErrNonFinite);
    s->conv[k] = 1;
    s->alpha[k] = 0.0;
    return;
  }
  switch (op) {
    case kOpBnorm:
      s->bnorm2[k] = sum;
      s->conv[k] = sum == 0.0;
      s->iters[k] = 0;
      s->rr[k] = sum;
      break;
    case kOpRzInit:
      s->rz[k] = sum;
      break;
    case kOpPAp:
      if (s->conv[k]) {
        s->alpha[k] = 0.0;
      } else if (!(sum > 0.0)) {
        atomicOr(&s->flags, kErrNotSPD);
        s->conv[k] = 1;
        s->alpha[k] = 0.0;
      } else {
        s->alpha[k] = s->rz[k] / sum;
      }
      break;
    case kOpRR:
      if (!s->conv[k]) {
        s->rr[k] = sum;
        s->iters[k] += 1;
        if (sum <= tol2 * s->bnorm2[k]) s->conv[k] = 1;
      }
      break;
    case kOpRz:
      s->beta[k] = s->conv[k] ? 0.0 : sum / s->rz[k];
      s->rz[k] = sum;
      break;
  }
}

// Write this block's partial; the last block to arrive reduces all partials
// of every right-hand side in a fixed order and updates the scalars.  With
// ipart, each block also posts the largest exponent bound of the vector it
// read (my_ex, valid in thread 0), and the last block keeps the maximum per
// RHS as fz (and fp for op kOpRzInit, where p = z).
__device__ void finalize(PcgScalars* s, double* __restrict__ partials, double my_partial, int nrhs, int op,
                         double tol2, int* __restrict__ ipart = nullptr, int my_ex = kExpNone) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.y * kMaxRedBlocks + blockIdx.x] = my_partial;
    if (ipart) ipart[blockIdx.y * kMaxRedBlocks + blockIdx.x] = my_ex;
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y;
    last = atomicInc(&s->counter, total - 1) == total - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // one warp per right-hand side (fixed order: lane, then stride 32, then
  // the shuffle tree), so the tail costs one warp reduction, not nrhs block ones
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < nrhs; k += kRedThreads / 32) {
    double v = 0.0;
    for (int g = lane; g < (int)gridDim.x; g += 32) v += __ldcg(&partials[k * kMaxRedBlocks + g]);
    v = warp_sum(v);
    if (lane == 0) apply_op(s, k, v, op, tol2);
    if (ipart) {
      int e = kExpNone;
      for (int g = lane; g < (int)gridDim.x; g += 32) e = max(e, __ldcg(&ipart[k * kMaxRedBlocks + g]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(kFull, e, o));
      if (lane == 0) {
        s->fz[k] = e;
        if (op == kOpRzInit) s->fp[k] = e;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int k = 0; k < nrhs; ++k) all &= s->conv[k] != 0;
    s->all_conv = all;
  }
}

// a_k . b_k per right-hand side; kCopy also writes dst = b (p = z); kEx also
// takes the largest exponent bound of b (z) for the float-float SpMV operand.
template <bool kCopy, bool kEx = false>
__global__ void __launch_bounds__(kRedThreads) k_dot(const double* __restrict__ a, const double* __restrict__ b,
                                                     double* __restrict__ dst, int64_t len, int nrhs,
                                                     PcgScalars* s, double* __restrict__ partials, int op,
                                                     int* __restrict__ ipart = nullptr) {
  if (s->all_conv && op != kOpBnorm && op != kOpRzInit) return;
  const int64_t o = (int64_t)blockIdx.y * len;
  int64_t i0, i1;
  chunk_of(len, i0, i1);
  // kUnroll strided elements per pass, loaded before they are summed: more
  // loads in flight per thread, and the thread's sum keeps its order
  double v = 0.0;
  int ex = kExpNone;
  const int64_t T = blockDim.x;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kUnroll * T) {
    double av[kUnroll], bv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t j = i + u * T;
      av[u] = j < i1 ? a[o + j] : 0.0;
      bv[u] = j < i1 ? b[o + j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t j = i + u * T;
      if (j < i1) {
        v += av[u] * bv[u];
        if (kCopy) dst[o + j] = bv[u];
        if (kEx) ex = max(ex, ex_bound(bv[u]));
      }
    }
  }
  if (kEx) ex = block_max(ex);
  finalize(s, partials, block_sum(v), nrhs, op, 0.0, kEx ? ipart : nullptr, ex);
}

__global__ void __launch_bounds__(kRedThreads) k_init(const double* __restrict__ bvec, double* __restrict__ x,
                                                      double* __restrict__ r, int64_t len, int nrhs, PcgScalars* s,
                                                      double* __restrict__ partials) {
  const int64_t o = (int64_t)blockIdx.y * len;
  int64_t i0, i1;
  chunk_of(len, i0, i1);
  double v = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double bb = bvec[o + i];
    x[o + i] = 0.0;
    r[o + i] = bb;
    v += bb * bb;
  }
  finalize(s, partials, block_sum(v), nrhs, kOpBnorm, 0.0);
}

__global__ void __launch_bounds__(kRedThreads) k_update_xr(double* __restrict__ x, double* __restrict__ r,
                                                           const double* __restrict__ p, const double* __restrict__ Ap,
                                                           int64_t len, int nrhs, PcgScalars* s,
                                                           double* __restrict__ partials, double tol2) {
  if (s->all_conv) return;
  const int k = blockIdx.y;
  const double al = s->alpha[k];
  const int64_t o = (int64_t)k * len;
  int64_t i0, i1;
  chunk_of(len, i0, i1);
  double v = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double rk = r[o + i];
    if (al != 0.0) {
      x[o + i] += al * p[o + i];
      rk -= al * Ap[o + i];
      r[o + i] = rk;
    }
    v += rk * rk;
  }
  finalize(s, partials, block_sum(v), nrhs, kOpRR, tol2);
}

__global__ void __launch_bounds__(kRedThreads) k_update_p(double* __restrict__ p, const double* __restrict__ z,
                                                          int64_t len, const PcgScalars* s) {
  const int k = blockIdx.y;
  if (s->all_conv || s->conv[k]) return;
  const double be = s->beta[k];
  const int64_t o = (int64_t)k * len;
  int64_t i0, i1;
  chunk_of(len, i0, i1);
  const int64_t T = blockDim.x;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kUnroll * T) {
    double zv[kUnroll], pv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t j = i + u * T;
      zv[u] = j < i1 ? z[o + j] : 0.0;
      pv[u] = j < i1 ? p[o + j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (i + u * T < i1) p[o + i + u * T] = zv[u] + be * pv[u];
  }
}

// p = z + beta p (as k_update_p), and the float-float operand of the next
// SpMV: ps = split(p 2^(k_node - K - F)) with 2^F above |p|, taken from the
// bounds |z| < 2^fz, |p_old| < 2^fp, |beta| < 2^eb as max(fz, fp + eb) + 1.
// ps is node-major across right-hand sides, ps[(node * nrhs + k) * 3 + c],
// so the SpMV gathers all RHS of a column in one contiguous stretch.
// The blocks also post the exponent bound of the new p, which the last block
// keeps as fp.  A converged RHS keeps p, ps, fp and fsplit unchanged.
__global__ void __launch_bounds__(kRedThreads) k_update_p_ff(double* __restrict__ p, const double* __restrict__ z,
                                                             float2* __restrict__ ps,
                                                             const int32_t* __restrict__ kk, int64_t len, int nrhs,
                                                             PcgScalars* s, int* __restrict__ ipart) {
  if (s->all_conv) return;  // every block leaves: no arrival is expected
  const int k = blockIdx.y;
  int ex = kExpNone;
  if (!s->conv[k]) {
    const double be = s->beta[k];
    const int eb = ex_bound(be);
    const int fp = s->fp[k], fz = s->fz[k];
    const int fb = (fp == kExpNone || eb == kExpNone) ? kExpNone : fp + eb;
    const int fmax = max(fz, fb);
    const int F = fmax == kExpNone ? 0 : fmax + 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) s->fsplit[k] = F;
    const int64_t o = (int64_t)k * len;
    int64_t i0, i1;
    chunk_of(len, i0, i1);
    const int64_t T = blockDim.x;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kUnroll * T) {
      double zv[kUnroll], pv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t j = i + u * T;
        zv[u] = j < i1 ? z[o + j] : 0.0;
        pv[u] = j < i1 ? p[o + j] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t j = i + u * T;
        if (j < i1) {
          const double v = zv[u] + be * pv[u];
          p[o + j] = v;
          ex = max(ex, ex_bound(v));
          const uint32_t node = (uint32_t)j / 3u;
          ps[((int64_t)node * nrhs + k) * 3 + ((uint32_t)j - 3u * node)] = ff_split_bits(v, kk[node] - F);
        }
      }
    }
  }
  ex = block_max(ex);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    ipart[blockIdx.y * kMaxRedBlocks + blockIdx.x] = ex;
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y;
    last = atomicInc(&s->counter, total - 1) == total - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = w; q < nrhs; q += kRedThreads / 32) {
    int e = kExpNone;
    for (int g = lane; g < (int)gridDim.x; g += 32) e = max(e, __ldcg(&ipart[q * kMaxRedBlocks + g]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(kFull, e, o));
    if (lane == 0 && !s->conv[q]) s->fp[q] = e;
  }
}

// The first split of p (p = z, |p| < 2^fp): fsplit = fp.
__global__ void __launch_bounds__(kRedThreads) k_split_p(const double* __restrict__ p, float2* __restrict__ ps,
                                                         const int32_t* __restrict__ kk, int64_t len, int nrhs,
                                                         PcgScalars* s) {
  const int k = blockIdx.y;
  const int F = s->fp[k] == kExpNone ? 0 : s->fp[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) s->fsplit[k] = F;
  const int64_t o = (int64_t)k * len;
  int64_t i0, i1;
  chunk_of(len, i0, i1);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const uint32_t node = (uint32_t)i / 3u;
    ps[((int64_t)node * nrhs + k) * 3 + ((uint32_t)i - 3u * node)] = ff_split_bits(p[o + i], kk[node] - F);
  }
}

}  // namespace gs

using namespace gs;

extern "C" int gs_pcg_solve(gs_ctx ctx, gs_mat mat, gs_mas mas, const double* b, int32_t nrhs, double tol,
                            int32_t max_iter, int32_t variant, double* x, int32_t* iters, double* rel_res) {
  GS_CHECK(ctx && mat && mas && b && x, GS_ERR_INVALID, "gs_pcg_solve: null argument");
  GS_CHECK(nrhs >= 1 && nrhs <= kMaxRhs, GS_ERR_INVALID, "gs_pcg_solve: nrhs %d (1..%d)", nrhs, kMaxRhs);
  GS_CHECK(mas->n == mat->n, GS_ERR_INVALID, "gs_pcg_solve: preconditioner built for another size");
  GS_CHECK(tol >= 0.0 && max_iter >= 0, GS_ERR_INVALID, "gs_pcg_solve: tol %g max_iter %d", tol, max_iter);
  GS_CHECK(variant == GS_SPMV_SRBK || variant == GS_SPMV_ROW || variant == GS_SPMV_ROW_FF, GS_ERR_INVALID,
           "gs_pcg_solve: variant %d", variant);
  GS_CHECK(b != x, GS_ERR_INVALID, "gs_pcg_solve: b and x alias");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int64_t len = 3LL * mat->n;
  const size_t vbytes = (size_t)nrhs * len * sizeof(double);
  const bool ff = variant == GS_SPMV_ROW_FF;
  double* vec = nullptr;
  GS_TRY(ctx->scratch_buf(kSlotPcgVectors, (ff ? 5 : 4) * vbytes, (void**)&vec));
  double *r = vec, *z = r + nrhs * len, *p = z + nrhs * len, *Ap = p + nrhs * len;
  float2* ps = (float2*)(Ap + nrhs * len);  // float-float operand (same size as a vector)
  char* sbuf = nullptr;
  const size_t part_bytes = kMaxRedBlocks * kMaxRhs * sizeof(double);
  GS_TRY(ctx->scratch_buf(kSlotPcgScalars, sizeof(PcgScalars) + part_bytes + kMaxRedBlocks * kMaxRhs * sizeof(int) + 256,
                          (void**)&sbuf));
  PcgScalars* s = (PcgScalars*)sbuf;
  double* partials = (double*)(sbuf + ((sizeof(PcgScalars) + 255) / 256) * 256);
  int* ipart = (int*)((char*)partials + part_bytes);
  double *rl, *zl;
  GS_TRY(mas_level_vectors(ctx, mas, nrhs, &rl, &zl));
  GS_CUDA(cudaMemsetAsync(s, 0, sizeof(PcgScalars), st));
  if (variant != GS_SPMV_SRBK) GS_TRY(ensure_row_order(ctx, mat));  // built once per matrix
  if (ff) GS_TRY(ensure_ff(ctx, mat));

  const double tol2 = tol * tol;
  const dim3 vg(red_blocks(len, nrhs, ctx->sm_count), nrhs);
  { GS_PROF(ctx, GS_K_PCG_VECTOR); k_init<<<vg, kRedThreads, 0, st>>>(b, x, r, len, nrhs, s, partials); }
  GS_TRY(mas_apply_launch(ctx, mas, r, z, nrhs, rl, zl));
  if (ff) {
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_dot<true, true><<<vg, kRedThreads, 0, st>>>(r, z, p, len, nrhs, s, partials, kOpRzInit, ipart); }
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_split_p<<<vg, kRedThreads, 0, st>>>(p, ps, mat->ff_k, len, nrhs, s); }
  } else {
    GS_PROF(ctx, GS_K_PCG_VECTOR);
    k_dot<true><<<vg, kRedThreads, 0, st>>>(r, z, p, len, nrhs, s, partials, kOpRzInit);
  }
  const int poll = 4;
  int* h_conv = ctx->h_pinned + 64;
  for (int it = 0; it < max_iter; ++it) {
    if (ff)
      GS_TRY(spmv_ff_split_launch(ctx, mat, ps, s->fsplit, Ap, nrhs, &s->all_conv));
    else
      GS_TRY(spmv_launch_skip(ctx, mat, p, Ap, nrhs, variant, &s->all_conv));
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_dot<false><<<vg, kRedThreads, 0, st>>>(p, Ap, nullptr, len, nrhs, s, partials, kOpPAp); }
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_update_xr<<<vg, kRedThreads, 0, st>>>(x, r, p, Ap, len, nrhs, s, partials, tol2); }
    if (it + 1 == max_iter) break;
    GS_TRY(mas_apply_launch_skip(ctx, mas, r, z, nrhs, rl, zl, &s->all_conv));
    if (ff) {
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_dot<false, true><<<vg, kRedThreads, 0, st>>>(r, z, nullptr, len, nrhs, s, partials, kOpRz, ipart); }
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_update_p_ff<<<vg, kRedThreads, 0, st>>>(p, z, ps, mat->ff_k, len, nrhs, s, ipart); }
    } else {
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_dot<false><<<vg, kRedThreads, 0, st>>>(r, z, nullptr, len, nrhs, s, partials, kOpRz); }
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_update_p<<<vg, kRedThreads, 0, st>>>(p, z, len, s); }
    }
    if ((it + 1) % poll == 0) {
      GS_CUDA(cudaMemcpyAsync(h_conv, &s->all_conv, 4, cudaMemcpyDeviceToHost, st));
      GS_CUDA(cudaStreamSynchronize(st));
      if (*h_conv) break;
    }
  }
  GS_CUDA(cudaGetLastError());
  PcgScalars hs;
  GS_CUDA(cudaMemcpyAsync(&hs, s, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  bool all = true;
  for (int k = 0; k < nrhs; ++k) {
    if (iters) iters[k] = hs.iters[k];
    if (rel_res) rel_res[k] = hs.bnorm2[k] > 0 ? std::sqrt(hs.rr[k] / hs.bnorm2[k]) : 0.0;
    all = all && hs.conv[k];
  }
  int flags = 0;
  GS_TRY(ctx->take_flags(&flags));
  if (hs.flags) return status_from_flags(hs.flags);
  if (flags) return status_from_flags(flags);
  if (!all) {
    set_error("gs_pcg_solve: not converged in %d iterations", max_iter);
    return GS_ERR_MAXITER;
  }
  return GS_OK;
}
