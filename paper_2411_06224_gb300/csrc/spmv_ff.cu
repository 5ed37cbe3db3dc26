// Symmetric block SpMV (Sec. 5.3) in float-float arithmetic on the FP32 units
// (GS_SPMV_ROW_FF).
//
// On this part the FP64 pipe issues 2 FMA per clock per SM against 128 FP32
// operations, and the FP64 row SpMV (spmv.cu) is bound by it.  Here every
// product and sum runs in FP32 as an error-free transformation, so the result
// keeps about 48 significant bits:
//
//   * The matrix is scaled once: row i gets k_i = ceil(E_i / 2), with 2^E_i
//     above the largest entry of block row i (both triangles), and the stored
//     block (r, c) becomes A_rc 2^-(k_r + k_c).  For a symmetric matrix
//     |A_rc| <= min(2^E_r, 2^E_c) <= 2^(k_r + k_c), so every scaled entry is
//     below 1 in magnitude, and one stored copy serves both triangles.  Each
//     entry is kept as (hi, lo) = (rn(a), rn(a - hi)).
//   * x is scaled per right-hand side: x~_j = x_j 2^(k_j - K - F), K = max k,
//     2^F above the RHS's largest |x|, so |x~| <= 1, and split from its bit
//     pattern without FP64 instructions (ff_split_bits: hi = x~ cut to 24
//     significant bits, lo = the rest rounded to 24), node-major across the
//     right-hand sides so that a column's values for all of them are one
//     contiguous gather.  PCG writes its direction vector in this form as it
//     updates it (pcg.cu); other callers go through two passes here
//     (exponent maximum, split).
//   * Each term a x = ah xh + (ah xl + al xh) + al xl: ah xh is taken exactly
//     as p + e (p = ah * xh rounded, e = fma(ah, xh, -p)), the row sum of the
//     p runs through Knuth's two-sum (s, err), and the small parts
//     err + e + ah xl + al xh gather in a second float; al xl (below 2^-47 of
//     the term) is dropped.  y_r = 2^(k_r + K + F) (S + L), added in FP64.
//
// Error per output (u = 2^-24, m = terms of the row, 3 per stored block of
// either triangle): the two-sum chain is exact; the small-part float sum has
// at most 3m + 1 roundings over terms whose magnitudes add up to at most
// (m + 4) u sum|t| (|err| <= u |partial sum|, |e| <= u |t|, |ah xl| <= 2u |t|,
// |al xh| <= u |t|); the splits (2^-48 |a|, 2^-47 |x|), the dropped al xl and
// the final FP64 addition add at most 6 u^2 sum|t|:
//   |dy_i| <= ((3m+1)(m+4) + 6) u^2 (|A||x|)_i.
// Terms below 2^-100 of the scale lose their low parts (an absolute error of
// at most 2^-126 each in the scaled units).
//
// The row walk, lanes per row, windowed row order and work stealing are the
// FP64 row kernel's (spmv.cu); lanes combine their pairs in a fixed order,
// so results are bit-reproducible.
#include <algorithm>

#include "common.cuh"
#include "ff.cuh"
#include "primitives.cuh"

namespace gs {

// ---------------------------------------------------------------- matrix preparation
__global__ void k_ff_row_exp(const int32_t* __restrict__ rid, const int32_t* __restrict__ cid,
                             const double* __restrict__ au, int64_t nnzb, int32_t* __restrict__ rowE) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nnzb) return;
  int e = kExpNone;
#pragma unroll
  for (int q = 0; q < 9; ++q) e = max(e, ex_bound(au[b * 9 + q]));
  if (e == kExpNone) return;
  atomicMax(&rowE[rid[b]], e);
  atomicMax(&rowE[cid[b]], e);
}

// k_i = ceil(E_i / 2) (0 for an empty row) and K = max k_i into k[n].
__global__ void k_ff_half(int32_t* __restrict__ k, int32_t n) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e = k[i];
  const int h = e == kExpNone ? 0 : (e + 1) >> 1;  // arithmetic shift: ceil for negative e too
  k[i] = h;
  atomicMax(&k[n], h);
}

__global__ void k_ff_blocks(const int32_t* __restrict__ rid, const int32_t* __restrict__ cid,
                            const double* __restrict__ au, int64_t nnzb, const int32_t* __restrict__ k,
                            float2* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb * 9) return;
  const int64_t b = t / 9;
  out[t] = ff_split_scaled(au[t], -(k[rid[b]] + k[cid[b]]));
}

__global__ void k_ff_minus_K(int32_t* __restrict__ k, int32_t n) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) k[i] -= k[n];
}

int ensure_ff(gs_ctx ctx, gs_mat m) {
  if (m->au_ff) return GS_OK;
  cudaStream_t st = ctx->stream;
  const int64_t nz = m->nnzb;
  GS_TRY(ctx->alloc((void**)&m->ff_k, (size_t)(m->n + 1) * 4));
  GS_TRY(ctx->alloc((void**)&m->au_ff, (size_t)std::max<int64_t>(nz, 1) * 9 * sizeof(float2)));
  GS_CUDA(cudaMemsetAsync(m->ff_k, 0x80, (size_t)m->n * 4, st));  // kExpNone
  GS_CUDA(cudaMemsetAsync(m->ff_k + m->n, 0x80, 4, st));
  {
    GS_PROF(ctx, GS_K_OTHER);
    if (nz > 0) k_ff_row_exp<<<ceil_div(nz, 256), 256, 0, st>>>(m->rid, m->cid, m->au, nz, m->ff_k);
  }
  // rows that no block touched still hold kExpNone: they read as empty
  { GS_PROF(ctx, GS_K_OTHER); k_ff_half<<<ceil_div(std::max(m->n, 1), 256), 256, 0, st>>>(m->ff_k, m->n); }
  {
    GS_PROF(ctx, GS_K_OTHER);
    if (nz > 0) k_ff_blocks<<<ceil_div(nz * 9, 256), 256, 0, st>>>(m->rid, m->cid, m->au, nz, m->ff_k, m->au_ff);
  }
  { GS_PROF(ctx, GS_K_OTHER); k_ff_minus_K<<<ceil_div(std::max(m->n, 1), 256), 256, 0, st>>>(m->ff_k, m->n); }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// ---------------------------------------------------------------- splitting x
// F[k] = max over RHS k of ex_bound(x); F zeroed to kExpNone first.
__global__ void __launch_bounds__(256) k_ff_maxexp(const double* __restrict__ x, int64_t len,
                                                   int* __restrict__ F) {
  const int k = blockIdx.y;
  int e = kExpNone;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    e = max(e, ex_bound(x[k * len + i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(kFull, e, o));
  if ((threadIdx.x & 31) == 0 && e != kExpNone) atomicMax(&F[k], e);
}

// xs node-major across right-hand sides: xs[(node * nrhs + k) * 3 + c].
__global__ void __launch_bounds__(256) k_ff_split(const double* __restrict__ x, int64_t len, int nrhs,
                                                  const int32_t* __restrict__ kk, const int* __restrict__ F,
                                                  float2* __restrict__ xs) {
  const int k = blockIdx.y;
  const int f = F[k] == kExpNone ? 0 : F[k];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t node = (uint32_t)i / 3u;
    xs[((int64_t)node * nrhs + k) * 3 + ((uint32_t)i - 3u * node)] = ff_split_bits(x[k * len + i], kk[node] - f);
  }
}

// ---------------------------------------------------------------- the product
// Accumulate the term (ah + al)(xh + xl) into the pair (S, L).  The rounded
// intrinsics keep the compiler from contracting or reordering the
// transformations.
__device__ __forceinline__ void ff_term(float ah, float al, float xh, float xl, float& S, float& L) {
  const float p = __fmul_rn(ah, xh);
  const float e = __fmaf_rn(ah, xh, -p);
  const float s = __fadd_rn(S, p);
  const float bp = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  S = s;
  L = __fadd_rn(L, __fadd_rn(err, e));
  L = __fmaf_rn(ah, xl, L);
  L = __fmaf_rn(al, xh, L);
}

// (S, L) += (S2, L2): two-sum of the large parts, the rest gathered in L.
__device__ __forceinline__ void ff_merge(float& S, float& L, float S2, float L2) {
  const float s = __fadd_rn(S, S2);
  const float bp = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(S2, bp));
  S = s;
  L = __fadd_rn(L, __fadd_rn(L2, err));
}

// f * 2^e as a double, built from f's bit pattern (no conversion
// instruction; on this part conversions run on the FP64 pipe).  A zero or
// subnormal f gives 0; e keeps the result inside the double range here.
__device__ __forceinline__ double f32_times_pow2(float f, int e) {
  const unsigned b = __float_as_uint(f);
  const int fe = (int)((b >> 23) & 0xffu);
  if (fe == 0) return 0.0;
  const int de = min(max(fe - 127 + 1023 + e, 1), 2046);
  const unsigned hi = (b & 0x80000000u) | ((unsigned)de << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// One thread's share of the product for thread t of the walk over the row
// order (kLanes threads per row).  kSplit = false: the row's lanes stride over
// its blocks and merge their pairs at the end (any RHS count).  kSplit = true:
// every lane walks all the row's blocks for its own groups of kR right-hand
// sides (groups sub, sub + kLanes, ...), so the lanes of a row read the same
// block (one broadcast load) and need no merge; fewer RHS per thread leaves
// more warps resident to cover the gathers' latency.
template <int kLanes, int kR, bool kSplit>
__device__ __forceinline__ void spmv_ff_row_group(int64_t t, const int32_t* __restrict__ row_order,
                                                  const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ cid, const int32_t* __restrict__ lo_ptr,
                                                  const int32_t* __restrict__ lo_idx,
                                                  const int32_t* __restrict__ lo_col, const float2* __restrict__ au,
                                                  const int32_t* __restrict__ kk, int32_t n, int64_t stride, int nrhs,
                                                  const float2* __restrict__ xs, const int* __restrict__ F,
                                                  double* __restrict__ y) {
  const int32_t slot = (int32_t)(t / kLanes);
  const int sub = threadIdx.x % kLanes;
  const bool in = slot < n;
  const int32_t row = in ? row_order[slot] : 0;
  int32_t u0 = 0, u1 = 0, l0 = 0, l1 = 0;
  if (in) {
    u0 = row_ptr[row], u1 = row_ptr[row + 1];
    l0 = lo_ptr[row], l1 = lo_ptr[row + 1];
  }
  const int32_t nu = u1 - u0, total = nu + (l1 - l0);
  const int e_first = kSplit ? 0 : sub, e_step = kSplit ? 1 : kLanes;
  const int r_first = kSplit ? sub * kR : 0, r_step = kSplit ? kLanes * kR : kR;
  // the operand's pairs are 16-byte aligned when the RHS count and kR are even
  const bool vec = kR % 2 == 0 && (nrhs & 1) == 0;
  for (int r0 = r_first; r0 < nrhs; r0 += r_step) {
    const int nh = min(kR, nrhs - r0);  // right-hand sides in this pass
    float S[kR * 3], L[kR * 3];
#pragma unroll
    for (int q = 0; q < kR * 3; ++q) S[q] = 0.f, L[q] = 0.f;
    for (int32_t e = e_first; e < total; e += e_step) {
      const bool upper = e < nu;
      int64_t blk;
      int32_t col;
      if (upper) {
        blk = u0 + e;
        col = cid[blk];
      } else {
        blk = lo_idx[l0 + e - nu];
        col = lo_col[l0 + e - nu];
      }
      float2 H[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) H[q] = au[blk * 9 + q];
      if (!upper) {  // use the transpose
        float2 t1 = H[1], t2 = H[2], t5 = H[5];
        H[1] = H[3], H[2] = H[6], H[5] = H[7];
        H[3] = t1, H[6] = t2, H[7] = t5;
      }
      // the column's operand for this pass's right-hand sides is one
      // contiguous stretch (node-major); two RHS at a time in 16-byte loads
      const float2* xb = xs + ((int64_t)col * nrhs + r0) * 3;
#pragma unroll
      for (int q = 0; q < kR; q += 2) {
        float2 xv[6];
        if (vec) {
          if (q < nh) {
            const float4* x4 = reinterpret_cast<const float4*>(xb + 3 * q);
            const float4 a = x4[0], b = x4[1], c = x4[2];
            xv[0] = make_float2(a.x, a.y), xv[1] = make_float2(a.z, a.w), xv[2] = make_float2(b.x, b.y);
            xv[3] = make_float2(b.z, b.w), xv[4] = make_float2(c.x, c.y), xv[5] = make_float2(c.z, c.w);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 6; ++i)
            if (q + i / 3 < nh && (q + i / 3) < kR) xv[i] = xb[3 * q + i];
        }
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
          const int qi = q + qq;
          if (qi < kR && qi < nh) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              ff_term(H[3 * c + 0].x, H[3 * c + 0].y, xv[3 * qq].x, xv[3 * qq].y, S[3 * qi + c], L[3 * qi + c]);
              ff_term(H[3 * c + 1].x, H[3 * c + 1].y, xv[3 * qq + 1].x, xv[3 * qq + 1].y, S[3 * qi + c],
                      L[3 * qi + c]);
              ff_term(H[3 * c + 2].x, H[3 * c + 2].y, xv[3 * qq + 2].x, xv[3 * qq + 2].y, S[3 * qi + c],
                      L[3 * qi + c]);
            }
          }
        }
      }
    }
    if (!kSplit) {
#pragma unroll
      for (int q = 0; q < kR * 3; ++q) {
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) {
          const float S2 = __shfl_xor_sync(kFull, S[q], o, kLanes);
          const float L2 = __shfl_xor_sync(kFull, L[q], o, kLanes);
          ff_merge(S[q], L[q], S2, L2);
        }
      }
    }
    if (in && (kSplit || sub == 0)) {
      const int kr = kk[row] + 2 * kk[n];  // k_row + K
#pragma unroll
      for (int q = 0; q < kR; ++q)
        if (q < nh) {
          const int f = F[r0 + q];
          double* yr = y + (r0 + q) * stride + 3 * (int64_t)row;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            yr[c] = f == kExpNone ? 0.0
                                  : f32_times_pow2(S[3 * q + c], kr + f) + f32_times_pow2(L[3 * q + c], kr + f);
        }
    }
  }
}

// Resident blocks of 256 threads per SM each shape is compiled for (the
// register cap follows): 2 for 8 RHS per thread, 3 for 4, 4 for 2 or 1.
template <int kR, bool kSplit>
constexpr int ff_blocks_per_sm() {
  return kR >= 8 ? 2 : (kR == 4 ? 3 : 4);
}

// Work-stealing form (the default shape of the row SpMVs): a persistent grid
// whose warps take the next 32 threads' worth of rows from a counter.
template <int kLanes, int kR, bool kSplit>
__global__ void __launch_bounds__(256, (ff_blocks_per_sm<kR, kSplit>())) k_spmv_ff_ws(const int32_t* __restrict__ row_order,
                                                       const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ cid,
                                                       const int32_t* __restrict__ lo_ptr,
                                                       const int32_t* __restrict__ lo_idx,
                                                       const int32_t* __restrict__ lo_col,
                                                       const float2* __restrict__ au, const int32_t* __restrict__ kk,
                                                       int32_t n, int64_t stride, int nrhs,
                                                       const float2* __restrict__ xs, const int* __restrict__ F,
                                                       double* __restrict__ y, int* __restrict__ counter,
                                                       const int* __restrict__ skip) {
  if (skip && *skip) return;  // every RHS of the solve has converged
  const int lane = threadIdx.x & 31;
  const int64_t chunks = ((int64_t)n * kLanes + 31) / 32;
#pragma unroll 1
  while (true) {
    int c = 0;
    if (lane == 0) c = atomicAdd(counter, 1);
    c = __shfl_sync(kFull, c, 0);
    if (c >= chunks) break;  // whole warp
    spmv_ff_row_group<kLanes, kR, kSplit>((int64_t)c * 32 + lane, row_order, row_ptr, cid, lo_ptr, lo_idx, lo_col,
                                          au, kk, n, stride, nrhs, xs, F, y);
  }
}

// One thread group per row (GS_TUNE_SPMV_WS = 0).
template <int kLanes, int kR, bool kSplit>
__global__ void __launch_bounds__(256, (ff_blocks_per_sm<kR, kSplit>())) k_spmv_ff_row(const int32_t* __restrict__ row_order,
                                                        const int32_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ cid,
                                                        const int32_t* __restrict__ lo_ptr,
                                                        const int32_t* __restrict__ lo_idx,
                                                        const int32_t* __restrict__ lo_col,
                                                        const float2* __restrict__ au, const int32_t* __restrict__ kk,
                                                        int32_t n, int64_t stride, int nrhs,
                                                        const float2* __restrict__ xs, const int* __restrict__ F,
                                                        double* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  spmv_ff_row_group<kLanes, kR, kSplit>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, row_order, row_ptr, cid,
                                        lo_ptr, lo_idx, lo_col, au, kk, n, stride, nrhs, xs, F, y);
}

int ensure_row_order(gs_ctx ctx, gs_mat m);

int spmv_ff_split_launch(gs_ctx ctx, gs_mat m, const float2* xs, const int* F, double* y, int nrhs,
                         const int* skip) {
  cudaStream_t st = ctx->stream;
  GS_TRY(ensure_row_order(ctx, m));
  GS_TRY(ensure_ff(ctx, m));
  const int64_t stride = 3LL * m->n;
  // GS_TUNE_SPMV_FF_RHS = 8: lanes (GS_TUNE_SPMV_LANES) stride over a row's
  // blocks, 8 RHS per pass (4 with 8 lanes).  4, 2 or 1: each lane walks all
  // blocks for its own RHS groups of that size, nrhs / size lanes per row
  // (a power of two, at most 8).
  const int rpp = ctx->tune[GS_TUNE_SPMV_FF_RHS];
  const bool split = rpp < 8 && nrhs > rpp;
  int lanes = ctx->tune[GS_TUNE_SPMV_LANES];
  if (split) {
    lanes = 1;
    while (lanes < 8 && lanes * rpp < nrhs) lanes *= 2;
  }
  const int64_t threads = (int64_t)m->n * lanes;
  const int grid = ceil_div(std::max<int64_t>(threads, 1), 256);
  const bool ws = ctx->tune[GS_TUNE_SPMV_WS] && ctx->sm_count > 0;
  int* counter = ctx->d_flags + kSpmvCounterWord;
  if (ws) GS_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
  const int per_sm = split ? (rpp == 4 ? 3 : 4) : (nrhs == 1 ? 4 : (lanes == 8 ? 3 : 2));  // ff_blocks_per_sm
  const int wgrid = std::min(grid, per_sm * std::max(ctx->sm_count, 1));
#define GS_FF_ARGS \
  m->row_order, m->row_ptr, m->cid, m->lo_ptr, m->lo_idx, m->lo_col, m->au_ff, m->ff_k, m->n, stride, nrhs, xs, F, y
#define GS_FF_LAUNCH(L, R, SPLIT)                                                              \
  do {                                                                                         \
    if (ws)                                                                                    \
      k_spmv_ff_ws<L, R, SPLIT><<<wgrid, 256, 0, st>>>(GS_FF_ARGS, counter, skip);            \
    else                                                                                       \
      k_spmv_ff_row<L, R, SPLIT><<<grid, 256, 0, st>>>(GS_FF_ARGS, skip);                     \
  } while (0)
  {
    GS_PROF(ctx, GS_K_SPMV);
    if (split) {
      if (rpp == 4) {
        if (lanes == 2) GS_FF_LAUNCH(2, 4, true);
        else if (lanes == 4) GS_FF_LAUNCH(4, 4, true);
        else GS_FF_LAUNCH(8, 4, true);
      } else if (rpp == 2) {
        if (lanes == 2) GS_FF_LAUNCH(2, 2, true);
        else if (lanes == 4) GS_FF_LAUNCH(4, 2, true);
        else GS_FF_LAUNCH(8, 2, true);
      } else {
        if (lanes == 2) GS_FF_LAUNCH(2, 1, true);
        else if (lanes == 4) GS_FF_LAUNCH(4, 1, true);
        else GS_FF_LAUNCH(8, 1, true);
      }
    } else if (nrhs == 1) {
      if (lanes == 8) GS_FF_LAUNCH(8, 1, false);
      else if (lanes == 2) GS_FF_LAUNCH(2, 1, false);
      else if (lanes == 1) GS_FF_LAUNCH(1, 1, false);
      else GS_FF_LAUNCH(4, 1, false);
    } else {
      if (lanes == 8) GS_FF_LAUNCH(8, 4, false);
      else if (lanes == 2) GS_FF_LAUNCH(2, 8, false);
      else if (lanes == 1) GS_FF_LAUNCH(1, 8, false);
      else GS_FF_LAUNCH(4, 8, false);
    }
  }
#undef GS_FF_LAUNCH
#undef GS_FF_ARGS
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// y = A x from a plain FP64 x: per-RHS exponent maximum, split into the
// context's scratch, then the product.
int spmv_ff_launch(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, const int* skip) {
  cudaStream_t st = ctx->stream;
  GS_TRY(ensure_ff(ctx, m));
  const int64_t len = 3LL * m->n;
  char* buf = nullptr;
  const size_t xs_bytes = (size_t)nrhs * std::max<int64_t>(len, 1) * sizeof(float2);
  GS_TRY(ctx->scratch_buf(kSlotFFSplit, xs_bytes + 256 + (size_t)nrhs * 4, (void**)&buf));
  float2* xs = (float2*)buf;
  int* F = (int*)(buf + ((xs_bytes + 255) / 256) * 256);
  GS_CUDA(cudaMemsetAsync(F, 0x80, (size_t)nrhs * 4, st));  // kExpNone
  if (len > 0) {
    const int gx = std::max(1, std::min<int>(ceil_div(len, 256 * 8), 4 * std::max(ctx->sm_count, 1)));
    { GS_PROF(ctx, GS_K_OTHER); k_ff_maxexp<<<dim3(gx, nrhs), 256, 0, st>>>(x, len, F); }
    { GS_PROF(ctx, GS_K_OTHER); k_ff_split<<<dim3(gx, nrhs), 256, 0, st>>>(x, len, nrhs, m->ff_k, F, xs); }
  }
  return spmv_ff_split_launch(ctx, m, xs, F, y, nrhs, skip);
}

}  // namespace gs
