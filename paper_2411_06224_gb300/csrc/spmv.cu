// Symmetric block SpMV on the stored diagonal + upper blocks (Sec. 5.3).
//
// GS_SPMV_SRBK follows Alg. SRBK: one thread per stored block (rows sorted),
// H x_j is reduced per row with the warp head-segmented reduction and
// finished with one atomic per segment head; off-diagonal blocks add
// H^T x_b to y_j atomically.  y is zeroed first.
//
// GS_SPMV_ROW gathers each row instead: y_r = sum_{c >= r} A_rc x_c +
// sum_{c < r} A_cr^T x_c, the second sum reading the same stored blocks
// through a per-row list of transposed references (4-byte indices, built
// once per matrix).  1, 2, 4 or 8 lanes share a row (GS_TUNE_SPMV_LANES) and
// reduce in a fixed order, so results are bit-reproducible and need no
// atomics or zeroing.  Rows are taken longest first within windows of
// consecutive rows (GS_TUNE_SPMV_WINDOW), so the warps see rows of equal
// length while the rows in flight stay neighbours in the mesh, and by
// default a persistent grid's warps take the next rows from a counter
// (GS_TUNE_SPMV_WS).
//
// On GB300 both are bound by FP64 FMA throughput (18 FMA per stored block
// per right-hand side against 80 bytes per block read once for all RHS).
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>

#include "common.cuh"
#include "primitives.cuh"

namespace gs {

template <int kR>
__global__ void __launch_bounds__(256) k_spmv_srbk(const int32_t* __restrict__ rid, const int32_t* __restrict__ cid,
                                                   const double* __restrict__ au, int64_t nnzb, int64_t stride,
                                                   int nrhs, const double* __restrict__ x, double* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lane = threadIdx.x & 31;
  bool in = i < nnzb;
  int32_t b = in ? rid[i] : -1;
  int32_t bp = (in && i > 0) ? rid[i - 1] : -1;
  int32_t j = in ? cid[i] : 0;
  bool head = lane == 0 || bp != b || !in;
  unsigned hm = __ballot_sync(kFull, head);
  int send = segment_end(hm, lane);
  double H[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) H[k] = in ? au[i * 9 + k] : 0.0;
  for (int r0 = 0; r0 < nrhs; r0 += kR) {
    double v[kR * 3];
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      const int r = r0 + q;
      double xj0 = 0, xj1 = 0, xj2 = 0;
      if (in && r < nrhs) {
        const double* xr = x + r * stride;
        xj0 = xr[3 * j], xj1 = xr[3 * j + 1], xj2 = xr[3 * j + 2];
        if (b != j) {
          double xb0 = xr[3 * b], xb1 = xr[3 * b + 1], xb2 = xr[3 * b + 2];
          double* yr = y + r * stride + 3 * j;
          atomicAdd(yr + 0, fma(H[6], xb2, fma(H[3], xb1, H[0] * xb0)));
          atomicAdd(yr + 1, fma(H[7], xb2, fma(H[4], xb1, H[1] * xb0)));
          atomicAdd(yr + 2, fma(H[8], xb2, fma(H[5], xb1, H[2] * xb0)));
        }
      }
      v[3 * q + 0] = fma(H[2], xj2, fma(H[1], xj1, H[0] * xj0));
      v[3 * q + 1] = fma(H[5], xj2, fma(H[4], xj1, H[3] * xj0));
      v[3 * q + 2] = fma(H[8], xj2, fma(H[7], xj1, H[6] * xj0));
    }
    head_segmented_reduce<kR * 3>(v, lane, send);
    if (head && in) {
#pragma unroll
      for (int q = 0; q < kR; ++q) {
        if (r0 + q < nrhs) {
          double* yr = y + (r0 + q) * stride + 3 * b;
          atomicAdd(yr + 0, v[3 * q + 0]);
          atomicAdd(yr + 1, v[3 * q + 1]);
          atomicAdd(yr + 2, v[3 * q + 2]);
        }
      }
    }
  }
}

// kLanes lanes per block row; each lane strides over the row's entries
// (its upper blocks first, then its transposed references) and keeps kR
// right-hand sides in registers, so every block is loaded once per kR RHS.
// One thread group's share of the product: thread t of the walk over the
// row order (kLanes threads per row).
template <int kLanes, int kR>
__device__ __forceinline__ void spmv_row_group(int64_t t, const int32_t* __restrict__ row_order,
                                               const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cid,
                                               const int32_t* __restrict__ lo_ptr, const int32_t* __restrict__ lo_idx,
                                               const int32_t* __restrict__ lo_col, const double* __restrict__ au,
                                               int32_t n, int64_t stride, int nrhs, const double* __restrict__ x,
                                               double* __restrict__ y) {
  const int32_t slot = (int32_t)(t / kLanes);
  int sub = threadIdx.x % kLanes;
  bool in = slot < n;
  // rows are taken longest first (stable), so the rows sharing a warp have
  // equal lengths and no lane idles while the FP64 pipe issues for the warp
  const int32_t row = in ? row_order[slot] : 0;
  int32_t u0 = 0, u1 = 0, l0 = 0, l1 = 0;
  if (in) {
    u0 = row_ptr[row], u1 = row_ptr[row + 1];
    l0 = lo_ptr[row], l1 = lo_ptr[row + 1];
  }
  const int32_t nu = u1 - u0, total = nu + (l1 - l0);
  for (int r0 = 0; r0 < nrhs; r0 += kR) {
    double acc[kR * 3];
#pragma unroll
    for (int k = 0; k < kR * 3; ++k) acc[k] = 0.0;
    for (int32_t e = sub; e < total; e += kLanes) {
      bool upper = e < nu;
      int64_t blk;
      int32_t col;
      if (upper) {
        blk = u0 + e;
        col = cid[blk];
      } else {
        blk = lo_idx[l0 + e - nu];
        col = lo_col[l0 + e - nu];
      }
      double H[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) H[k] = au[blk * 9 + k];
      if (!upper) {  // use the transpose
        double t1 = H[1], t2 = H[2], t5 = H[5];
        H[1] = H[3], H[2] = H[6], H[5] = H[7];
        H[3] = t1, H[6] = t2, H[7] = t5;
      }
#pragma unroll
      for (int q = 0; q < kR; ++q) {
        if (r0 + q < nrhs) {
          const double* xr = x + (r0 + q) * stride + 3 * col;
          const double x0 = xr[0], x1 = xr[1], x2 = xr[2];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double a = acc[3 * q + c];
            a = fma(H[3 * c + 0], x0, a);
            a = fma(H[3 * c + 1], x1, a);
            acc[3 * q + c] = fma(H[3 * c + 2], x2, a);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kR * 3; ++k) {
#pragma unroll
      for (int o = kLanes / 2; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(kFull, acc[k], o, kLanes);
    }
    if (in && sub == 0) {
#pragma unroll
      for (int q = 0; q < kR; ++q)
        if (r0 + q < nrhs) {
          double* yr = y + (r0 + q) * stride + 3 * row;
          yr[0] = acc[3 * q + 0], yr[1] = acc[3 * q + 1], yr[2] = acc[3 * q + 2];
        }
    }
  }
}

template <int kLanes, int kR>
__global__ void __launch_bounds__(256) k_spmv_row(const int32_t* __restrict__ row_order,
                                                  const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cid,
                                                  const int32_t* __restrict__ lo_ptr,
                                                  const int32_t* __restrict__ lo_idx,
                                                  const int32_t* __restrict__ lo_col, const double* __restrict__ au,
                                                  int32_t n, int64_t stride, int nrhs, const double* __restrict__ x,
                                                  double* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;  // every RHS of the solve has converged
  spmv_row_group<kLanes, kR>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, row_order, row_ptr, cid, lo_ptr, lo_idx,
                             lo_col, au, n, stride, nrhs, x, y);
}

// Work-stealing form (GS_TUNE_SPMV_WS): a persistent grid whose warps take
// the next 32 threads' worth of rows of the row order from a counter, so the
// rows in flight stay one contiguous stretch of the order and no SM idles in
// a tail of long rows.  Capped at the one-pass kernel's 88 registers, so two
// blocks per SM leave the same room to other streams' kernels.
template <int kLanes, int kR>
__global__ void __maxnreg__(88) k_spmv_row_ws(const int32_t* __restrict__ row_order,
                                              const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cid,
                                              const int32_t* __restrict__ lo_ptr, const int32_t* __restrict__ lo_idx,
                                              const int32_t* __restrict__ lo_col, const double* __restrict__ au,
                                              int32_t n, int64_t stride, int nrhs, const double* __restrict__ x,
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
    spmv_row_group<kLanes, kR>((int64_t)c * 32 + lane, row_order, row_ptr, cid, lo_ptr, lo_idx, lo_col, au, n,
                               stride, nrhs, x, y);
  }
}

__global__ void k_lower_keys(const int32_t* __restrict__ rid, const int32_t* __restrict__ cid, int64_t nnzb,
                             uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnzb) return;
  bool off = rid[i] != cid[i];
  key[i] = off ? (uint32_t)cid[i] : 0xffffffffu;  // transposed entry lands in row cid
  val[i] = (uint32_t)i;
}

__global__ void k_lower_fill(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sval,
                             const int32_t* __restrict__ rid, int64_t m, int32_t n, int32_t* __restrict__ lo_ptr,
                             int32_t* __restrict__ lo_idx, int32_t* __restrict__ lo_col) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e > m) return;
  int32_t r_here = (e < m) ? (int32_t)skey[e] : n;
  int32_t r_prev = (e > 0) ? (int32_t)skey[e - 1] : -1;
  for (int32_t r = r_prev + 1; r <= r_here; ++r) lo_ptr[r] = (int32_t)e;
  if (e < m) {
    lo_idx[e] = (int32_t)sval[e];
    lo_col[e] = rid[sval[e]];
  }
}

// Sort key of each row for the row order: entries counted from the longest
// possible, so an ascending (stable) radix sort lists long rows first.
// shift < 0: one global order.  Otherwise rows are ordered by window
// (r >> shift) first and by length only inside it: the warps still see rows
// of equal length, and the rows in flight stay neighbours in the mesh, so
// their x gathers and transposed blocks hit L2.
__global__ void k_row_len_keys(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ lo_ptr, int32_t n,
                               int shift, uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
  int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t len = (uint32_t)(row_ptr[r + 1] - row_ptr[r] + lo_ptr[r + 1] - lo_ptr[r]);
  key[r] = shift < 0 ? 0xffffffffu - len : ((uint32_t)(r >> shift) << 16) | (0xffffu - min(len, 0xffffu));
  val[r] = (uint32_t)r;
}

// Number of valid (non-sentinel) keys in a sorted key array.
__global__ void k_count_valid(const uint32_t* __restrict__ k, int64_t nz, int32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nz) return;
  bool v = k[i] != 0xffffffffu;
  bool vn = (i + 1 < nz) && (k[i + 1] != 0xffffffffu);
  if (v && !vn) *out = (int32_t)(i + 1);
}

// Build the per-row transposed references once (the radix sort is stable,
// so each row's references stay in ascending source row).
int ensure_lower(gs_ctx ctx, gs_mat m) {
  if (m->lo_ptr) return GS_OK;
  cudaStream_t st = ctx->stream;
  const int64_t nz = m->nnzb;
  const int64_t cap = std::max<int64_t>(nz, 1);
  uint32_t *k_in, *k_out, *v_in, *v_out;
  int32_t* d_cnt;
  GS_TRY(ctx->scratch_buf(kSlotSortKeysIn, cap * 4, (void**)&k_in));
  GS_TRY(ctx->scratch_buf(kSlotSortKeysOut, cap * 4, (void**)&k_out));
  GS_TRY(ctx->scratch_buf(kSlotSortValsIn, cap * 4, (void**)&v_in));
  GS_TRY(ctx->scratch_buf(kSlotSortValsOut, cap * 4, (void**)&v_out));
  GS_TRY(ctx->scratch_buf(kSlotReduce, 64, (void**)&d_cnt));
  GS_CUDA(cudaMemsetAsync(d_cnt, 0, 4, st));
  if (nz > 0) {
    { GS_PROF(ctx, GS_K_OTHER); k_lower_keys<<<ceil_div(nz, 256), 256, 0, st>>>(m->rid, m->cid, nz, k_in, v_in); }
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, k_in, k_out, v_in, v_out, (int64_t)nz, 0, 32, st);
    void* temp;
    GS_TRY(ctx->scratch_buf(kSlotSortTemp, tb, &temp));
    { GS_PROF(ctx, GS_K_LIBPRIM); GS_CUDA(cub::DeviceRadixSort::SortPairs(temp, tb, k_in, k_out, v_in, v_out, (int64_t)nz, 0, 32, st)); }
    { GS_PROF(ctx, GS_K_OTHER); k_count_valid<<<ceil_div(nz, 256), 256, 0, st>>>(k_out, nz, d_cnt); }
  }
  GS_CUDA(cudaMemcpyAsync(ctx->h_pinned, d_cnt, 4, cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  const int64_t n_off = ctx->h_pinned[0];
  GS_TRY(ctx->alloc((void**)&m->lo_ptr, (size_t)(m->n + 1) * 4));
  GS_TRY(ctx->alloc((void**)&m->lo_idx, (size_t)std::max<int64_t>(n_off, 1) * 4));
  GS_TRY(ctx->alloc((void**)&m->lo_col, (size_t)std::max<int64_t>(n_off, 1) * 4));
  { GS_PROF(ctx, GS_K_OTHER); k_lower_fill<<<ceil_div(n_off + 1, 256), 256, 0, st>>>(k_out, v_out, m->rid, n_off, m->n, m->lo_ptr, m->lo_idx,
                                                         m->lo_col); }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// Row order of the row-gather SpMV for the context's window
// (GS_TUNE_SPMV_WINDOW): by total entries, longest first, ties by row index,
// inside windows of consecutive rows (0: over all rows).  Rebuilt when the
// window changes.
int ensure_row_order(gs_ctx ctx, gs_mat m) {
  GS_TRY(ensure_lower(ctx, m));
  const int window = ctx->tune[GS_TUNE_SPMV_WINDOW];
  if (m->row_order && m->row_order_window == window) return GS_OK;
  cudaStream_t st = ctx->stream;
  int shift = -1;
  if (window > 0) {
    int bits = 0;  // rows need bits - 16 bits of window index above the 16 length bits
    while (bits < 31 && (1LL << bits) < (int64_t)m->n) ++bits;
    shift = 0;
    while ((1 << shift) < window) ++shift;
    shift = std::max(shift, bits - 16);
  }
  if (!m->row_order) GS_TRY(ctx->alloc((void**)&m->row_order, (size_t)std::max(m->n, 1) * 4));
  {
    uint32_t *lk_in, *lk_out, *lv_in;
    GS_TRY(ctx->scratch_buf(kSlotSortKeysIn, (size_t)m->n * 4 + 16, (void**)&lk_in));
    GS_TRY(ctx->scratch_buf(kSlotSortKeysOut, (size_t)m->n * 4 + 16, (void**)&lk_out));
    GS_TRY(ctx->scratch_buf(kSlotSortValsIn, (size_t)m->n * 4 + 16, (void**)&lv_in));
    { GS_PROF(ctx, GS_K_OTHER); k_row_len_keys<<<ceil_div(m->n, 256), 256, 0, st>>>(m->row_ptr, m->lo_ptr, m->n, shift, lk_in, lv_in); }
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, lk_in, lk_out, lv_in, (uint32_t*)m->row_order, m->n, 0, 32, st);
    void* temp;
    GS_TRY(ctx->scratch_buf(kSlotSortTemp, tb, &temp));
    { GS_PROF(ctx, GS_K_LIBPRIM); GS_CUDA(cub::DeviceRadixSort::SortPairs(temp, tb, lk_in, lk_out, lv_in, (uint32_t*)m->row_order, m->n, 0, 32, st)); }
  }
  GS_CUDA(cudaGetLastError());
  m->row_order_window = window;
  return GS_OK;
}

// y = A x on the context stream (no validation; used inside PCG).
int spmv_launch(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, int variant) {
  return spmv_launch_skip(ctx, m, x, y, nrhs, variant, nullptr);
}

// The same, but the row kernels return at once while *skip (device) is set:
// PCG passes its all-converged word, so the iterations between the last
// convergence and the host's next poll cost no SpMV work.
int spmv_launch_skip(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, int variant, const int* skip) {
  cudaStream_t st = ctx->stream;
  const int64_t stride = 3LL * m->n;
  if (variant == GS_SPMV_ROW_FF) return spmv_ff_launch(ctx, m, x, y, nrhs, skip);
  if (variant == GS_SPMV_SRBK) {
    GS_CUDA(cudaMemsetAsync(y, 0, (size_t)nrhs * stride * sizeof(double), st));
    if (m->nnzb > 0)
      { GS_PROF(ctx, GS_K_SPMV); k_spmv_srbk<4><<<ceil_div(m->nnzb, 256), 256, 0, st>>>(m->rid, m->cid, m->au, m->nnzb, stride, nrhs, x, y); }
  } else {
    GS_TRY(ensure_row_order(ctx, m));
    // lanes per block row (GS_TUNE_SPMV_LANES); 8 lanes keep 4 RHS per pass
    const int lanes = ctx->tune[GS_TUNE_SPMV_LANES];
    const int64_t threads = (int64_t)m->n * lanes;
    const int grid = ceil_div(threads, 256);
#define GS_ROW_ARGS m->row_order, m->row_ptr, m->cid, m->lo_ptr, m->lo_idx, m->lo_col, m->au, m->n, stride, nrhs, x, y
    if (ctx->tune[GS_TUNE_SPMV_WS] && ctx->sm_count > 0) {  // work stealing over a persistent grid
      int* counter = ctx->d_flags + kSpmvCounterWord;
      GS_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
      const int wgrid = std::min(grid, 2 * ctx->sm_count);  // 88 registers: two blocks of 256 per SM
      GS_PROF(ctx, GS_K_SPMV);
      if (nrhs == 1) {
        if (lanes == 8) k_spmv_row_ws<8, 1><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
        else if (lanes == 2) k_spmv_row_ws<2, 1><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
        else if (lanes == 1) k_spmv_row_ws<1, 1><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
        else k_spmv_row_ws<4, 1><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
      } else {
        if (lanes == 8) k_spmv_row_ws<8, 4><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
        else if (lanes == 2) k_spmv_row_ws<2, 8><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
        else if (lanes == 1) k_spmv_row_ws<1, 8><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
        else k_spmv_row_ws<4, 8><<<wgrid, 256, 0, st>>>(GS_ROW_ARGS, counter, skip);
      }
    } else if (nrhs == 1) {
      if (lanes == 8) { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<8, 1><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
      else if (lanes == 2) { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<2, 1><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
      else if (lanes == 1) { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<1, 1><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
      else { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<4, 1><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
    } else {
      if (lanes == 8) { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<8, 4><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
      else if (lanes == 2) { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<2, 8><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
      else if (lanes == 1) { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<1, 8><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
      else { GS_PROF(ctx, GS_K_SPMV); k_spmv_row<4, 8><<<grid, 256, 0, st>>>(GS_ROW_ARGS, skip); }
    }
#undef GS_ROW_ARGS
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs

extern "C" int gs_spmv(gs_ctx ctx, gs_mat m, const double* x, double* y, int32_t nrhs, int32_t variant) {
  GS_CHECK(ctx && m, GS_ERR_INVALID, "gs_spmv: null context or matrix");
  GS_CHECK(nrhs >= 1, GS_ERR_INVALID, "gs_spmv: nrhs %d", nrhs);
  GS_CHECK(x && y && x != y, GS_ERR_INVALID, "gs_spmv: null or aliased vectors");
  GS_CHECK(variant == GS_SPMV_SRBK || variant == GS_SPMV_ROW || variant == GS_SPMV_ROW_FF, GS_ERR_INVALID,
           "gs_spmv: variant %d", variant);
  GS_CUDA(cudaSetDevice(ctx->device));
  return gs::spmv_launch(ctx, m, x, y, nrhs, variant);
}
