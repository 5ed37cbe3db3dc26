// Global Hessian assembly by hash-key reduction (Sec. 5.1-5.2).
//
// FastHashReduction: encode every consumed (row <= col) block with a key,
// radix-sort (key, input index) pairs so duplicates become adjacent, mark
// P[i] = K[i] != K[i+1], take O = ExclusiveSum(P) as each entry's unique-key
// index, and reduce runs with FastSegmentReduction (a warp head-segmented
// reduction; segments crossing a warp boundary finish with atomics).
//
// GB300 choices: keys are packed as (row << b) | col with b the bit width
// of n, which keeps the (row, col) order of the paper's (row << 32) | col
// encoding while shortening the radix sort to 2b bits; values are gathered
// through the sorted index instead of being sorted along (72-byte payloads
// are read once, in the reduction).
#include <cub/device/device_reduce.cuh>

#include "common.cuh"
#include "sort_scan.cuh"
#include "primitives.cuh"

namespace gs {

__global__ void k_encode_keys(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols, int64_t nb,
                              int32_t n, int shift, uint64_t sentinel, uint64_t* __restrict__ keys,
                              uint32_t* __restrict__ idx, int* flags) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int32_t r = rows[i], c = cols[i];
  uint64_t key = sentinel;
  if (r < 0 || r >= n || c < 0 || c >= n) {
    atomicOr(flags, kErrIndex);
  } else if (r <= c) {
    key = ((uint64_t)r << shift) | (uint64_t)c;
  }
  keys[i] = key;
  idx[i] = (uint32_t)i;
}

// P[i] = K[i] != K[i+1]; the last entry closes the final run.
__global__ void k_run_flags(const uint64_t* __restrict__ keys, int64_t nb, int32_t* __restrict__ P) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  P[i] = (i + 1 == nb) ? 1 : (keys[i] != keys[i + 1]);
}

// FastSegmentReduction over the sorted entries.  Thread i holds the block
// of sorted entry i (gathered through idx) and its unique-key index O[i].
// The first entry of each run also writes the decoded (row, col).
__global__ void k_fast_segment_reduce(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx,
                                      const int32_t* __restrict__ O, const double* __restrict__ blocks,
                                      int64_t nb, uint64_t sentinel, int shift, double* __restrict__ R,
                                      int32_t* __restrict__ rid, int32_t* __restrict__ cid,
                                      int32_t* __restrict__ key_of_input) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lane = threadIdx.x & 31;
  bool in = i < nb;
  uint64_t key = in ? keys[i] : sentinel;
  bool valid = in && key != sentinel;
  int32_t b = in ? O[i] : -1;
  int32_t b_prev = (in && i > 0) ? O[i - 1] : -1;
  bool head = (lane == 0) || (b_prev != b);
  double v[9];
  if (valid) {
    const double* src = blocks + (size_t)idx[i] * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = src[k];
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = 0.0;
  }
  unsigned hm = __ballot_sync(kFull, head);
  int send = segment_end(hm, lane);
  head_segmented_reduce<9>(v, lane, send);
  if (in) key_of_input[idx[i]] = valid ? b : -1;  // which stored block each input fed
  if (!valid) return;
  if (b_prev != b) {  // first entry of its run: record the key
    rid[b] = (int32_t)(key >> shift);
    cid[b] = (int32_t)(key & ((1ull << shift) - 1));
  }
  if (!head) return;
  // A segment that began in an earlier warp or continues into the next one
  // is shared between warps: finish it with atomics; otherwise store.
  bool cont_prev = (lane == 0) && (b_prev == b);
  bool cont_next = false;
  if (send == 32) {
    int64_t nxt = i - lane + 32;
    cont_next = nxt < nb && O[nxt] == b;
  }
  double* dst = R + (size_t)b * 9;
  if (cont_prev || cont_next) {
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(dst + k, v[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) dst[k] = v[k];
  }
}

// row_ptr[r] = first stored block of row r (rows without blocks get the
// next row's start); row_ptr[n] = U.
__global__ void k_row_ptr(const int32_t* __restrict__ rid, int64_t U, int32_t n, int32_t* __restrict__ row_ptr) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u > U) return;
  int32_t r_here = (u < U) ? rid[u] : n;
  int32_t r_prev = (u > 0) ? rid[u - 1] : -1;
  for (int32_t r = r_prev + 1; r <= r_here; ++r) row_ptr[r] = (int32_t)u;
}

// Reduce (rows, cols, blocks) to a new matrix.  Shared by gs_assemble and
// the second level of gs_assemble_abd.
int reduce_blocks(gs_ctx ctx, int32_t n, const int32_t* rows, const int32_t* cols, const double* blocks,
                  int64_t nb, gs_mat* out) {
  cudaStream_t st = ctx->stream;
  gs_mat m = new gs_mat_s();
  m->n = n;
  m->owner = ctx;
  const int shift = bits_for(n);
  const uint64_t sentinel = (shift * 2 >= 64) ? ~0ull : ((1ull << (2 * shift)) - 1);
  const int end_bit = 2 * shift;
  uint64_t *k_in = nullptr, *k_out = nullptr;
  uint32_t *i_in = nullptr, *i_out = nullptr;
  int32_t *P = nullptr, *O = nullptr;
  int64_t U = 0;
  auto fail = [&](int s) {
    gs_mat_destroy(m);
    return s;
  };
  if (nb > 0) {
    int s;
    if ((s = ctx->scratch_buf(kSlotSortKeysIn, nb * 8, (void**)&k_in)) ||
        (s = ctx->scratch_buf(kSlotSortKeysOut, nb * 8, (void**)&k_out)) ||
        (s = ctx->scratch_buf(kSlotSortValsIn, nb * 4, (void**)&i_in)) ||
        (s = ctx->scratch_buf(kSlotSortValsOut, nb * 4, (void**)&i_out)) ||
        (s = ctx->scratch_buf(kSlotScan, nb * 8, (void**)&P)))
      return fail(s);
    O = P + nb;
    const int T = 256;
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_encode_keys<<<ceil_div(nb, T), T, 0, st>>>(rows, cols, nb, n, shift, sentinel, k_in, i_in, ctx->d_flags); }
    // radix sort of (key, index) and the exclusive scan of the run flags
    // (sort_scan.cu: hand-written, stable)
    const size_t tb = std::max(radix_sort_temp_bytes(nb), scan_temp_bytes(nb));
    void* temp = nullptr;
    if ((s = ctx->scratch_buf(kSlotSortTemp, tb, &temp))) return fail(s);
    {
      GS_PROF(ctx, GS_K_ASSEMBLE);
      if ((s = radix_sort_pairs(st, k_in, k_out, i_in, i_out, nb, end_bit, temp, tb))) return fail(s);
    }
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_run_flags<<<ceil_div(nb, T), T, 0, st>>>(k_out, nb, P); }
    {
      GS_PROF(ctx, GS_K_ASSEMBLE);
      if ((s = exclusive_scan_i32(st, P, O, nb, temp, tb))) return fail(s);
    }
    // U = distinct keys, minus the sentinel group if present.
    uint64_t* hk = (uint64_t*)ctx->h_pinned;
    int32_t* ho = (int32_t*)(ctx->h_pinned + 4);
    if (cudaMemcpyAsync(hk, k_out + nb - 1, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(ho, O + nb - 1, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("assembly readback failed");
      return fail(GS_ERR_CUDA);
    }
    U = (int64_t)ho[0] + 1 - (hk[0] == sentinel ? 1 : 0);
  }
  int flags = 0;
  GS_TRY(ctx->take_flags(&flags));
  if (flags) return fail(status_from_flags(flags));
  m->nnzb = U;
  int s;
  m->n_input = nb;
  if ((s = ctx->alloc((void**)&m->key_of_input, (size_t)std::max<int64_t>(nb, 1) * 4)) ||
      (s = ctx->alloc((void**)&m->au, (size_t)U * 9 * sizeof(double))) ||
      (s = ctx->alloc((void**)&m->rid, (size_t)U * 4)) || (s = ctx->alloc((void**)&m->cid, (size_t)U * 4)) ||
      (s = ctx->alloc((void**)&m->row_ptr, (size_t)(n + 1) * 4)))
    return fail(s);
  if (U > 0) {
    if (cudaMemsetAsync(m->au, 0, (size_t)U * 9 * sizeof(double), st) != cudaSuccess) return fail(GS_ERR_CUDA);
    const int T = 256;
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_fast_segment_reduce<<<ceil_div(nb, T), T, 0, st>>>(k_out, i_out, O, blocks, nb, sentinel, shift, m->au,
                                                            m->rid, m->cid, m->key_of_input); }
  }
  if (U == 0 && nb > 0 && cudaMemsetAsync(m->key_of_input, 0xff, (size_t)nb * 4, st) != cudaSuccess)
    return fail(GS_ERR_CUDA);
  { GS_PROF(ctx, GS_K_ASSEMBLE); k_row_ptr<<<ceil_div(U + 1, 256), 256, 0, st>>>(m->rid, U, n, m->row_ptr); }
  if (cudaGetLastError() != cudaSuccess) {
    set_error("assembly kernel launch failed");
    return fail(GS_ERR_CUDA);
  }
  *out = m;
  return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" {

int gs_assemble(gs_ctx ctx, int32_t n, const int32_t* rows, const int32_t* cols, const double* blocks,
                int64_t nb, gs_mat* out) {
  GS_CHECK(ctx && out, GS_ERR_INVALID, "gs_assemble: null context or output");
  *out = nullptr;
  GS_CHECK(n > 0 && n < (1 << 30), GS_ERR_INVALID, "gs_assemble: n_block_rows %d out of range", n);
  GS_CHECK(nb >= 0 && nb < (1LL << 31), GS_ERR_INVALID, "gs_assemble: n_blocks %lld out of range", (long long)nb);
  GS_CHECK(nb == 0 || (rows && cols && blocks), GS_ERR_INVALID, "gs_assemble: null input");
  GS_CUDA(cudaSetDevice(ctx->device));
  return reduce_blocks(ctx, n, rows, cols, blocks, nb, out);
}

int gs_mat_info(gs_mat m, int32_t* n, int64_t* nnzb) {
  GS_CHECK(m, GS_ERR_INVALID, "gs_mat_info: null matrix");
  if (n) *n = m->n;
  if (nnzb) *nnzb = m->nnzb;
  return GS_OK;
}

int gs_mat_export(gs_ctx ctx, gs_mat m, int32_t* rid, int32_t* cid, double* au) {
  GS_CHECK(ctx && m, GS_ERR_INVALID, "gs_mat_export: null argument");
  cudaStream_t st = ctx->stream;
  if (m->nnzb == 0) return GS_OK;
  if (rid) GS_CUDA(cudaMemcpyAsync(rid, m->rid, m->nnzb * 4, cudaMemcpyDeviceToDevice, st));
  if (cid) GS_CUDA(cudaMemcpyAsync(cid, m->cid, m->nnzb * 4, cudaMemcpyDeviceToDevice, st));
  if (au) GS_CUDA(cudaMemcpyAsync(au, m->au, m->nnzb * 72, cudaMemcpyDeviceToDevice, st));
  return GS_OK;
}

int gs_mat_destroy(gs_mat m) {
  if (!m) return GS_OK;
  gs_ctx c = m->owner;
  c->release(m->au);
  c->release(m->rid);
  c->release(m->cid);
  c->release(m->row_ptr);
  c->release(m->lo_ptr);
  c->release(m->lo_idx);
  c->release(m->lo_col);
  c->release(m->au32);
  c->release(m->au_ff);
  c->release(m->ff_k);
  c->release(m->row_order);
  c->release(m->key_of_input);
  delete m;
  return GS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ measurement
// Segmented reduction of already sorted keys, for comparing the paper's
// FastHashReduction (run flags + exclusive scan + warp head-segmented
// reduction, Sec. 5.2) with a library reduce-by-key on the same input.
namespace gs {
struct Block9 {
  double v[9];
};
struct Sum9 {
  __device__ __forceinline__ Block9 operator()(const Block9& a, const Block9& b) const {
    Block9 c;
#pragma unroll
    for (int k = 0; k < 9; ++k) c.v[k] = a.v[k] + b.v[k];
    return c;
  }
};
__global__ void k_iota(uint32_t* __restrict__ a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (uint32_t)i;
}
}  // namespace gs

extern "C" int gs_micro_segment_reduce(gs_ctx ctx, int64_t nb, const uint64_t* keys, const double* blocks,
                                       int32_t method, double* out, int64_t* n_unique, float* ms) {
  using namespace gs;
  GS_CHECK(ctx && keys && blocks && out && n_unique && ms && nb > 0 && nb < (1LL << 31), GS_ERR_INVALID,
           "gs_micro_segment_reduce: bad argument");
  GS_CHECK(method == 0 || method == 1, GS_ERR_INVALID, "gs_micro_segment_reduce: method %d", method);
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0, e1;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  int s = GS_OK;
  void* temp = nullptr;
  size_t tb = 0;
  int32_t *P = nullptr, *rid = nullptr, *cid = nullptr, *koi = nullptr;
  uint32_t* idx = nullptr;
  uint64_t* ukeys = nullptr;
  int64_t* nruns = nullptr;
  const int T = 256;
  if (method == 0) {
    if ((s = ctx->alloc((void**)&P, (size_t)nb * 8)) || (s = ctx->alloc((void**)&idx, (size_t)nb * 4)) ||
        (s = ctx->alloc((void**)&rid, (size_t)nb * 4)) || (s = ctx->alloc((void**)&cid, (size_t)nb * 4)) ||
        (s = ctx->alloc((void**)&koi, (size_t)nb * 4)))
      goto done;
    k_iota<<<ceil_div(nb, T), T, 0, st>>>(idx, nb);
    int32_t* O = P + nb;
    tb = scan_temp_bytes(nb);
    if ((s = ctx->alloc(&temp, tb))) goto done;
    // phase 1: flags + scan (then the unique count is read back, untimed);
    // phase 2: zero the U outputs + segmented reduction
    cudaEvent_t e2, e3;
    GS_CUDA(cudaEventCreate(&e2));
    GS_CUDA(cudaEventCreate(&e3));
    cudaEventRecord(e0, st);
    k_run_flags<<<ceil_div(nb, T), T, 0, st>>>(keys, nb, P);
    if ((s = exclusive_scan_i32(st, P, O, nb, temp, tb))) goto done;
    cudaEventRecord(e1, st);
    int32_t* ho = (int32_t*)ctx->h_pinned;
    if (cudaMemcpyAsync(ho, O + nb - 1, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) s = GS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) s = GS_ERR_CUDA;
    *n_unique = (int64_t)ho[0] + 1;
    cudaEventRecord(e2, st);
    cudaMemsetAsync(out, 0, (size_t)*n_unique * 72, st);
    k_fast_segment_reduce<<<ceil_div(nb, T), T, 0, st>>>(keys, idx, O, blocks, nb, ~0ull, 32, out, rid, cid, koi);
    cudaEventRecord(e3, st);
    float m1 = 0.f, m2 = 0.f;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaEventElapsedTime(&m1, e0, e1) != cudaSuccess ||
        cudaEventElapsedTime(&m2, e2, e3) != cudaSuccess)
      s = GS_ERR_CUDA;
    cudaEventDestroy(e2);
    cudaEventDestroy(e3);
    *ms = m1 + m2;
  } else {
    if ((s = ctx->alloc((void**)&ukeys, (size_t)nb * 8)) || (s = ctx->alloc((void**)&nruns, 8))) goto done;
    cub::DeviceReduce::ReduceByKey(nullptr, tb, keys, ukeys, (const Block9*)blocks, (Block9*)out, nruns, Sum9(), nb,
                                   st);
    if ((s = ctx->alloc(&temp, tb))) goto done;
    cudaEventRecord(e0, st);
    cub::DeviceReduce::ReduceByKey(temp, tb, keys, ukeys, (const Block9*)blocks, (Block9*)out, nruns, Sum9(), nb,
                                   st);
    cudaEventRecord(e1, st);
    int64_t* hn = (int64_t*)ctx->h_pinned;
    if (cudaMemcpyAsync(hn, nruns, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) s = GS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) s = GS_ERR_CUDA;
    *n_unique = hn[0];
  }
  if (s == GS_OK) {
    if (cudaGetLastError() != cudaSuccess || (method == 1 && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)) {
      set_error("gs_micro_segment_reduce: launch failed");
      s = GS_ERR_CUDA;
    }
  } else {
    set_error("gs_micro_segment_reduce: readback failed");
  }
done:
  ctx->release(temp);
  ctx->release(P);
  ctx->release(idx);
  ctx->release(rid);
  ctx->release(cid);
  ctx->release(koi);
  ctx->release(ukeys);
  ctx->release(nruns);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}
