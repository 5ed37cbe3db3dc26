// Connectivity-enhanced MAS construction on the device (Sec. 3.2-3.3,
// Alg. 1; supplement Sec. 2.3, Algorithms 2-5).
//
// Levels.  Level-0 items are the N * M slots of the padded partition
// (node u at slot map[u]); level-l items (l >= 1) are supernodes numbered
// consecutively, domain d of level l being items [d N, d N + N).
//   * k_edge_masks (Alg. 2 initial hash + Alg. 3 contact handling): every
//     directed mesh / contact edge (u, v) whose endpoints sit in distinct
//     items a, b of one level-l domain ORs b's lane bit into a's 32-bit mask.
//   * k_expand_number (Alg. 4 connection expansion + Alg. 5 numbering): one
//     warp per domain holds the masks in registers, closes them under
//     "neighbour of a neighbour" with shuffles (the paper's __ffs walk over
//     shared memory, done as a doubling iteration), elects the lowest lane
//     of each component with a ballot and numbers the components by
//     __popc of the elected lanes below.
//   * a scan over the per-domain counts gives each domain's first supernode.
// Level matrices (Alg. 1).  Level 0 is written directly (each stored block
// of a domain has a unique position).  For l >= 1 the blocks inside a
// level-0 domain are first summed per (item, item) pair of that domain --
// one warp per domain, the paper's warp reduction -- and added atomically;
// blocks between level-0 domains are added atomically one by one.
// Inverses (Alg. 1 "invert unpadded parts"): one CTA per domain factorises
// the real items' part in shared memory (Cholesky, FP64), inverts the
// factor and forms L^-T L^-1, overwriting the matrix with its inverse.
#include <cub/device/device_scan.cuh>
#include <cuda_bf16.h>

#include "common.cuh"
#include "primitives.cuh"

namespace gs {

// ------------------------------------------------------------------ validation / remap
__global__ void k_build_remap(const int32_t* __restrict__ map, int32_t n, int32_t n_slots,
                              int32_t* __restrict__ remap, int* flags) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int32_t s = map[v];
  if (s < 0 || s >= n_slots) {
    atomicOr(flags, kErrIndex);
    return;
  }
  if (atomicCAS(&remap[s], -1, v) != -1) atomicOr(flags, kErrIndex);  // two nodes in one slot
}

// Directed edge list: every CSR entry (u, adj[k]) plus both directions of
// every contact pair.
__global__ void k_edges_from_csr(const int32_t* __restrict__ ptr, const int32_t* __restrict__ adj, int32_t n,
                                 int32_t* __restrict__ src, int32_t* __restrict__ dst, int* flags) {
  int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int32_t b = ptr[u], e = ptr[u + 1];
  for (int32_t k = b; k < e; ++k) {
    int32_t v = adj[k];
    if (v < 0 || v >= n) {
      atomicOr(flags, kErrIndex);
      v = u;
    }
    src[k] = u;
    dst[k] = v;
  }
}

__global__ void k_edges_from_contacts(const int32_t* __restrict__ pairs, int64_t P, int32_t n, int64_t base,
                                      int32_t* __restrict__ src, int32_t* __restrict__ dst, int* flags) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int32_t a = pairs[2 * p], b = pairs[2 * p + 1];
  if (a < 0 || a >= n || b < 0 || b >= n) {
    atomicOr(flags, kErrIndex);
    a = b = 0;
  }
  src[base + 2 * p] = a, dst[base + 2 * p] = b;
  src[base + 2 * p + 1] = b, dst[base + 2 * p + 1] = a;
}

__global__ void k_csr_ptr_check(const int32_t* __restrict__ ptr, int32_t n, int* flags) {
  int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  if (ptr[u] > ptr[u + 1] || ptr[u] < 0) atomicOr(flags, kErrIndex);
}

// ------------------------------------------------------------------ levels
// Own lane bit for every item that holds a fine node (padding keeps 0).
__global__ void k_mask_init(const int32_t* __restrict__ item_of_node, int32_t n, int N, uint32_t* __restrict__ mask) {
  int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int32_t a = item_of_node[u];
  mask[a] = 1u << (a % N);  // idempotent: all nodes of an item write the same bit
}

__global__ void k_edge_masks(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t E,
                             const int32_t* __restrict__ item_of_node, int N, uint32_t* __restrict__ mask) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int32_t a = item_of_node[src[e]], b = item_of_node[dst[e]];
  if (a != b && a / N == b / N) atomicOr(&mask[a], 1u << (b % N));
}

// One warp per domain.  Outputs the local supernode id of every item
// (-1 for empty items) and the domain's supernode count.
__global__ void k_expand_number(const uint32_t* __restrict__ mask, int32_t n_dom, int N,
                                int32_t* __restrict__ local_id, int32_t* __restrict__ count) {
  int32_t d = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (d >= n_dom) return;  // whole warp leaves together
  uint32_t m = (lane < N) ? mask[(int64_t)d * N + lane] : 0u;
  // Closure: OR in the masks of every lane already reached until stable.
  bool changed;
  do {
    uint32_t acc = m;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      uint32_t mj = __shfl_sync(kFull, m, j);
      if ((m >> j) & 1u) acc |= mj;
    }
    changed = __any_sync(kFull, acc != m);
    m = acc;
  } while (changed);
  const bool real = m != 0u;
  const int lead = real ? (__ffs(m) - 1) : 0;  // lowest lane of the component
  const uint32_t elect = __ballot_sync(kFull, real && lead == lane);
  if (lane < N) local_id[(int64_t)d * N + lane] = real ? __popc(elect & ((1u << lead) - 1u)) : -1;
  if (lane == 0) count[d] = __popc(elect);
}

__global__ void k_next_of_node(const int32_t* __restrict__ item_of_node, int32_t n, int N,
                               const int32_t* __restrict__ local_id, const int32_t* __restrict__ dom_off,
                               int32_t* __restrict__ next_of_node) {
  int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int32_t a = item_of_node[u];
  next_of_node[u] = dom_off[a / N] + local_id[a];
}

// Parent (level-(l+1) item) of every level-l item, l >= 1, from the same
// numbering as k_next_of_node; -1 for padded (empty) items.
__global__ void k_up_of_item(int32_t n_items_pad, int N, const int32_t* __restrict__ local_id,
                             const int32_t* __restrict__ dom_off, int32_t* __restrict__ up) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_items_pad) return;
  const int32_t id = local_id[a];
  up[a] = id >= 0 ? dom_off[a / N] + id : -1;
}

// ------------------------------------------------------------------ level matrices
struct LevelPtrs {
  const int32_t* coarse[8];
  double* mat[8];
  int L;
  int N;
};

__device__ __forceinline__ void add_block(double* M, int N, int32_t i, int32_t j, const double* H, bool transpose) {
  // block (i, j) of a 3N x 3N row-major domain matrix; i, j lanes
  const int ld = 3 * N;
  double* p = M + (int64_t)(3 * i) * ld + 3 * j;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) atomicAdd(p + x * ld + y, transpose ? H[3 * y + x] : H[3 * x + y]);
}

// Thread per stored block: level-0 direct write; cross-domain blocks are
// added to the coarser levels atomically.
__global__ void k_scatter_blocks(const int32_t* __restrict__ rid, const int32_t* __restrict__ cid,
                                 const double* __restrict__ au, int64_t nnzb, LevelPtrs lp) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nnzb) return;
  const int N = lp.N;
  const int ld = 3 * N;
  int32_t r = rid[u], c = cid[u];
  double H[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) H[k] = au[u * 9 + k];
  int32_t a = lp.coarse[0][r], b = lp.coarse[0][c];
  if (a / N == b / N) {
    double* M = lp.mat[0] + (int64_t)(a / N) * ld * ld;
    int32_t i = a % N, j = b % N;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = 0; y < 3; ++y) {
        M[(int64_t)(3 * i + x) * ld + 3 * j + y] = H[3 * x + y];
        if (r != c) M[(int64_t)(3 * j + y) * ld + 3 * i + x] = H[3 * x + y];
      }
    return;  // coarser levels receive this block through k_domain_reduce
  }
  for (int l = 1; l < lp.L; ++l) {
    int32_t A = lp.coarse[l][r], B = lp.coarse[l][c];
    if (A / N != B / N) continue;
    double* M = lp.mat[l] + (int64_t)(A / N) * ld * ld;
    if (A == B) {
      double S[9];
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) S[3 * x + y] = H[3 * x + y] + H[3 * y + x];
      add_block(M, N, A % N, A % N, S, false);
    } else {
      add_block(M, N, A % N, B % N, H, false);
      add_block(M, N, B % N, A % N, H, true);
    }
  }
}

// One warp per level-0 domain: sum the domain's blocks per (level-1 row
// group, level-1 column group) and add each sum at the groups' items of
// every level l >= 1 (a level-1 group maps to one item at every level).
__global__ void k_domain_reduce(const int32_t* __restrict__ remap, int32_t n_dom0, LevelPtrs lp) {
  int32_t d = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (d >= n_dom0) return;
  const int N = lp.N;
  const int ld = 3 * N;
  const double* M0 = lp.mat[0] + (int64_t)d * ld * ld;
  int32_t node = (lane < N) ? remap[(int64_t)d * N + lane] : -1;
  bool real = node >= 0;
  int32_t c1 = real ? lp.coarse[1][node] : -1;
  uint32_t rows_left = __ballot_sync(kFull, real);
  while (rows_left) {
    const int lr = __ffs(rows_left) - 1;
    const int32_t ci = __shfl_sync(kFull, c1, lr);
    const uint32_t rmask = __ballot_sync(kFull, real && c1 == ci);
    rows_left &= ~rmask;
    const int32_t node_i = __shfl_sync(kFull, node, lr);
    // T_j = sum over rows i of group ci of block (i, j); lane j owns column block j
    double T[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) T[k] = 0.0;
    if (real) {
      uint32_t rm = rmask;
      while (rm) {
        int i = __ffs(rm) - 1;
        rm &= rm - 1;
        const double* p = M0 + (int64_t)(3 * i) * ld + 3 * lane;
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
          for (int y = 0; y < 3; ++y) T[3 * x + y] += p[x * ld + y];
      }
    }
    uint32_t cols_left = __ballot_sync(kFull, real);
    while (cols_left) {
      const int lc = __ffs(cols_left) - 1;
      const int32_t cj = __shfl_sync(kFull, c1, lc);
      const uint32_t cmask = __ballot_sync(kFull, real && c1 == cj);
      cols_left &= ~cmask;
      const int32_t node_j = __shfl_sync(kFull, node, lc);
      double v[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) v[k] = warp_sum(((cmask >> lane) & 1u) ? T[k] : 0.0);
      if (lane == 0) {
        for (int l = 1; l < lp.L; ++l) {
          int32_t A = lp.coarse[l][node_i], B = lp.coarse[l][node_j];
          if (A / N != B / N) continue;
          double* M = lp.mat[l] + (int64_t)(A / N) * ld * ld;
          add_block(M, N, A % N, B % N, v, false);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ inversion
struct InvJob {
  double* mat;              // 3N x 3N row-major, overwritten by the inverse
  const int32_t* remap;     // level 0: slot -> node (-1 padding); nullptr for l >= 1
  int32_t items_in_domain;  // l >= 1: real items of this domain
};

// One CTA per domain.  Shared memory holds the lower triangle of the
// compacted real part, packed by rows (entry (i, j), j <= i, at
// i (i + 1) / 2 + j: 37 KB at 3k = 96, so five CTAs share an SM), plus a
// contiguous copy of the current Cholesky column.  The arithmetic is that of
// the full-storage form, operation for operation.
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

__global__ void __launch_bounds__(256) k_invert_domains(double* const* mats,
                                                         const int32_t* __restrict__ remap0, int32_t n_dom0,
                                                         const int32_t* __restrict__ dom_level,
                                                         const int32_t* __restrict__ dom_index,
                                                         const int32_t* __restrict__ n_items, int N, int* flags,
                                                         double* __restrict__ fac0) {
  extern __shared__ double sA[];
  __shared__ double colp[96];  // column p of the factor, rows p+1 ..
  __shared__ int s_lane[32];
  __shared__ int s_k;
  __shared__ int s_bad;
  __shared__ double s_rdiag;  // 1 / L_pp of the current Cholesky step
  const int job = blockIdx.x;
  const int l = dom_level[job];
  const int d = dom_index[job];
  const int ld = 3 * N;
  double* M = mats[l] + (int64_t)d * ld * ld;
  const int tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = T >> 5;
  if (tid < 32) {
    bool real;
    if (l == 0)
      real = tid < N && remap0[(int64_t)d * N + tid] >= 0;
    else
      real = tid < N && (int64_t)d * N + tid < n_items[l];
    uint32_t rm = __ballot_sync(kFull, real);
    if (real) s_lane[__popc(rm & ((1u << tid) - 1u))] = tid;
    if (tid == 0) {
      s_k = __popc(rm);
      s_bad = 0;
    }
  }
  __syncthreads();
  const int k = s_k;
  const int n3 = 3 * k;
  if (k == 0) return;
  // load the lower triangle of the compacted real part (a warp per row)
  for (int i = wid; i < n3; i += nw) {
    const int gi = 3 * s_lane[i / 3] + i % 3;
    for (int j = lane; j <= i; j += 32) sA[tri(i, j)] = M[(int64_t)gi * ld + 3 * s_lane[j / 3] + j % 3];
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle.  FP64 is the scarce unit: one
  // reciprocal per step (not one per thread), and the trailing update walks
  // only the lower triangle (a warp per row, lanes along it, the column read
  // from its contiguous copy).
  for (int p = 0; p < n3; ++p) {
    if (tid == 0) {
      double dpp = sA[tri(p, p)];
      if (!(dpp > 0.0)) {
        s_bad = 1;
        dpp = 1.0;
      }
      const double lpp = sqrt(dpp);
      sA[tri(p, p)] = lpp;
      s_rdiag = 1.0 / lpp;
    }
    __syncthreads();
    if (s_bad) break;
    const double inv = s_rdiag;
    for (int i = p + 1 + tid; i < n3; i += T) {
      const double v = sA[tri(i, p)] * inv;
      sA[tri(i, p)] = v;
      colp[i] = v;
    }
    __syncthreads();
    for (int i = p + 1 + wid; i < n3; i += nw) {
      const double lip = colp[i];
      const int ri = tri(i, 0);
      for (int j = p + 1 + lane; j <= i; j += 32) sA[ri + j] -= lip * colp[j];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) atomicOr(flags, kErrNotSPD);
    return;
  }
  // W = L^{-1} in place.  The diagonal first becomes 1 / L_jj (= W_jj), then
  // W_ij = -(sum_{q=j+1..i} W_iq L_qj) W_jj, column by column from the last.
  for (int j = tid; j < n3; j += T) sA[tri(j, j)] = 1.0 / sA[tri(j, j)];
  __syncthreads();
  for (int j = n3 - 1; j >= 0; --j) {
    const double wjj = sA[tri(j, j)];
    double w = 0.0;
    const int i = j + 1 + tid;
    if (i < n3) {
      double acc = 0.0;
      const int ri = tri(i, 0);
      for (int q = j + 1; q <= i; ++q) acc += sA[ri + q] * sA[tri(q, j)];
      w = -acc * wjj;
    }
    __syncthreads();
    if (i < n3) sA[tri(i, j)] = w;
    __syncthreads();
  }
  // level 0, low-precision form: keep the factor W = L^{-1} (M^{-1} = W^T W)
  if (fac0 && l == 0) {
    double* F = fac0 + (int64_t)d * ld * ld;
    for (int i = wid; i < n3; i += nw) {
      const int gi = 3 * s_lane[i / 3] + i % 3;
      for (int j = lane; j <= i; j += 32) F[(int64_t)gi * ld + 3 * s_lane[j / 3] + j % 3] = sA[tri(i, j)];
    }
  }
  // inverse = W^T W, written over the real part of the global matrix; entry
  // (i, j) and (j, i) are the same sum in the same order, so the lower
  // triangle is computed and mirrored
  for (int e = tid; e < n3 * n3; e += T) {
    int i = e / n3, j = e % n3;
    if (j > i) continue;
    double acc = 0.0;
    for (int q = i; q < n3; ++q) acc += sA[tri(q, i)] * sA[tri(q, j)];
    int gi = 3 * s_lane[i / 3] + i % 3, gj = 3 * s_lane[j / 3] + j % 3;
    M[(int64_t)gi * ld + gj] = acc;
    M[(int64_t)gj * ld + gi] = acc;
  }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// Level-0 inverses (FP64, full, symmetric) -> FP32 lower triangles packed by
// rows, rounded to nearest as k_to_float rounds them; `pitch` floats per domain.
__global__ void k_pack_lower_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n_dom, int ld,
                                 int pitch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_dom * pitch) return;
  const int64_t d = t / pitch;
  const int p = (int)(t - d * pitch);
  if (p >= ld * (ld + 1) / 2) {
    b[t] = 0.0f;
    return;
  }
  int i = (int)((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);  // row of packed index p
  while (i * (i + 1) / 2 > p) --i;
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  const int j = p - i * (i + 1) / 2;
  b[t] = (float)a[d * ld * ld + (int64_t)i * ld + j];
}

// double -> float -> bfloat16, both roundings to nearest even
__global__ void k_to_bf16(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn((float)a[i]);
}

// Level matrices, inverses and the stored forms of the precision for the
// level structure already in `mas` (the numeric part of the build; the
// structure depends only on the partition and the graph, so a matrix with
// new values on the same nodes reuses it).
static int mas_numeric(gs_ctx ctx, gs_mas mas, gs_mat mat) {
  cudaStream_t st = ctx->stream;
  const int L = mas->L;
  const int N = mas->N;
  const int32_t n_dom0 = mas->n_domains[0];
  const int precision = mas->precision;
  int s;
  int flags = 0;
  // level matrices
  const int ld = 3 * N;
  LevelPtrs lp{};
  lp.L = L;
  lp.N = N;
  for (int l = 0; l < L; ++l) {
    double* m = nullptr;
    size_t bytes = (size_t)mas->n_domains[l] * ld * ld * sizeof(double);
    if ((s = ctx->alloc((void**)&m, bytes))) return s;
    mas->inv64.push_back(m);
    if (cudaMemsetAsync(m, 0, bytes, st) != cudaSuccess) return GS_ERR_CUDA;
    lp.coarse[l] = mas->coarse[l];
    lp.mat[l] = m;
  }
  if (mat->nnzb > 0)
    { GS_PROF(ctx, GS_K_MAS_MATRICES); k_scatter_blocks<<<ceil_div(mat->nnzb, 256), 256, 0, st>>>(mat->rid, mat->cid, mat->au, mat->nnzb, lp); }
  if (L > 1) { GS_PROF(ctx, GS_K_MAS_MATRICES); k_domain_reduce<<<ceil_div((int64_t)n_dom0 * 32, 256), 256, 0, st>>>(mas->remap0, n_dom0, lp); }
  // inversion jobs: every domain of every level
  std::vector<int32_t> h_level, h_index;
  for (int l = 0; l < L; ++l)
    for (int32_t d = 0; d < mas->n_domains[l]; ++d) h_level.push_back(l), h_index.push_back(d);
  const int jobs = (int)h_level.size();
  int32_t* djobs = nullptr;
  if ((s = ctx->scratch_buf(kSlotMasBuild3, (size_t)jobs * 8 + (L + 1) * 8 + 8 * sizeof(double*) + 64,
                            (void**)&djobs)))
    return s;
  int32_t* d_items = djobs + 2 * jobs;
  double** d_mats = (double**)(((uintptr_t)(d_items + L + 1) + 15) & ~(uintptr_t)15);
  std::vector<double*> hm(mas->inv64.begin(), mas->inv64.end());
  if (cudaMemcpyAsync(djobs, h_level.data(), jobs * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(djobs + jobs, h_index.data(), jobs * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_items, mas->n_items.data(), L * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_mats, hm.data(), L * sizeof(double*), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return GS_ERR_CUDA;
  const size_t smem = (size_t)(3 * N) * (3 * N + 1) / 2 * sizeof(double);  // packed lower triangle
  if (cudaFuncSetAttribute(k_invert_domains, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GS_ERR_CUDA;
  // BF16 form: level 0 keeps its inverse Cholesky factors (rounding W keeps
  // W^T W positive semi-definite; rounding M^{-1} itself does not once a
  // domain's condition number passes ~1e3), coarse levels FP32 inverses
  double* fac0 = nullptr;
  const int64_t cnt0 = (int64_t)n_dom0 * ld * ld;
  if (precision == GS_PREC_BF16) {
    if ((s = ctx->alloc((void**)&fac0, (size_t)std::max<int64_t>(cnt0, 1) * 8))) return s;
    if (cudaMemsetAsync(fac0, 0, (size_t)cnt0 * 8, st) != cudaSuccess) return GS_ERR_CUDA;
  }
  { GS_PROF(ctx, GS_K_MAS_INVERT); k_invert_domains<<<jobs, 256, smem, st>>>(d_mats, mas->remap0, n_dom0, djobs, djobs + jobs, d_items, N,
                                            ctx->d_flags, fac0); }
  if (precision == GS_PREC_BF16) {
    void* f = nullptr;
    s = ctx->alloc(&f, (size_t)std::max<int64_t>(cnt0, 1) * 2);
    if (s == GS_OK) {
      mas->inv16.push_back(f);
      if (cnt0) { GS_PROF(ctx, GS_K_MAS_INVERT); k_to_bf16<<<ceil_div(cnt0, 256), 256, 0, st>>>(fac0, (__nv_bfloat16*)f, cnt0); }
      s = level0_bf16_prepare(ctx, mas, fac0);
    }
    ctx->release(fac0);
    if (s) return s;
  }
  if (precision == GS_PREC_FP64 && (s = level0_f64tc_prepare(ctx, mas))) return s;
  if (precision == GS_PREC_FP32 || precision == GS_PREC_BF16) {
    mas->inv32.assign(L, nullptr);
    for (int l = precision == GS_PREC_BF16 ? 1 : 0; l < L; ++l) {
      float* f = nullptr;
      int64_t cnt = (int64_t)mas->n_domains[l] * ld * ld;
      if ((s = ctx->alloc((void**)&f, (size_t)cnt * 4))) return s;
      mas->inv32[l] = f;
      { GS_PROF(ctx, GS_K_MAS_INVERT); k_to_float<<<ceil_div(cnt, 256), 256, 0, st>>>(mas->inv64[l], f, cnt); }
    }
    if (precision == GS_PREC_FP32) {  // level 0 also as packed lower triangles (the streamed apply)
      const int pitch = ((ld * (ld + 1) / 2 + 3) / 4) * 4;
      const int64_t cnt = (int64_t)mas->n_domains[0] * pitch;
      if ((s = ctx->alloc((void**)&mas->inv32p, (size_t)cnt * 4))) return s;
      { GS_PROF(ctx, GS_K_MAS_INVERT); k_pack_lower_f32<<<ceil_div(cnt, 256), 256, 0, st>>>(mas->inv64[0], mas->inv32p, mas->n_domains[0], ld, pitch); }
    }
  }
  // multilevel vector layout for the apply (levels >= 1, padded per domain)
  mas->vec_off.assign(L, 0);
  int64_t off = 0;
  for (int l = 1; l < L; ++l) {
    mas->vec_off[l] = off;
    off += (int64_t)mas->n_domains[l] * N;
  }
  mas->vec_items = off;
  // constant tables of the apply: inverse pointers and the coarse domain jobs
  {
    std::vector<void*> hp(8, nullptr);
    for (int l = 0; l < L; ++l)
      hp[l] = precision == GS_PREC_FP32   ? (void*)mas->inv32[l]
              : precision == GS_PREC_BF16 ? (l == 0 ? mas->inv16[0] : (void*)mas->inv32[l])
                                                : (void*)mas->inv64[l];
    std::vector<int32_t> lev, dom;
    for (int l = 1; l < L; ++l)
      for (int32_t d = 0; d < mas->n_domains[l]; ++d) lev.push_back(l), dom.push_back(d);
    mas->n_coarse_jobs = (int32_t)lev.size();
    lev.insert(lev.end(), dom.begin(), dom.end());
    if ((s = ctx->alloc((void**)&mas->d_inv_tab, 8 * sizeof(void*))) ||
        (s = ctx->alloc((void**)&mas->d_coarse_jobs, std::max<size_t>(lev.size(), 1) * 4)))
      return s;
    if (cudaMemcpyAsync(mas->d_inv_tab, hp.data(), 8 * sizeof(void*), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (!lev.empty() && cudaMemcpyAsync(mas->d_coarse_jobs, lev.data(), lev.size() * 4, cudaMemcpyHostToDevice,
                                         st) != cudaSuccess))
      return GS_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
  if ((s = ctx->take_flags(&flags))) return s;
  if (flags) return status_from_flags(flags);
  return GS_OK;
}

// Releases what mas_numeric made (lazily built copies included).
static void mas_release_numeric(gs_mas mas) {
  gs_ctx c = mas->owner;
  for (auto p : mas->inv64) c->release(p);
  for (auto p : mas->inv32) c->release(p);
  for (auto p : mas->inv16) c->release(p);
  for (auto p : mas->dig64) c->release(p);
  for (auto p : mas->dig64_exp) c->release(p);
  for (auto p : mas->dig8) c->release(p);
  for (auto p : mas->dig8_scale) c->release(p);
  c->release(mas->inv32p);
  c->release(mas->inv16_tc);
  c->release(mas->d_dig_tab);
  c->release(mas->d_sym_tab);
  c->release(mas->d_inv_tab);
  c->release(mas->d_coarse_jobs);
  c->release(mas->d_inv32_tab);
  mas->inv64.clear();
  mas->inv32.clear();
  mas->inv16.clear();
  mas->dig64.clear();
  mas->dig64_exp.clear();
  mas->dig8.clear();
  mas->dig8_scale.clear();
  mas->d_sym_tab = nullptr;
  mas->inv32p = nullptr;
  mas->inv16_tc = nullptr;
  mas->d_dig_tab = nullptr;
  mas->d_inv_tab = nullptr;
  mas->d_coarse_jobs = nullptr;
  mas->d_inv32_tab = nullptr;
  mas->vec_off.clear();
  mas->vec_items = 0;
  mas->n_coarse_jobs = 0;
}

}  // namespace gs

using namespace gs;

extern "C" {

int gs_mas_destroy(gs_mas mas) {
  if (!mas) return GS_OK;
  gs_ctx c = mas->owner;
  for (auto p : mas->coarse) c->release(p);
  for (auto p : mas->up) c->release(p);
  for (auto p : mas->inv64) c->release(p);
  for (auto p : mas->inv32) c->release(p);
  c->release(mas->inv32p);
  for (auto p : mas->inv16) c->release(p);
  c->release(mas->inv16_tc);
  for (auto p : mas->dig64) c->release(p);
  for (auto p : mas->dig64_exp) c->release(p);
  c->release(mas->d_dig_tab);
  for (auto p : mas->dig8) c->release(p);
  for (auto p : mas->dig8_scale) c->release(p);
  c->release(mas->d_sym_tab);
  c->release(mas->remap0);
  c->release(mas->d_inv_tab);
  c->release(mas->d_coarse_jobs);
  c->release(mas->d_inv32_tab);
  delete mas;
  return GS_OK;
}

int gs_build_mas(gs_ctx ctx, gs_mat mat, const int32_t* map, int32_t n_dom0, const int32_t* adj_ptr,
                 const int32_t* adj, const int32_t* contacts, int64_t n_contacts, const gs_mas_opts* opts,
                 gs_mas* out) {
  GS_CHECK(ctx && mat && out && opts, GS_ERR_INVALID, "gs_build_mas: null argument");
  *out = nullptr;
  const int N = opts->domain_size;
  GS_CHECK(N >= 1, GS_ERR_INVALID, "gs_build_mas: domain_size %d", N);
  GS_CHECK(N <= 32, GS_ERR_UNSUPPORTED, "gs_build_mas: domain_size %d > 32", N);
  GS_CHECK(opts->max_levels >= 1 && opts->max_levels <= 8, GS_ERR_INVALID, "gs_build_mas: max_levels %d",
           opts->max_levels);
  GS_CHECK(opts->precision == GS_PREC_FP64 || opts->precision == GS_PREC_FP32 || opts->precision == GS_PREC_BF16,
           GS_ERR_INVALID,
           "gs_build_mas: precision %d", opts->precision);
  const int32_t n = mat->n;
  GS_CHECK(map && adj_ptr && (adj || true), GS_ERR_INVALID, "gs_build_mas: null map or graph");
  GS_CHECK(n_dom0 >= 1 && (int64_t)n_dom0 * N >= n && (int64_t)n_dom0 * N < (1LL << 31), GS_ERR_INVALID,
           "gs_build_mas: n_domains0 %d too small for %d nodes", n_dom0, n);
  GS_CHECK(n_contacts >= 0 && (n_contacts == 0 || contacts), GS_ERR_INVALID, "gs_build_mas: contacts");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;

  gs_mas mas = new gs_mas_s();
  mas->owner = ctx;
  mas->N = N;
  mas->n = n;
  mas->precision = opts->precision;
  auto fail = [&](int s) {
    gs_mas_destroy(mas);
    return s;
  };
  int s;
  const int32_t n_slots = n_dom0 * N;
  // remap + validation of map
  if ((s = ctx->alloc((void**)&mas->remap0, (size_t)n_slots * 4))) return fail(s);
  if (cudaMemsetAsync(mas->remap0, 0xff, (size_t)n_slots * 4, st) != cudaSuccess) return fail(GS_ERR_CUDA);
  { GS_PROF(ctx, GS_K_OTHER); k_build_remap<<<ceil_div(n, 256), 256, 0, st>>>(map, n, n_slots, mas->remap0, ctx->d_flags); }
  { GS_PROF(ctx, GS_K_OTHER); k_csr_ptr_check<<<ceil_div(n, 256), 256, 0, st>>>(adj_ptr, n, ctx->d_flags); }
  int flags = 0;
  if ((s = ctx->take_flags(&flags))) return fail(s);
  if (flags) return fail(status_from_flags(flags));
  // directed edges
  if (cudaMemcpyAsync(ctx->h_pinned, adj_ptr + n, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(GS_ERR_CUDA);
  const int32_t nnz_adj = ctx->h_pinned[0];
  GS_CHECK(nnz_adj >= 0 && (nnz_adj == 0 || adj), GS_ERR_INVALID, "gs_build_mas: bad adjacency");
  const int64_t E = (int64_t)nnz_adj + 2 * n_contacts;
  int32_t *src = nullptr, *dst = nullptr;
  if ((s = ctx->scratch_buf(kSlotMasBuild0, (size_t)std::max<int64_t>(E, 1) * 8, (void**)&src))) return fail(s);
  dst = src + std::max<int64_t>(E, 1);
  { GS_PROF(ctx, GS_K_MAS_LEVELS); k_edges_from_csr<<<ceil_div(n, 256), 256, 0, st>>>(adj_ptr, adj, n, src, dst, ctx->d_flags); }
  if (n_contacts > 0)
    { GS_PROF(ctx, GS_K_MAS_LEVELS); k_edges_from_contacts<<<ceil_div(n_contacts, 256), 256, 0, st>>>(contacts, n_contacts, n, nnz_adj, src, dst,
                                                                     ctx->d_flags); }
  if ((s = ctx->take_flags(&flags))) return fail(s);
  if (flags) return fail(status_from_flags(flags));

  // level 0
  int32_t* c0 = nullptr;
  if ((s = ctx->alloc((void**)&c0, (size_t)n * 4))) return fail(s);
  mas->coarse.push_back(c0);
  if (cudaMemcpyAsync(c0, map, (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return fail(GS_ERR_CUDA);
  mas->n_items.push_back(n_slots);
  mas->n_domains.push_back(n_dom0);
  int64_t n_real = n;

  // coarser levels
  uint32_t* mask = nullptr;
  int32_t *local_id = nullptr, *count = nullptr, *dom_off = nullptr;
  if ((s = ctx->scratch_buf(kSlotMasBuild1, (size_t)n_slots * 8 + 64, (void**)&mask))) return fail(s);
  local_id = (int32_t*)(mask + n_slots);
  if ((s = ctx->scratch_buf(kSlotMasBuild2, (size_t)(n_dom0 + 1) * 8 + 64, (void**)&count))) return fail(s);
  dom_off = count + n_dom0 + 1;
  while ((int)mas->coarse.size() < opts->max_levels) {
    const int l = (int)mas->coarse.size() - 1;
    const int32_t items = mas->n_items[l], ndom = mas->n_domains[l];
    if (items <= N) break;
    const int32_t* cl = mas->coarse[l];
    if (cudaMemsetAsync(mask, 0, (size_t)ndom * N * 4, st) != cudaSuccess) return fail(GS_ERR_CUDA);
    { GS_PROF(ctx, GS_K_MAS_LEVELS); k_mask_init<<<ceil_div(n, 256), 256, 0, st>>>(cl, n, N, mask); }
    if (E > 0) { GS_PROF(ctx, GS_K_MAS_LEVELS); k_edge_masks<<<ceil_div(E, 256), 256, 0, st>>>(src, dst, E, cl, N, mask); }
    { GS_PROF(ctx, GS_K_MAS_LEVELS); k_expand_number<<<ceil_div((int64_t)ndom * 32, 256), 256, 0, st>>>(mask, ndom, N, local_id, count); }
    cudaMemsetAsync(count + ndom, 0, 4, st);
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, count, dom_off, ndom + 1, st);
    void* temp;
    if ((s = ctx->scratch_buf(kSlotSortTemp, tb, &temp))) return fail(s);
    { GS_PROF(ctx, GS_K_LIBPRIM); cub::DeviceScan::ExclusiveSum(temp, tb, count, dom_off, ndom + 1, st); }
    if (cudaMemcpyAsync(ctx->h_pinned, dom_off + ndom, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(GS_ERR_CUDA);
    const int32_t n_next = ctx->h_pinned[0];
    if (n_next >= n_real) break;  // no merge happened
    int32_t* cn = nullptr;
    if ((s = ctx->alloc((void**)&cn, (size_t)n * 4))) return fail(s);
    mas->coarse.push_back(cn);
    { GS_PROF(ctx, GS_K_MAS_LEVELS); k_next_of_node<<<ceil_div(n, 256), 256, 0, st>>>(cl, n, N, local_id, dom_off, cn); }
    mas->up.resize(l + 1, nullptr);
    if (l >= 1) {  // item-to-item map for the ordered restriction of level l + 1
      int32_t* u = nullptr;
      if ((s = ctx->alloc((void**)&u, (size_t)ndom * N * 4))) return fail(s);
      mas->up[l] = u;
      { GS_PROF(ctx, GS_K_MAS_LEVELS); k_up_of_item<<<ceil_div((int64_t)ndom * N, 256), 256, 0, st>>>(ndom * N, N, local_id, dom_off, u); }
    }
    mas->n_items.push_back(n_next);
    mas->n_domains.push_back(ceil_div(n_next, N));
    n_real = n_next;
  }
  mas->L = (int)mas->coarse.size();
  mas->up.resize(mas->L, nullptr);
  if ((s = mas_numeric(ctx, mas, mat))) return fail(s);
  *out = mas;
  return GS_OK;
}

int gs_mas_refresh(gs_ctx ctx, gs_mas mas, gs_mat mat) {
  GS_CHECK(ctx && mas && mat, GS_ERR_INVALID, "gs_mas_refresh: null argument");
  GS_CHECK(mas->owner == ctx, GS_ERR_INVALID, "gs_mas_refresh: preconditioner of another context");
  GS_CHECK(mat->n == mas->n, GS_ERR_INVALID, "gs_mas_refresh: matrix has %d block rows, preconditioner %d", mat->n,
           mas->n);
  GS_CUDA(cudaSetDevice(ctx->device));
  mas_release_numeric(mas);
  return mas_numeric(ctx, mas, mat);
}

int gs_mas_info(gs_mas mas, int32_t* n_levels, int32_t* n_items) {
  GS_CHECK(mas, GS_ERR_INVALID, "gs_mas_info: null handle");
  if (n_levels) *n_levels = mas->L;
  if (n_items)
    for (int l = 0; l < mas->L; ++l) n_items[l] = mas->n_items[l];
  return GS_OK;
}

int gs_mas_export_coarse(gs_ctx ctx, gs_mas mas, int32_t level, int32_t* coarse) {
  GS_CHECK(ctx && mas && coarse, GS_ERR_INVALID, "gs_mas_export_coarse: null argument");
  GS_CHECK(level >= 0 && level < mas->L, GS_ERR_INVALID, "gs_mas_export_coarse: level %d", level);
  GS_CUDA(cudaMemcpyAsync(coarse, mas->coarse[level], (size_t)mas->n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return GS_OK;
}

int gs_mas_export_inverse(gs_ctx ctx, gs_mas mas, int32_t level, double* inv) {
  GS_CHECK(ctx && mas && inv, GS_ERR_INVALID, "gs_mas_export_inverse: null argument");
  GS_CHECK(level >= 0 && level < mas->L, GS_ERR_INVALID, "gs_mas_export_inverse: level %d", level);
  const int64_t ld = 3 * mas->N;
  GS_CUDA(cudaMemcpyAsync(inv, mas->inv64[level], (size_t)mas->n_domains[level] * ld * ld * 8,
                          cudaMemcpyDeviceToDevice, ctx->stream));
  return GS_OK;
}

}  // extern "C"
