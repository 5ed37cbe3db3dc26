// Level-0 domain partition on the device (Sec. 3.2, Eq. num_subdomains;
// supplement Algorithm 1), the same rules as the host partition, bit for bit.
//
// GS_PART_RCB: recursive coordinate bisection of the rest positions.  All
// sets of one depth are split together: per set the extent along each axis
// (atomic min / max on order-preserving integer images of the coordinates),
// the axis of largest extent (first on ties), then one stable radix sort of
// the vertices by that coordinate and a stable sort by set, so each set's
// vertices stand in (coordinate, vertex index) order; the first
// N * ceil(P / 2) go left.  New sets are numbered left before right, in set
// order, so the leaves come out numbered left to right.
//
// GS_PART_RCB_COMPONENTS: the same bisection started from the connected
// components of the mesh graph (numbered by their smallest vertex), found by
// hooking roots onto smaller roots with atomic minima and compressing paths
// until nothing changes; no part then mixes two bodies.
//
// GS_PART_MORTON: N consecutive vertices in Morton order (10 bits per axis
// over the bounding box, ties by vertex index), the level-0 subdomains of the
// earlier MAS the paper compares against.
//
// Finally every vertex takes slot N * part + (rank among its part's vertices
// in ascending index): a stable sort by part of the vertices in index order.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gs {
namespace part {

// Order-preserving unsigned image of a double (-0.0 taken as +0.0, so equal
// coordinates compare equal as they do in the host rule).
__device__ __forceinline__ unsigned long long okey(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if (b == 0x8000000000000000ull) b = 0;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_okey(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

__global__ void k_check_finite(const double* __restrict__ X, int64_t n3, int* __restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3 && !isfinite(X[i])) atomicOr(flags, kErrNonFinite);
}

__global__ void k_iota(int32_t* __restrict__ a, int32_t n) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

// ---------------------------------------------------------------- components
__device__ __forceinline__ int32_t find_root(const int32_t* parent, int32_t v) {
  int32_t p = parent[v];
  while (p != v) {
    v = p;
    p = parent[v];
  }
  return v;
}

__global__ void k_hook(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj, int32_t n,
                       int32_t* parent, int* __restrict__ changed, int* __restrict__ flags) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  for (int32_t e = adj_ptr[v]; e < adj_ptr[v + 1]; ++e) {
    const int32_t w = adj[e];
    if (w < 0 || w >= n) {
      atomicOr(flags, kErrIndex);
      continue;
    }
    const int32_t rv = find_root(parent, v), rw = find_root(parent, w);
    if (rv != rw) {
      const int32_t hi = max(rv, rw), lo = min(rv, rw);
      if (atomicMin(&parent[hi], lo) > lo) *changed = 1;
    }
  }
}

__global__ void k_compress(int32_t* parent, int32_t n) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) parent[v] = find_root(parent, v);
}

__global__ void k_root_flags(const int32_t* __restrict__ parent, int32_t n, int32_t* __restrict__ f) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) f[v] = parent[v] == v;
}

__global__ void k_label_from_roots(const int32_t* __restrict__ parent, const int32_t* __restrict__ rank, int32_t n,
                                   int32_t* __restrict__ label) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) label[v] = rank[parent[v]];
}

// ---------------------------------------------------------------- one bisection round
__global__ void k_set_init(int32_t S, int32_t* __restrict__ size, unsigned long long* __restrict__ lo,
                           unsigned long long* __restrict__ hi) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  size[s] = 0;
  for (int a = 0; a < 3; ++a) lo[3 * s + a] = ~0ull, hi[3 * s + a] = 0ull;
}

__global__ void k_set_extent(const double* __restrict__ X, const int32_t* __restrict__ label, int32_t n,
                             int32_t* __restrict__ size, unsigned long long* __restrict__ lo,
                             unsigned long long* __restrict__ hi) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t s = label[v];
  atomicAdd(&size[s], 1);
  for (int a = 0; a < 3; ++a) {
    const unsigned long long k = okey(X[3 * (int64_t)v + a]);
    atomicMin(&lo[3 * s + a], k);
    atomicMax(&hi[3 * s + a], k);
  }
}

// Per set: axis of largest extent (first on ties, the extents computed in
// double as max - min), whether it splits, its left size and its new ids.
__global__ void k_set_plan(int32_t S, int N, const int32_t* __restrict__ size,
                           const unsigned long long* __restrict__ lo, const unsigned long long* __restrict__ hi,
                           int8_t* __restrict__ axis, int32_t* __restrict__ width, int32_t* __restrict__ left) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  int best = 0;
  double ext = from_okey(hi[3 * s]) - from_okey(lo[3 * s]);
  for (int a = 1; a < 3; ++a) {
    const double e = from_okey(hi[3 * s + a]) - from_okey(lo[3 * s + a]);
    if (e > ext) ext = e, best = a;
  }
  axis[s] = (int8_t)best;
  const int32_t P = (size[s] + N - 1) / N;
  width[s] = P > 1 ? 2 : 1;
  left[s] = N * ((P + 1) / 2);
}

__global__ void k_coord_keys(const double* __restrict__ X, const int32_t* __restrict__ label,
                             const int8_t* __restrict__ axis, int32_t n, unsigned long long* __restrict__ key) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) key[v] = okey(X[3 * (int64_t)v + axis[label[v]]]);
}

__global__ void k_gather_label(const int32_t* __restrict__ label, const int32_t* __restrict__ order, int32_t n,
                               uint32_t* __restrict__ out) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = (uint32_t)label[order[p]];
}

// order: vertices by (set, coordinate, index); start: first position of each
// set (exclusive scan of the sizes); first: first new id of each set.
__global__ void k_relabel(const int32_t* __restrict__ order, int32_t n, const int32_t* __restrict__ start,
                          const int32_t* __restrict__ first, const int32_t* __restrict__ width,
                          const int32_t* __restrict__ left, int32_t* __restrict__ label) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t v = order[p];
  const int32_t s = label[v];
  const int32_t rank = p - start[s];
  label[v] = first[s] + ((width[s] == 2 && rank >= left[s]) ? 1 : 0);
}

// ---------------------------------------------------------------- Morton order
__global__ void k_box(const double* __restrict__ X, int32_t n, unsigned long long* __restrict__ lo,
                      unsigned long long* __restrict__ hi) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  for (int a = 0; a < 3; ++a) {
    const unsigned long long k = okey(X[3 * (int64_t)v + a]);
    atomicMin(&lo[a], k);
    atomicMax(&hi[a], k);
  }
}

constexpr int kMortonBits = 10;

__global__ void k_morton(const double* __restrict__ X, int32_t n, const unsigned long long* __restrict__ lo,
                         const unsigned long long* __restrict__ hi, uint32_t* __restrict__ code) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t c = 0;
  for (int a = 0; a < 3; ++a) {
    const double l = from_okey(lo[a]), e = from_okey(hi[a]) - l;
    uint32_t q = 0;
    if (e > 0.0) {
      // the host rule's arithmetic, operation for operation (no contraction)
      const double t = __dmul_rn(__ddiv_rn(__dsub_rn(X[3 * (int64_t)v + a], l), e), (double)(1 << kMortonBits));
      q = (uint32_t)min(floor(t), (double)((1 << kMortonBits) - 1));
    }
    for (int b = 0; b < kMortonBits; ++b) c |= ((q >> b) & 1u) << (3 * b + a);
  }
  code[v] = c;
}

__global__ void k_morton_parts(const int32_t* __restrict__ order, int32_t n, int N, int32_t* __restrict__ label) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) label[order[p]] = p / N;
}

// ---------------------------------------------------------------- slots
__global__ void k_part_sizes(const int32_t* __restrict__ label, int32_t n, int32_t* __restrict__ size) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) atomicAdd(&size[label[v]], 1);
}

__global__ void k_slots(const int32_t* __restrict__ order, int32_t n, const int32_t* __restrict__ label,
                        const int32_t* __restrict__ start, int N, int32_t* __restrict__ map, int* __restrict__ flags) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t v = order[p];
  const int32_t q = label[v];
  const int32_t rank = p - start[q];
  if (rank >= N) atomicOr(flags, kErrIndex);  // a part larger than the domain size (not reachable)
  map[v] = q * N + rank;
}

}  // namespace part

namespace {

// Device buffers of one partition call, freed on every return.
struct Tmp {
  gs_ctx ctx;
  std::vector<void*> ptrs;
  ~Tmp() {
    for (void* p : ptrs) ctx->release(p);
  }
  template <typename T>
  int get(T** out, size_t count) {
    void* p = nullptr;
    GS_TRY(ctx->alloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
    ptrs.push_back(p);
    *out = (T*)p;
    return GS_OK;
  }
};

int read_int(gs_ctx ctx, const int32_t* d, int32_t* h) {
  GS_CUDA(cudaMemcpyAsync(ctx->h_pinned + 8, d, 4, cudaMemcpyDeviceToHost, ctx->stream));
  GS_CUDA(cudaStreamSynchronize(ctx->stream));
  *h = ctx->h_pinned[8];
  return GS_OK;
}

int exclusive_sum(gs_ctx ctx, Tmp& tmp, const int32_t* in, int32_t* out, int32_t count) {
  size_t tb = 0;
  GS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, count, ctx->stream));
  void* t;
  GS_TRY(tmp.get((char**)&t, tb));
  GS_PROF(ctx, GS_K_LIBPRIM);
  GS_CUDA(cub::DeviceScan::ExclusiveSum(t, tb, in, out, count, ctx->stream));
  return GS_OK;
}

template <typename K>
int sort_pairs(gs_ctx ctx, Tmp& tmp, const K* kin, K* kout, const int32_t* vin, int32_t* vout, int32_t count,
               int end_bit) {
  size_t tb = 0;
  GS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, kin, kout, vin, vout, count, 0, end_bit, ctx->stream));
  void* t;
  GS_TRY(tmp.get((char**)&t, tb));
  GS_PROF(ctx, GS_K_LIBPRIM);
  GS_CUDA(cub::DeviceRadixSort::SortPairs(t, tb, kin, kout, vin, vout, count, 0, end_bit, ctx->stream));
  return GS_OK;
}

}  // namespace

// Part label of every vertex by `rule` (GS_PART_*); *n_parts on the host.
int partition_labels(gs_ctx ctx, int32_t n, const double* X, const int32_t* adj_ptr, const int32_t* adj, int32_t N,
                     int32_t rule, int32_t* label, int32_t* n_parts) {
  using namespace part;
  cudaStream_t st = ctx->stream;
  const int gv = ceil_div(n, 256);
  Tmp tmp{ctx};
  int flags = 0;
  { GS_PROF(ctx, GS_K_OTHER); k_check_finite<<<ceil_div(3LL * n, 256), 256, 0, st>>>(X, 3LL * n, ctx->d_flags); }
  GS_TRY(ctx->take_flags(&flags));
  GS_CHECK(!flags, GS_ERR_INVALID, "partition: non-finite position");
  int32_t *order, *order2, *iota;
  GS_TRY(tmp.get(&order, n));
  GS_TRY(tmp.get(&order2, n));
  GS_TRY(tmp.get(&iota, n));
  { GS_PROF(ctx, GS_K_OTHER); k_iota<<<gv, 256, 0, st>>>(iota, n); }

  if (rule == GS_PART_MORTON) {
    unsigned long long* box;
    uint32_t *code, *code2;
    GS_TRY(tmp.get(&box, 6));
    GS_TRY(tmp.get(&code, n));
    GS_TRY(tmp.get(&code2, n));
    GS_CUDA(cudaMemsetAsync(box, 0xff, 3 * 8, st));
    GS_CUDA(cudaMemsetAsync(box + 3, 0, 3 * 8, st));
    { GS_PROF(ctx, GS_K_OTHER); k_box<<<gv, 256, 0, st>>>(X, n, box, box + 3); }
    { GS_PROF(ctx, GS_K_OTHER); k_morton<<<gv, 256, 0, st>>>(X, n, box, box + 3, code); }
    GS_TRY(sort_pairs(ctx, tmp, code, code2, iota, order, n, 3 * kMortonBits));
    { GS_PROF(ctx, GS_K_OTHER); k_morton_parts<<<gv, 256, 0, st>>>(order, n, N, label); }
    *n_parts = (n + N - 1) / N;
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  }

  int32_t S = 1;
  if (rule == GS_PART_RCB_COMPONENTS) {
    GS_CHECK(adj_ptr && adj, GS_ERR_INVALID, "partition: the component rule needs the mesh graph");
    int32_t *parent, *rootf, *rank;
    GS_TRY(tmp.get(&parent, n));
    GS_TRY(tmp.get(&rootf, n + 1));
    GS_TRY(tmp.get(&rank, n + 1));
    int* changed = ctx->d_flags + 32;
    GS_CUDA(cudaMemcpyAsync(parent, iota, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    for (int round = 0;; ++round) {
      GS_CHECK(round < 64 * 1024, GS_ERR_INVALID, "partition: components did not settle");
      GS_CUDA(cudaMemsetAsync(changed, 0, 4, st));
      { GS_PROF(ctx, GS_K_OTHER); k_hook<<<gv, 256, 0, st>>>(adj_ptr, adj, n, parent, changed, ctx->d_flags); }
      { GS_PROF(ctx, GS_K_OTHER); k_compress<<<gv, 256, 0, st>>>(parent, n); }
      int32_t ch = 0;
      GS_TRY(read_int(ctx, changed, &ch));
      if (!ch) break;
    }
    GS_TRY(ctx->take_flags(&flags));
    GS_CHECK(!flags, GS_ERR_INVALID, "partition: a neighbour index is out of range");
    GS_CUDA(cudaMemsetAsync(rootf + n, 0, 4, st));
    { GS_PROF(ctx, GS_K_OTHER); k_root_flags<<<gv, 256, 0, st>>>(parent, n, rootf); }
    GS_TRY(exclusive_sum(ctx, tmp, rootf, rank, n + 1));
    GS_TRY(read_int(ctx, rank + n, &S));
    { GS_PROF(ctx, GS_K_OTHER); k_label_from_roots<<<gv, 256, 0, st>>>(parent, rank, n, label); }
  } else {
    GS_CUDA(cudaMemsetAsync(label, 0, (size_t)n * 4, st));
  }

  // bisection rounds: every set of one depth at once
  int32_t *size, *start, *width, *first, *left;
  unsigned long long *lo, *hi, *key, *key2;
  int8_t* axis;
  uint32_t *lab32, *lab32b;
  GS_TRY(tmp.get(&size, n + 1));
  GS_TRY(tmp.get(&start, n + 1));
  GS_TRY(tmp.get(&width, n + 1));
  GS_TRY(tmp.get(&first, n + 1));
  GS_TRY(tmp.get(&left, n + 1));
  GS_TRY(tmp.get(&lo, 3 * (size_t)n));
  GS_TRY(tmp.get(&hi, 3 * (size_t)n));
  GS_TRY(tmp.get(&key, n));
  GS_TRY(tmp.get(&key2, n));
  GS_TRY(tmp.get(&axis, n));
  GS_TRY(tmp.get(&lab32, n));
  GS_TRY(tmp.get(&lab32b, n));
  for (;;) {
    const int gs_ = ceil_div(S, 256);
    { GS_PROF(ctx, GS_K_OTHER); k_set_init<<<gs_, 256, 0, st>>>(S, size, lo, hi); }
    { GS_PROF(ctx, GS_K_OTHER); k_set_extent<<<gv, 256, 0, st>>>(X, label, n, size, lo, hi); }
    { GS_PROF(ctx, GS_K_OTHER); k_set_plan<<<gs_, 256, 0, st>>>(S, N, size, lo, hi, axis, width, left); }
    GS_CUDA(cudaMemsetAsync(width + S, 0, 4, st));
    GS_TRY(exclusive_sum(ctx, tmp, width, first, S + 1));
    int32_t S2 = 0;
    GS_TRY(read_int(ctx, first + S, &S2));
    if (S2 == S) break;  // no set splits
    { GS_PROF(ctx, GS_K_OTHER); k_coord_keys<<<gv, 256, 0, st>>>(X, label, axis, n, key); }
    GS_TRY(sort_pairs(ctx, tmp, key, key2, iota, order2, n, 64));  // by coordinate, ties by index
    { GS_PROF(ctx, GS_K_OTHER); part::k_gather_label<<<gv, 256, 0, st>>>(label, order2, n, lab32); }
    GS_TRY(sort_pairs(ctx, tmp, lab32, lab32b, order2, order, n, bits_for(S)));  // then by set (stable)
    GS_CUDA(cudaMemsetAsync(size + S, 0, 4, st));
    GS_TRY(exclusive_sum(ctx, tmp, size, start, S + 1));
    { GS_PROF(ctx, GS_K_OTHER); k_relabel<<<gv, 256, 0, st>>>(order, n, start, first, width, left, label); }
    S = S2;
  }
  *n_parts = S;
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs

extern "C" int gs_partition_device(gs_ctx ctx, int32_t n, const double* X, const int32_t* adj_ptr,
                                   const int32_t* adj, int32_t N, int32_t rule, int32_t* map, int32_t* n_domains) {
  using namespace gs;
  GS_CHECK(ctx && X && map && n_domains, GS_ERR_INVALID, "gs_partition_device: null argument");
  GS_CHECK(n >= 1 && N >= 1, GS_ERR_INVALID, "gs_partition_device: n %d, domain size %d", n, N);
  GS_CHECK(rule == GS_PART_RCB || rule == GS_PART_RCB_COMPONENTS || rule == GS_PART_MORTON, GS_ERR_INVALID,
           "gs_partition_device: rule %d", rule);
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  Tmp tmp{ctx};
  int32_t *label, *iota, *order, *lab_sorted, *size, *start;
  GS_TRY(tmp.get(&label, n));
  int32_t M = 0;
  GS_TRY(partition_labels(ctx, n, X, adj_ptr, adj, N, rule, label, &M));
  GS_TRY(tmp.get(&iota, n));
  GS_TRY(tmp.get(&order, n));
  GS_TRY(tmp.get(&lab_sorted, n));
  GS_TRY(tmp.get(&size, M + 1));
  GS_TRY(tmp.get(&start, M + 1));
  const int gv = ceil_div(n, 256);
  { GS_PROF(ctx, GS_K_OTHER); part::k_iota<<<gv, 256, 0, st>>>(iota, n); }
  GS_TRY(sort_pairs(ctx, tmp, label, lab_sorted, iota, order, n, bits_for(M)));  // by part, ties by index
  GS_CUDA(cudaMemsetAsync(size, 0, (size_t)(M + 1) * 4, st));
  { GS_PROF(ctx, GS_K_OTHER); part::k_part_sizes<<<gv, 256, 0, st>>>(label, n, size); }
  GS_TRY(exclusive_sum(ctx, tmp, size, start, M + 1));
  { GS_PROF(ctx, GS_K_OTHER); part::k_slots<<<gv, 256, 0, st>>>(order, n, label, start, N, map, ctx->d_flags); }
  int flags = 0;
  GS_TRY(ctx->take_flags(&flags));
  if (flags) return status_from_flags(flags);
  *n_domains = M;
  return GS_OK;
}

extern "C" int gs_build_mas_mesh(gs_ctx ctx, gs_mat mat, const double* X, int32_t part_rule, const int32_t* adj_ptr,
                                 const int32_t* adj, const int32_t* contacts, int64_t n_contacts,
                                 const gs_mas_opts* opts, gs_mas* out) {
  using namespace gs;
  GS_CHECK(ctx && mat && X && opts && out, GS_ERR_INVALID, "gs_build_mas_mesh: null argument");
  GS_CUDA(cudaSetDevice(ctx->device));
  int32_t* map = nullptr;
  GS_TRY(ctx->alloc((void**)&map, (size_t)std::max(mat->n, 1) * 4));
  int32_t nd = 0;
  int s = gs_partition_device(ctx, mat->n, X, adj_ptr, adj, opts->domain_size, part_rule, map, &nd);
  if (s == GS_OK) s = gs_build_mas(ctx, mat, map, nd, adj_ptr, adj, contacts, n_contacts, opts, out);
  ctx->release(map);
  return s;
}
