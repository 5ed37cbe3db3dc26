// Device primitives of the hash assembly (Sec. 5.2, Alg. FastHashReduction):
// the radix sort of (key, index) pairs that brings duplicate keys together,
// and the exclusive scan of the run flags that numbers the unique keys.
//
// Sort: least-significant-digit radix sort, 8-bit digits, stable, one pass
// per digit up to end_bit (the last digit masked at end_bit).  A pass is (1) a per-tile digit histogram written
// digit-major (hist[digit * tiles + tile]), (2) an exclusive scan of that
// matrix, which gives every (digit, tile) its first output position, and (3)
// a scatter in which each tile ranks its keys per digit: a warp takes its
// contiguous part of the tile item by item (32 consecutive keys at a time),
// lanes with the same digit find each other by match.any, and their rank is
// the warp's running count of that digit plus the lanes below them in the
// match; the warps' counts are then prefixed in warp order.  Keys keep their
// input order within a digit, so the sort is stable.
//
// Scan: reduce-then-scan over blocks of 4,096 entries: block totals, one
// block scanning the totals, then each block's scan plus its offset.
#include <algorithm>

#include "common.cuh"
#include "primitives.cuh"
#include "sort_scan.cuh"

namespace gs {
namespace prim {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;  // keys per thread per tile
constexpr int kTile = kSortThreads * kSortItems;
constexpr int kWarps = kSortThreads / 32;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanBlock = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                             uint32_t mask, int64_t tiles, int32_t* __restrict__ hist) {
  __shared__ int32_t cnt[256];
  const int tid = threadIdx.x;
  cnt[tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int64_t e = base + i * kSortThreads + tid;
    if (e < n) atomicAdd(&cnt[(int)((keys[e] >> shift) & mask)], 1);
  }
  __syncthreads();
  hist[(int64_t)tid * tiles + blockIdx.x] = cnt[tid];
}

__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(const uint64_t* __restrict__ kin,
                                                                const uint32_t* __restrict__ vin,
                                                                uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                int64_t n, int shift, uint32_t mask, int64_t tiles,
                                                                const int32_t* __restrict__ offs) {
  __shared__ int32_t wcnt[kWarps][256];  // running, then prefixed, count of each digit per warp
  __shared__ int32_t toff[256];          // the tile's first output position per digit
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int d = tid; d < kWarps * 256; d += kSortThreads) (&wcnt[0][0])[d] = 0;
  toff[tid] = offs[(int64_t)tid * tiles + blockIdx.x];
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t wbase = (int64_t)blockIdx.x * kTile + (int64_t)warp * 32 * kSortItems;
  uint64_t k[kSortItems];
  uint32_t v[kSortItems];
  int dg[kSortItems], rank[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int64_t e = wbase + i * 32 + lane;
    const bool valid = e < n;
    k[i] = valid ? kin[e] : 0;
    v[i] = valid ? vin[e] : 0;
    dg[i] = valid ? (int)((k[i] >> shift) & mask) : 256 + lane;  // an invalid lane matches nobody
  }
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const unsigned peers = __match_any_sync(kFull, dg[i]);
    const bool valid = dg[i] < 256;
    const int before = valid ? wcnt[warp][dg[i]] : 0;
    __syncwarp();
    rank[i] = before + __popc(peers & lt);
    if (valid && (peers & lt) == 0) wcnt[warp][dg[i]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive prefix of the warps' counts, per digit, in warp order
    const int d = tid;
    int s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int c = wcnt[w][d];
      wcnt[w][d] = s;
      s += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if (dg[i] >= 256) continue;
    const int64_t pos = (int64_t)toff[dg[i]] + wcnt[warp][dg[i]] + rank[i];
    kout[pos] = k[i];
    vout[pos] = v[i];
  }
}

// ---------------------------------------------------------------- scan
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x, int32_t* s_warp, int32_t* total) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  return s_warp[warp] + inc - x;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* __restrict__ in, int64_t n,
                                                              int32_t* __restrict__ sums) {
  __shared__ int32_t s_warp[32];
  __shared__ int32_t total;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  block_exclusive_scan(s, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of the nb block totals in place.
__global__ void __launch_bounds__(1024) k_scan_top(int32_t* __restrict__ sums, int64_t nb) {
  __shared__ int32_t s_warp[32];
  __shared__ int32_t total;
  const int per = (int)((nb + blockDim.x - 1) / blockDim.x);
  const int64_t base = (int64_t)threadIdx.x * per;
  int32_t s = 0;
  for (int i = 0; i < per; ++i)
    if (base + i < nb) s += sums[base + i];
  int32_t run = block_exclusive_scan(s, s_warp, &total);
  for (int i = 0; i < per; ++i)
    if (base + i < nb) {
      const int32_t v = sums[base + i];
      sums[base + i] = run;
      run += v;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int32_t* in, int32_t* out, int64_t n,
                                                            const int32_t* __restrict__ sums) {
  __shared__ int32_t s_warp[32];
  __shared__ int32_t total;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  int32_t x[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    x[i] = base + i < n ? in[base + i] : 0;
    s += x[i];
  }
  int32_t run = sums[blockIdx.x] + block_exclusive_scan(s, s_warp, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) {
      out[base + i] = run;
      run += x[i];
    }
}

}  // namespace prim

static inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t scan_temp_bytes(int64_t n) {
  const int64_t nb = (n + prim::kScanBlock - 1) / prim::kScanBlock;
  return align256((size_t)std::max<int64_t>(nb, 1) * 4);
}

int exclusive_scan_i32(cudaStream_t st, const int32_t* in, int32_t* out, int64_t n, void* temp, size_t temp_bytes) {
  if (n <= 0) return GS_OK;
  const int64_t nb = (n + prim::kScanBlock - 1) / prim::kScanBlock;
  GS_CHECK(temp_bytes >= scan_temp_bytes(n) && n < (1LL << 31), GS_ERR_INVALID, "exclusive scan: temp or size");
  int32_t* sums = (int32_t*)temp;
  prim::k_scan_reduce<<<(unsigned)nb, prim::kScanThreads, 0, st>>>(in, n, sums);
  prim::k_scan_top<<<1, 1024, 0, st>>>(sums, nb);
  prim::k_scan_down<<<(unsigned)nb, prim::kScanThreads, 0, st>>>(in, out, n, sums);
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

size_t radix_sort_temp_bytes(int64_t n) {
  const int64_t tiles = std::max<int64_t>((n + prim::kTile - 1) / prim::kTile, 1);
  return align256((size_t)std::max<int64_t>(n, 1) * 8) + align256((size_t)std::max<int64_t>(n, 1) * 4) +
         align256((size_t)256 * tiles * 4) + scan_temp_bytes(256 * tiles);
}

int radix_sort_pairs(cudaStream_t st, const uint64_t* k_in, uint64_t* k_out, const uint32_t* v_in, uint32_t* v_out,
                     int64_t n, int end_bit, void* temp, size_t temp_bytes) {
  if (n <= 0) return GS_OK;
  GS_CHECK(temp_bytes >= radix_sort_temp_bytes(n) && end_bit >= 1 && end_bit <= 64 && 256 * ((n + prim::kTile - 1) / prim::kTile) < (1LL << 31),
           GS_ERR_INVALID, "radix sort: temp, end bit or size");
  const int64_t tiles = (n + prim::kTile - 1) / prim::kTile;
  char* t = (char*)temp;
  uint64_t* tk = (uint64_t*)t;
  t += align256((size_t)n * 8);
  uint32_t* tv = (uint32_t*)t;
  t += align256((size_t)n * 4);
  int32_t* hist = (int32_t*)t;
  t += align256((size_t)256 * tiles * 4);
  void* stemp = t;
  const int passes = (end_bit + 7) / 8;
  const uint64_t* ki = k_in;
  const uint32_t* vi = v_in;
  for (int p = 1; p <= passes; ++p) {
    // the last pass lands in the output: pass p writes there when passes - p is even
    uint64_t* ko = (passes - p) % 2 == 0 ? k_out : tk;
    uint32_t* vo = (passes - p) % 2 == 0 ? v_out : tv;
    const int shift = 8 * (p - 1);
    const uint32_t mask = (1u << std::min(8, end_bit - shift)) - 1u;  // the last digit stops at end_bit
    prim::k_digit_hist<<<(unsigned)tiles, prim::kSortThreads, 0, st>>>(ki, n, shift, mask, tiles, hist);
    GS_TRY(exclusive_scan_i32(st, hist, hist, 256 * tiles, stemp, scan_temp_bytes(256 * tiles)));
    prim::k_digit_scatter<<<(unsigned)tiles, prim::kSortThreads, 0, st>>>(ki, vi, ko, vo, n, shift, mask, tiles,
                                                                           hist);
    ki = ko;
    vi = vo;
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs

extern "C" int gs_prim_sort_pairs(gs_ctx ctx, const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                  uint32_t* vals_out, int64_t n, int32_t end_bit) {
  GS_CHECK(ctx && n >= 0 && (n == 0 || (keys_in && vals_in && keys_out && vals_out)), GS_ERR_INVALID,
           "gs_prim_sort_pairs: null argument or negative size");
  GS_CHECK(end_bit >= 1 && end_bit <= 64, GS_ERR_INVALID, "gs_prim_sort_pairs: end_bit %d", end_bit);
  GS_CHECK(keys_in != keys_out && vals_in != vals_out, GS_ERR_INVALID, "gs_prim_sort_pairs: in place");
  if (n == 0) return GS_OK;
  GS_CUDA(cudaSetDevice(ctx->device));
  void* temp = nullptr;
  GS_TRY(ctx->scratch_buf(gs::kSlotSortTemp, gs::radix_sort_temp_bytes(n), &temp));
  GS_PROF(ctx, GS_K_LIBPRIM);
  return gs::radix_sort_pairs(ctx->stream, keys_in, keys_out, vals_in, vals_out, n, end_bit, temp,
                              gs::radix_sort_temp_bytes(n));
}

extern "C" int gs_prim_exclusive_scan(gs_ctx ctx, const int32_t* in, int32_t* out, int64_t n) {
  GS_CHECK(ctx && n >= 0 && (n == 0 || (in && out)), GS_ERR_INVALID, "gs_prim_exclusive_scan: null argument");
  GS_CHECK(n < (1LL << 31), GS_ERR_INVALID, "gs_prim_exclusive_scan: n %lld", (long long)n);
  if (n == 0) return GS_OK;
  GS_CUDA(cudaSetDevice(ctx->device));
  void* temp = nullptr;
  GS_TRY(ctx->scratch_buf(gs::kSlotSortTemp, gs::scan_temp_bytes(n), &temp));
  GS_PROF(ctx, GS_K_LIBPRIM);
  return gs::exclusive_scan_i32(ctx->stream, in, out, n, temp, gs::scan_temp_bytes(n));
}
