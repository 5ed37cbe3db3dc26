// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gipc_mas_pcg.h"

namespace gs {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);

#define GS_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ::gs::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return GS_ERR_CUDA;                                                                 \
    }                                                                                     \
  } while (0)

#define GS_CHECK(cond, status, ...) \
  do {                              \
    if (!(cond)) {                  \
      ::gs::set_error(__VA_ARGS__); \
      return (status);              \
    }                               \
  } while (0)

#define GS_TRY(expr)         \
  do {                       \
    int s_ = (expr);         \
    if (s_ != GS_OK) return s_; \
  } while (0)

// Device-side error flags (bitwise OR of these) written by kernels that
// validate their inputs; the host reads the word at the next sync point.
enum : int {
  kErrIndex = 1,      // an index out of range
  kErrNotSPD = 2,     // non-positive Cholesky pivot / p.Ap <= 0
  kErrNonFinite = 4,  // NaN / Inf in a reduction
  kErrTimeout = 8,    // a bounded device wait gave up
};

int status_from_flags(int flags);

// Word of the context's 256-byte device flag area that counts the chunks
// taken by the work-stealing SpMV (zeroed before each launch).
constexpr int kSpmvCounterWord = 16;

// ------------------------------------------------------------------ memory
// A grow-only device buffer from the stream-ordered pool.
struct Buffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace gs

namespace gs {
// Per-context launch counters and optional CUDA-event timing per class.
struct Prof {
  bool on = false;
  uint32_t timed = 0;
  int64_t launches[GS_K_COUNT] = {};
  double ms[GS_K_COUNT] = {};
  struct Pending {
    int klass;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
};
}  // namespace gs

struct gs_ctx_s {
  gs::Prof prof;
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int tune[GS_TUNE_COUNT] = {2, 2, 4, 4096, 1, 4, 1024, 1, 8};  // GS_TUNE_* launch shapes
  cudaStream_t capture_stream = nullptr;  // private stream for CUDA-graph capture
  int* d_flags = nullptr;     // 256 device bytes: [0] error word, [kSpmvCounterWord] SpMV work counter
  int* h_pinned = nullptr;    // pinned host staging (small readbacks), 4 KiB
  double* noalloc_scratch = nullptr;  // gs_mas_apply_noalloc's fixed array in this context
  std::vector<gs::Buffer> scratch;  // named scratch slots, reused across calls
  int64_t n_allocs = 0;       // device allocations made through alloc() so far
  int64_t alloc_bytes = 0;    // and their total size

  // Stream-ordered allocation on this context's stream.
  int alloc(void** p, size_t bytes);
  void release(void* p);
  // Scratch slot `slot` with at least `bytes` bytes (contents undefined).
  int scratch_buf(int slot, size_t bytes, void** p);
  // Read and clear the device error word (synchronises the stream).
  int take_flags(int* flags);
  int sync();
};

namespace gs {

// Scratch slot ids (each a separate grow-only buffer in the context).
enum ScratchSlot : int {
  kSlotSortKeysIn = 0,
  kSlotSortKeysOut,
  kSlotSortValsIn,
  kSlotSortValsOut,
  kSlotSortTemp,
  kSlotScan,
  kSlotReduce,
  kSlotPcgVectors,
  kSlotPcgScalars,
  kSlotMasLevelVec,
  kSlotMasBuild0,
  kSlotMasBuild1,
  kSlotMasBuild2,
  kSlotMasBuild3,
  kSlotFFSplit,
  kSlotCount
};

// Counts (and, if requested, times) the launch made inside its scope.
struct ProfScope {
  gs_ctx ctx;
  int klass;
  cudaEvent_t a = nullptr;
  ProfScope(gs_ctx c, int k);
  ~ProfScope();
};
#define GS_PROF(ctx, klass) ::gs::ProfScope gs_prof_scope_((ctx), (klass))

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Number of bits needed to write values 0..n (inclusive).
inline int bits_for(long long n) {
  int b = 0;
  while ((1LL << b) <= n) ++b;
  return b;
}

}  // namespace gs

namespace gs {
// Level-0 product of the BF16 form (z = W^T (W r) with BF16 inverse Cholesky
// factors W, FP32 accumulation): tensor cores or FP32 cores; mas_apply_bf16.cu.
bool level0_bf16_on_tensor_cores(gs_ctx ctx, gs_mas mas, int nrhs);
int level0_bf16_prepare(gs_ctx ctx, gs_mas mas, const double* fac0);
int level0_bf16_launch(gs_ctx ctx, gs_mas mas, bool f32_node_major, int nrhs, const void* r, int64_t stride,
                       const void* zl, int64_t lstride, void* z, const int* skip, int* flags);
// Level-0 product of the FP64 form on the BF16 tensor cores by exact digit
// splitting (FP64 accuracy); mas_apply_f64tc.cu.
bool level0_f64tc_usable(gs_ctx ctx, gs_mas mas, int nrhs);
// FP32 level-0 product from a bulk-copied inverse (mas_apply.cu)
bool level0_f32_bulk_usable(gs_mas mas, int nrhs);
int level0_f64tc_prepare(gs_ctx ctx, gs_mas mas);
// skip (device, may be null): the kernels return at once while *skip is set
int level0_f64tc_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* r, int64_t stride, const double* zl,
                        int64_t lstride, double* z, const int* skip = nullptr);
int coarse_f64tc_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* rl, double* zl, int64_t lstride,
                        const int* skip = nullptr);
// The same product from the block lower triangles of the symmetric inverses
// as digit bytes (GS_TUNE_F64_TC = 3, N = 16 or 32); mas_apply_f64sym.cu.
bool f64sym_shape_ok(int N);
int f64sym_prepare(gs_ctx ctx, gs_mas mas);
int f64sym_level0_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* r, int64_t stride, const double* zl,
                         int64_t lstride, double* z, const int* skip);
int f64sym_coarse_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* rl, double* zl, int64_t lstride,
                         const int* skip);
// y = A x (row or SRBK variant) and z = M^{-1} r, with the same skip word
int spmv_launch_skip(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, int variant, const int* skip);
int mas_apply_launch_skip(gs_ctx ctx, gs_mas mas, const double* r, double* z, int nrhs, double* rl, double* zl,
                          const int* skip);
// Float-float SpMV (spmv_ff.cu).  ensure_ff builds the matrix's scaled
// float-float copy once.  spmv_ff_split_launch: y = A x from x already split,
// node-major across RHS: xs[(node * nrhs + k) * 3 + c] = (hi, lo) of
// x_k[3 node + c] * 2^(ff_k[node] - F[k]) (|.| <= 1), F device int[nrhs];
// spmv_ff_launch splits x itself (two extra passes).
int ensure_ff(gs_ctx ctx, gs_mat m);
int spmv_ff_split_launch(gs_ctx ctx, gs_mat m, const float2* xs, const int* F, double* y, int nrhs, const int* skip);
int spmv_ff_launch(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, const int* skip);
}  // namespace gs

struct gs_mat_s {
  int32_t n = 0;        // block rows
  int64_t nnzb = 0;     // stored diagonal + upper blocks
  int32_t* rid = nullptr;
  int32_t* cid = nullptr;
  double* au = nullptr;       // nnzb * 9, row-major blocks
  int32_t* row_ptr = nullptr; // n + 1, over the sorted upper blocks
  // Transposed references for the row-gather SpMV (built lazily):
  // for block row r, the stored blocks (c, r) with c < r, as indices into au.
  int32_t* lo_ptr = nullptr;  // n + 1
  int32_t* lo_idx = nullptr;  // nnzb - n_diag
  int32_t* lo_col = nullptr;  // the c of each such block
  int32_t* row_order = nullptr;  // rows by descending entry count (row-gather SpMV)
  int32_t row_order_window = -1;  // GS_TUNE_SPMV_WINDOW it was built for
  int32_t* key_of_input = nullptr;  // per input block: index of the stored block it was summed into, -1 if dropped
  int64_t n_input = 0;
  float* au32 = nullptr;      // FP32 copy of au for the mixed-precision solve (built lazily)
  // Float-float copy for GS_SPMV_ROW_FF (built lazily): block (r, c) scaled by
  // 2^-(k_r + k_c), k_i = ceil(E_i / 2) with 2^E_i bounding row i's largest
  // entry, so every scaled entry is below 1 in magnitude; stored per entry as
  // (hi, lo) = (rn(a), rn(a - hi)) floats.
  float2* au_ff = nullptr;    // nnzb * 9
  int32_t* ff_k = nullptr;    // n + 1: k_i - K per row; [n] holds K = max_i k_i
  const void* pattern_owner = nullptr;  // the elastic body whose fixed pattern this matrix uses (or null)
  uint64_t pattern_version = 0;        // and that pattern's version
  gs_ctx owner = nullptr;
};

struct gs_mas_s {
  int32_t N = 0;          // domain size
  int32_t n = 0;          // fine nodes
  int32_t L = 0;          // levels
  int32_t precision = 0;
  std::vector<int32_t> n_items;    // per level (level 0: padded slots)
  std::vector<int32_t> n_domains;  // per level
  std::vector<int32_t*> coarse;    // per level: device int32[n] (level 0 = map)
  std::vector<int32_t*> up;        // per level l >= 1 below the top: device int32[n_domains[l] * N],
                                   // the level-(l+1) item of each level-l item (-1: padding)
  int32_t* remap0 = nullptr;       // device int32[n_items[0]], slot -> node or -1
  std::vector<double*> inv64;      // per level: n_domains * (3N)^2
  std::vector<float*> inv32;       // per level (FP32 precision, or made for the mixed solve)
  float* inv32p = nullptr;         // FP32 precision, level 0: each domain's inverse as its lower triangle
                                   // packed by rows (ld(ld+1)/2 floats, padded to a multiple of 4)
  std::vector<void*> inv16;        // BF16 precision: level 0 only, inverse Cholesky factor W, row-major
  void* inv16_tc = nullptr;        // BF16 precision: level-0 W in the tensor-core operand layout
  std::vector<void*> dig64;        // FP64 precision: per level, the inverses as 7 BF16 digit matrices per domain
  std::vector<int32_t*> dig64_exp; // FP64 precision: per level, their row exponents
  void** d_dig_tab = nullptr;      // device table: digit pointers [0..7], exponent pointers [8..15]
  std::vector<void*> dig8;         // FP64 precision, GS_TUNE_F64_TC = 3: per level, the inverses' block lower
                                   // triangles as 8 base-128 digit bytes per entry
  std::vector<int32_t*> dig8_scale;  // their symmetric row scales c_i
  void** d_sym_tab = nullptr;      // device table: digit-byte pointers [0..7], scale pointers [8..15]
  std::vector<int64_t> vec_off;    // per level l >= 1: offset (in items) into the multilevel vector
  int64_t vec_items = 0;           // total items of levels >= 1
  void** d_inv_tab = nullptr;      // device table: inverse pointer per level (FP64 or FP32)
  int32_t* d_coarse_jobs = nullptr;  // device: level then domain of every coarse-level domain
  int32_t n_coarse_jobs = 0;
  float** d_inv32_tab = nullptr;   // device table of FP32 inverse pointers (mixed solve)
  gs_ctx owner = nullptr;
};
