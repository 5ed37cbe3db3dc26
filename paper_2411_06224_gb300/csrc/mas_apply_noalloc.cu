// gs_mas_apply_noalloc: the MAS apply without any device allocation.
//
// gs_mas_apply keeps the restricted and coarse-level vectors of an apply in
// a scratch buffer that the context grows on demand from the CUDA memory
// pool.  Some callers cannot allow that: a host application that hands the
// library a fixed device-memory budget at start-up and forbids any later
// cudaMalloc (an allocation there can fail under the cap, or stall every
// stream on the device while the CUDA driver maps memory), or code that must
// not allocate at all once it is running.  This entry point keeps that
// scratch in a fixed array compiled into the library instead.
//
// The array is a file-scope __device__ symbol of kNoAllocDoubles doubles
// (4 MiB).  Every GPU on which the library's module is loaded holds it until
// the process exits.  Host code cannot use the symbol's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call per device should therefore be made before any stream capture
// begins.  The cached address belongs to the device's primary context, so no
// call may follow a cudaDeviceReset in the same process.  All calls share the
// array: the restricted vectors are cleared at the start of every call, and
// two calls whose work overlaps on the GPU (different streams, or different
// threads on one device) race on it.  Where the level-0 product waits on an
// asynchronous copy (tensor-core and bulk-copy kernels), the call waits for
// its stream and returns the status of those bounded waits, like
// gs_mas_apply.
// With the profiler switched on (gs_profile_begin) the library may create
// CUDA events; it is off unless the caller turns it on.

#include "common.cuh"

namespace gs {
constexpr size_t kNoAllocDoubles = size_t(1) << 19;  // 4 MiB of float64
}

// The fixed scratch: restricted vectors (first half of the used part) and
// coarse-level results (second half) of one apply.
static __device__ __align__(256) double g_level_scratch[gs::kNoAllocDoubles];

namespace gs {

int mas_apply_launch(gs_ctx ctx, gs_mas mas, const double* r, double* z, int nrhs, double* rl, double* zl);

namespace {

// Device address of the scratch array, looked up at the context's first call
// (with its device current) and kept in the context: a context made after a
// device reset looks it up again, and later calls make no CUDA call for it
// (so they may run under stream capture).
int scratch_address(gs_ctx ctx, double** out) {
  if (!ctx->noalloc_scratch) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_level_scratch);
    if (e != cudaSuccess) {
      set_error("gs_mas_apply_noalloc: cudaGetSymbolAddress failed on device %d: %s", ctx->device,
                cudaGetErrorString(e));
      return GS_ERR_CUDA;
    }
    ctx->noalloc_scratch = (double*)p;
  }
  *out = ctx->noalloc_scratch;
  return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" int gs_mas_apply_noalloc(gs_ctx ctx, gs_mas mas, const double* r, double* z, int32_t nrhs) {
  GS_CHECK(ctx && mas && r && z && r != z, GS_ERR_INVALID, "gs_mas_apply_noalloc: null or aliased argument");
  GS_CHECK(nrhs >= 1, GS_ERR_INVALID, "gs_mas_apply_noalloc: nrhs %d", nrhs);
  const size_t per = (size_t)nrhs * 3 * (size_t)std::max<int64_t>(mas->vec_items, 1);
  GS_CHECK(2 * per <= gs::kNoAllocDoubles, GS_ERR_INVALID,
           "gs_mas_apply_noalloc: needs %zu doubles of coarse-level scratch (2 x %d RHS x 3 x %lld items), "
           "above the fixed %zu; use gs_mas_apply",
           2 * per, nrhs, (long long)mas->vec_items, gs::kNoAllocDoubles);
  GS_CUDA(cudaSetDevice(ctx->device));
  double* base = nullptr;
  GS_TRY(gs::scratch_address(ctx, &base));
  GS_TRY(gs::mas_apply_launch(ctx, mas, r, z, nrhs, base, base + per));
  if (gs::level0_bf16_on_tensor_cores(ctx, mas, nrhs) || gs::level0_f64tc_usable(ctx, mas, nrhs) ||
      gs::level0_f32_bulk_usable(mas, nrhs)) {
    // The tensor-core kernels end a wait that runs past its limit with a bit
    // in the context's device error word.  Read and clear it here (a copy
    // into the context's pinned word, no allocation), so that this call
    // reports its own timeout and no later call inherits it.
    int flags = 0;
    GS_TRY(ctx->take_flags(&flags));
    if (flags) return gs::status_from_flags(flags);
  }
  return GS_OK;
}
