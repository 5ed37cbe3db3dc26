// Context, errors and stream-ordered memory.
#include <cstdarg>

#include "common.cuh"

namespace gs {

static thread_local char g_last_error[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int status_from_flags(int flags) {
  if (flags & kErrIndex) {
    set_error("an input index is out of range");
    return GS_ERR_INVALID;
  }
  if (flags & kErrNotSPD) {
    set_error("matrix or preconditioner is not positive definite");
    return GS_ERR_NOT_SPD;
  }
  if (flags & kErrNonFinite) {
    set_error("non-finite value in a reduction");
    return GS_ERR_NONFINITE;
  }
  if (flags & kErrTimeout) {
    set_error("a bounded wait inside a kernel gave up");
    return GS_ERR_TIMEOUT;
  }
  return GS_OK;
}

static cudaEvent_t take_event(Prof& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(gs_ctx c, int k) : ctx(c), klass(k) {
  Prof& p = ctx->prof;
  if (!p.on) return;
  p.launches[k] += 1;
  if (p.timed & (1u << k)) {
    a = take_event(p);
    cudaEventRecord(a, ctx->stream);
  }
}

ProfScope::~ProfScope() {
  if (!a) return;
  Prof& p = ctx->prof;
  cudaEvent_t b = take_event(p);
  cudaEventRecord(b, ctx->stream);
  p.pending.push_back({klass, a, b});
}

}  // namespace gs

int gs_ctx_s::alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return GS_OK;
  GS_CUDA(cudaMallocAsync(p, bytes, stream));
  n_allocs += 1;
  alloc_bytes += (int64_t)bytes;
  return GS_OK;
}

void gs_ctx_s::release(void* p) {
  if (p) cudaFreeAsync(p, stream);
}

int gs_ctx_s::scratch_buf(int slot, size_t bytes, void** p) {
  if ((int)scratch.size() <= slot) scratch.resize(slot + 1);
  gs::Buffer& b = scratch[slot];
  if (b.bytes < bytes) {
    release(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 8 + 256;
    GS_TRY(alloc(&b.ptr, want));
    b.bytes = want;
  }
  *p = b.ptr;
  return GS_OK;
}

int gs_ctx_s::take_flags(int* flags) {
  GS_CUDA(cudaMemcpyAsync(h_pinned, d_flags, sizeof(int), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int), stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  *flags = h_pinned[0];
  return GS_OK;
}

int gs_ctx_s::sync() {
  GS_CUDA(cudaStreamSynchronize(stream));
  return GS_OK;
}

extern "C" {

const char* gs_status_string(int s) {
  switch (s) {
    case GS_OK: return "GS_OK";
    case GS_ERR_INVALID: return "GS_ERR_INVALID";
    case GS_ERR_CUDA: return "GS_ERR_CUDA";
    case GS_ERR_NOT_SPD: return "GS_ERR_NOT_SPD";
    case GS_ERR_MAXITER: return "GS_ERR_MAXITER";
    case GS_ERR_NONFINITE: return "GS_ERR_NONFINITE";
    case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
    case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT";
    default: return "GS_ERR_UNKNOWN";
  }
}

const char* gs_last_error(void) { return gs::g_last_error; }

int gs_create(gs_ctx* out, int device, void* stream) {
  GS_CHECK(out != nullptr, GS_ERR_INVALID, "gs_create: out is null");
  *out = nullptr;
  int count = 0;
  GS_CUDA(cudaGetDeviceCount(&count));
  GS_CHECK(device >= 0 && device < count, GS_ERR_INVALID, "gs_create: device %d of %d", device, count);
  GS_CUDA(cudaSetDevice(device));
  gs_ctx c = new gs_ctx_s();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete c;
    gs::set_error("gs_create: cudaGetDeviceProperties failed");
    return GS_ERR_CUDA;
  }
  c->sm_count = prop.multiProcessorCount;
  // Keep freed pool memory cached by the pool instead of returning it to
  // the CUDA driver at every synchronisation.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (cudaMalloc(&c->d_flags, 256) != cudaSuccess || cudaMallocHost(&c->h_pinned, 4096) != cudaSuccess ||
      cudaMemset(c->d_flags, 0, 256) != cudaSuccess) {
    gs::set_error("gs_create: allocation failed");
    if (c->d_flags) cudaFree(c->d_flags);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
    return GS_ERR_CUDA;
  }
  *out = c;
  return GS_OK;
}

int gs_profile_begin(gs_ctx ctx, uint32_t timed_classes) {
  GS_CHECK(ctx, GS_ERR_INVALID, "gs_profile_begin: null context");
  gs::Prof& p = ctx->prof;
  for (auto& q : p.pending) p.pool.push_back(q.a), p.pool.push_back(q.b);
  p.pending.clear();
  for (int k = 0; k < GS_K_COUNT; ++k) p.launches[k] = 0, p.ms[k] = 0.0;
  p.timed = timed_classes;
  p.on = true;
  return GS_OK;
}

int gs_profile_end(gs_ctx ctx, int64_t* launches, double* ms) {
  GS_CHECK(ctx, GS_ERR_INVALID, "gs_profile_end: null context");
  gs::Prof& p = ctx->prof;
  GS_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& q : p.pending) {
    float t = 0.f;
    GS_CUDA(cudaEventElapsedTime(&t, q.a, q.b));
    p.ms[q.klass] += t;
    p.pool.push_back(q.a);
    p.pool.push_back(q.b);
  }
  p.pending.clear();
  p.on = false;
  for (int k = 0; k < GS_K_COUNT; ++k) {
    if (launches) launches[k] = p.launches[k];
    if (ms) ms[k] = p.ms[k];
  }
  return GS_OK;
}

int gs_tune_set(gs_ctx ctx, int32_t param, int32_t value) {
  GS_CHECK(ctx, GS_ERR_INVALID, "gs_tune_set: null context");
  bool ok = false;
  switch (param) {
    case GS_TUNE_SPMV_LANES: ok = value == 1 || value == 2 || value == 4 || value == 8; break;
    case GS_TUNE_SPMV32_LANES: ok = value == 2 || value == 4; break;
    case GS_TUNE_APPLY_RHS: ok = value == 1 || value == 2 || value == 4 || value == 8; break;
    case GS_TUNE_BATCH_CHUNK: ok = value >= 1024 && value <= 16384 && (value & (value - 1)) == 0; break;
    case GS_TUNE_BF16_TC: ok = value == 0 || value == 1; break;
    case GS_TUNE_F64_TC: ok = value >= 0 && value <= 4; break;
    case GS_TUNE_SPMV_WS: ok = value == 0 || value == 1; break;
    case GS_TUNE_SPMV_FF_RHS: ok = value == 1 || value == 2 || value == 4 || value == 8; break;
    case GS_TUNE_SPMV_WINDOW: ok = value == 0 || (value >= 256 && value <= 65536 && (value & (value - 1)) == 0); break;
    default: break;
  }
  GS_CHECK(ok, GS_ERR_INVALID, "gs_tune_set: value %d not allowed for parameter %d", value, param);
  ctx->tune[param] = value;
  return GS_OK;
}

int gs_tune_get(gs_ctx ctx, int32_t param, int32_t* value) {
  GS_CHECK(ctx && value && param >= 0 && param < GS_TUNE_COUNT, GS_ERR_INVALID, "gs_tune_get: bad argument");
  *value = ctx->tune[param];
  return GS_OK;
}

int gs_ctx_alloc_stats(gs_ctx ctx, int64_t* n_allocs, int64_t* bytes) {
  GS_CHECK(ctx, GS_ERR_INVALID, "gs_ctx_alloc_stats: null context");
  if (n_allocs) *n_allocs = ctx->n_allocs;
  if (bytes) *bytes = ctx->alloc_bytes;
  return GS_OK;
}

int gs_debug_raise_flags(gs_ctx ctx, int32_t flags) {
  GS_CHECK(ctx, GS_ERR_INVALID, "gs_debug_raise_flags: null context");
  GS_CHECK((flags & ~15) == 0, GS_ERR_INVALID, "gs_debug_raise_flags: unknown bits 0x%x", flags);
  GS_CUDA(cudaSetDevice(ctx->device));
  GS_CUDA(cudaStreamSynchronize(ctx->stream));
  GS_CUDA(cudaMemcpy(ctx->h_pinned, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost));
  ctx->h_pinned[0] |= flags;
  GS_CUDA(cudaMemcpy(ctx->d_flags, ctx->h_pinned, sizeof(int), cudaMemcpyHostToDevice));
  return GS_OK;
}

int gs_set_stream(gs_ctx ctx, void* stream) {
  GS_CHECK(ctx != nullptr, GS_ERR_INVALID, "gs_set_stream: null context");
  ctx->stream = (cudaStream_t)stream;
  return GS_OK;
}

int gs_destroy(gs_ctx ctx) {
  if (!ctx) return GS_OK;
  cudaSetDevice(ctx->device);
  for (auto& q : ctx->prof.pending) ctx->prof.pool.push_back(q.a), ctx->prof.pool.push_back(q.b);
  for (auto e : ctx->prof.pool) cudaEventDestroy(e);
  for (auto& b : ctx->scratch) ctx->release(b.ptr);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  cudaFree(ctx->d_flags);
  cudaFreeHost(ctx->h_pinned);
  delete ctx;
  return GS_OK;
}

}  // extern "C"
