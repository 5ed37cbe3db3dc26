// Batched PCG over independent systems (this library's batching form; the
// paper solves one system at a time).
//
// The systems are the diagonal blocks of one block-diagonal matrix: system s
// owns block rows [node_off[s], node_off[s+1]).  Assembled and preconditioned
// as one matrix -- each system partitioned on its own, so no level-0 domain
// and, having no edges between systems, no supernode mixes two systems --
// they share every SpMV and MAS-apply launch, while PCG keeps one recurrence
// per system: each dot product is reduced per system (a list of
// (system, chunk) work items; the last block sums each system's partials in
// work order, so the result is deterministic), and alpha, beta and the
// convergence test are per system.  A converged system stops moving.
//
// The iteration loop can run inside one CUDA graph: a conditional WHILE node
// whose body is one PCG iteration and whose last kernel clears the condition
// once every system converged or max_iter iterations ran, so a whole batched
// solve is one graph launch with no host round trip.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "primitives.cuh"

namespace gs {

int spmv_launch(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, int variant);
int mas_apply_launch(gs_ctx ctx, gs_mas mas, const double* r, double* z, int nrhs, double* rl, double* zl);
int mas_level_vectors(gs_ctx ctx, gs_mas mas, int nrhs, double** rl, double** zl);
int ensure_row_order(gs_ctx ctx, gs_mat m);

namespace batch {

constexpr int kT = 256;

struct Head {  // per-batch control words (device)
  int all_conv;
  unsigned counter;
  int flags;
  int iter;  // iterations run (graph mode)
};

struct Arrays {  // per-system scalars (device arrays of length S)
  double *bnorm2, *rz, *alpha, *beta, *rr;
  int *conv, *iters;
  const int32_t *w_seg;  // work item -> system
  const int64_t *w_beg, *w_end;
  const int32_t* w_start;  // system -> first work item (S + 1 entries)
  int S;
};

enum Op : int { kBnorm = 0, kRz0, kPAp, kRR, kRz };

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kT / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

__device__ void finalize(Head* h, const Arrays a, double* __restrict__ partials, double mine, int op, double tol2) {
  __shared__ bool last;
  __shared__ int all;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = mine;
    __threadfence();
    last = atomicInc(&h->counter, gridDim.x - 1) == gridDim.x - 1;
    all = 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  int my_all = 1;
  for (int s = threadIdx.x; s < a.S; s += blockDim.x) {
    double sum = 0.0;
    for (int w = a.w_start[s]; w < a.w_start[s + 1]; ++w) sum += __ldcg(&partials[w]);
    if (!isfinite(sum)) {
      atomicOr(&h->flags, kErrNonFinite);
      a.conv[s] = 1;
      a.alpha[s] = 0.0;
    } else if (op == kBnorm) {
      a.bnorm2[s] = sum;
      a.rr[s] = sum;
      a.conv[s] = sum == 0.0;
      a.iters[s] = 0;
    } else if (op == kRz0) {
      a.rz[s] = sum;
    } else if (op == kPAp) {
      if (a.conv[s]) {
        a.alpha[s] = 0.0;
      } else if (!(sum > 0.0)) {
        atomicOr(&h->flags, kErrNotSPD);
        a.conv[s] = 1;
        a.alpha[s] = 0.0;
      } else {
        a.alpha[s] = a.rz[s] / sum;
      }
    } else if (op == kRR) {
      if (!a.conv[s]) {
        a.rr[s] = sum;
        a.iters[s] += 1;
        if (sum <= tol2 * a.bnorm2[s]) a.conv[s] = 1;
      }
    } else {  // kRz
      a.beta[s] = a.conv[s] ? 0.0 : sum / a.rz[s];
      a.rz[s] = sum;
    }
    my_all &= a.conv[s] != 0;
  }
  if (!my_all) atomicAnd(&all, 0);
  __syncthreads();
  if (threadIdx.x == 0) h->all_conv = all;
}

__global__ void __launch_bounds__(kT) k_binit(const double* __restrict__ b, double* __restrict__ x,
                                              double* __restrict__ r, Head* h, Arrays a,
                                              double* __restrict__ partials) {
  const int w = blockIdx.x;
  double v = 0.0;
  for (int64_t i = a.w_beg[w] + threadIdx.x; i < a.w_end[w]; i += blockDim.x) {
    const double bb = b[i];
    x[i] = 0.0;
    r[i] = bb;
    v += bb * bb;
  }
  finalize(h, a, partials, block_sum(v), kBnorm, 0.0);
}

template <bool kCopy>
__global__ void __launch_bounds__(kT) k_bdot(const double* __restrict__ u, const double* __restrict__ v_,
                                             double* __restrict__ dst, Head* h, Arrays a,
                                             double* __restrict__ partials, int op) {
  if (h->all_conv && op != kRz0) return;
  const int w = blockIdx.x;
  double v = 0.0;
  for (int64_t i = a.w_beg[w] + threadIdx.x; i < a.w_end[w]; i += blockDim.x) {
    const double q = v_[i];
    v = fma(u[i], q, v);
    if (kCopy) dst[i] = q;
  }
  finalize(h, a, partials, block_sum(v), op, 0.0);
}

__global__ void __launch_bounds__(kT) k_bupdate_xr(double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ Ap,
                                                   Head* h, Arrays a, double* __restrict__ partials, double tol2) {
  if (h->all_conv) return;
  const int w = blockIdx.x;
  const double al = a.alpha[a.w_seg[w]];
  double v = 0.0;
  for (int64_t i = a.w_beg[w] + threadIdx.x; i < a.w_end[w]; i += blockDim.x) {
    double ri = r[i];
    if (al != 0.0) {
      x[i] = fma(al, p[i], x[i]);
      ri = fma(-al, Ap[i], ri);
      r[i] = ri;
    }
    v = fma(ri, ri, v);
  }
  finalize(h, a, partials, block_sum(v), kRR, tol2);
}

__global__ void __launch_bounds__(kT) k_bupdate_p(double* __restrict__ p, const double* __restrict__ z, Head* h,
                                                  Arrays a) {
  const int w = blockIdx.x;
  const int s = a.w_seg[w];
  if (h->all_conv || a.conv[s]) return;
  const double be = a.beta[s];
  for (int64_t i = a.w_beg[w] + threadIdx.x; i < a.w_end[w]; i += blockDim.x) p[i] = fma(be, p[i], z[i]);
}

// Last kernel of a graph iteration: keep looping while some system runs and
// fewer than max_iter iterations have been done (the loop always ends).
__global__ void k_loop_condition(cudaGraphConditionalHandle cond, Head* h, int max_iter) {
  const int it = ++h->iter;
  cudaGraphSetConditional(cond, (!h->all_conv && !h->flags && it < max_iter) ? 1u : 0u);
}

}  // namespace batch

extern "C" int gs_pcg_solve_batch(gs_ctx ctx, gs_mat mat, gs_mas mas, int32_t n_sys, const int32_t* node_off,
                                  const double* b, double tol, int32_t max_iter, int32_t use_graph, double* x,
                                  int32_t* iters, double* rel_res) {
  using namespace batch;
  GS_CHECK(ctx && mat && mas && node_off && b && x && b != x, GS_ERR_INVALID, "gs_pcg_solve_batch: null argument");
  GS_CHECK(n_sys >= 1, GS_ERR_INVALID, "gs_pcg_solve_batch: n_sys %d", n_sys);
  GS_CHECK(mas->n == mat->n && node_off[0] == 0 && node_off[n_sys] == mat->n, GS_ERR_INVALID,
           "gs_pcg_solve_batch: node offsets do not span the matrix");
  for (int s = 0; s < n_sys; ++s)
    GS_CHECK(node_off[s + 1] >= node_off[s], GS_ERR_INVALID, "gs_pcg_solve_batch: offsets not ascending");
  GS_CHECK(tol >= 0.0 && max_iter >= 0, GS_ERR_INVALID, "gs_pcg_solve_batch: tol %g max_iter %d", tol, max_iter);
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int64_t len = 3LL * mat->n;
  // work list: chunks of every system's entries, in system order
  const int64_t kChunk = ctx->tune[GS_TUNE_BATCH_CHUNK];
  std::vector<int32_t> w_seg, w_start(n_sys + 1);
  std::vector<int64_t> w_beg, w_end;
  for (int s = 0; s < n_sys; ++s) {
    w_start[s] = (int32_t)w_seg.size();
    const int64_t b0 = 3LL * node_off[s], b1 = 3LL * node_off[s + 1];
    for (int64_t c = b0; c < b1; c += kChunk) {
      w_seg.push_back(s);
      w_beg.push_back(c);
      w_end.push_back(std::min(c + kChunk, b1));
    }
  }
  w_start[n_sys] = (int32_t)w_seg.size();
  if (w_seg.empty()) {  // all systems empty
    w_seg.push_back(0), w_beg.push_back(0), w_end.push_back(0);
  }
  const int W = (int)w_seg.size();
  // device buffers: vectors r, z, p, Ap; scalars; work list; partials
  double* vec = nullptr;
  GS_TRY(ctx->scratch_buf(kSlotPcgVectors, 4 * (size_t)len * sizeof(double) + 64, (void**)&vec));
  double *r = vec, *z = r + len, *p = z + len, *Ap = p + len;
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t sz = r256(sizeof(Head)) + 5 * r256((size_t)n_sys * 8) + 2 * r256((size_t)n_sys * 4) +
                    r256((size_t)W * 4) + 2 * r256((size_t)W * 8) + r256((size_t)(n_sys + 1) * 4) +
                    r256((size_t)W * 8) + 256;
  char* buf = nullptr;
  GS_TRY(ctx->scratch_buf(kSlotPcgScalars, sz, (void**)&buf));
  auto take = [&](size_t bytes) {
    char* q = buf;
    buf += (bytes + 255) / 256 * 256;
    return q;
  };
  Head* h = (Head*)take(sizeof(Head));
  Arrays a{};
  a.S = n_sys;
  a.bnorm2 = (double*)take(n_sys * 8);
  a.rz = (double*)take(n_sys * 8);
  a.alpha = (double*)take(n_sys * 8);
  a.beta = (double*)take(n_sys * 8);
  a.rr = (double*)take(n_sys * 8);
  a.conv = (int*)take(n_sys * 4);
  a.iters = (int*)take(n_sys * 4);
  int32_t* d_wseg = (int32_t*)take(W * 4);
  int64_t* d_wbeg = (int64_t*)take(W * 8);
  int64_t* d_wend = (int64_t*)take(W * 8);
  int32_t* d_wstart = (int32_t*)take((n_sys + 1) * 4);
  double* partials = (double*)take(W * 8);
  a.w_seg = d_wseg, a.w_beg = d_wbeg, a.w_end = d_wend, a.w_start = d_wstart;
  GS_CUDA(cudaMemcpyAsync(d_wseg, w_seg.data(), W * 4, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyAsync(d_wbeg, w_beg.data(), W * 8, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyAsync(d_wend, w_end.data(), W * 8, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyAsync(d_wstart, w_start.data(), (n_sys + 1) * 4, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemsetAsync(h, 0, sizeof(Head), st));
  GS_TRY(ensure_row_order(ctx, mat));
  double *rl, *zl;
  GS_TRY(mas_level_vectors(ctx, mas, 1, &rl, &zl));
  const double tol2 = tol * tol;
  { GS_PROF(ctx, GS_K_PCG_VECTOR); k_binit<<<W, kT, 0, st>>>(b, x, r, h, a, partials); }
  GS_TRY(mas_apply_launch(ctx, mas, r, z, 1, rl, zl));
  { GS_PROF(ctx, GS_K_PCG_VECTOR); k_bdot<true><<<W, kT, 0, st>>>(r, z, p, h, a, partials, kRz0); }

  // One PCG iteration on the context's current stream (the capture stream
  // while a graph body is being recorded).
  auto iteration = [&]() -> int {
    const cudaStream_t cs = ctx->stream;
    GS_TRY(spmv_launch(ctx, mat, p, Ap, 1, GS_SPMV_ROW));
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_bdot<false><<<W, kT, 0, cs>>>(p, Ap, nullptr, h, a, partials, kPAp); }
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_bupdate_xr<<<W, kT, 0, cs>>>(x, r, p, Ap, h, a, partials, tol2); }
    GS_TRY(mas_apply_launch(ctx, mas, r, z, 1, rl, zl));
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_bdot<false><<<W, kT, 0, cs>>>(r, z, nullptr, h, a, partials, kRz); }
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_bupdate_p<<<W, kT, 0, cs>>>(p, z, h, a); }
    return GS_OK;
  };

  if (use_graph && max_iter > 0) {
    // One graph: a WHILE node whose body is one iteration plus the condition
    // update.  Capture needs a stream other than the legacy default stream,
    // so the body is captured on the context's private capture stream.
    if (!ctx->capture_stream) GS_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int status = GS_OK;
    const bool prof = ctx->prof.on;
    const cudaStream_t main_stream = ctx->stream;
    ctx->prof.on = false;  // no event records inside the captured body
    do {
      if (cudaGraphCreate(&graph, 0) != cudaSuccess) { status = GS_ERR_CUDA; break; }
      cudaGraphConditionalHandle cond;
      if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        status = GS_ERR_CUDA;
        break;
      }
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = cond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) != cudaSuccess) { status = GS_ERR_CUDA; break; }
      cudaGraph_t body = np.conditional.phGraph_out[0];
      ctx->stream = ctx->capture_stream;
      if (cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
          cudaSuccess) {
        status = GS_ERR_CUDA;
        break;
      }
      const cudaStream_t cs = ctx->stream;
      int s1 = iteration();
      batch::k_loop_condition<<<1, 1, 0, cs>>>(cond, h, max_iter);
      cudaError_t el = cudaGetLastError();
      cudaGraph_t captured = nullptr;
      cudaError_t ec = cudaStreamEndCapture(cs, &captured);
      if (ec == cudaSuccess && el != cudaSuccess) ec = el;
      ctx->stream = main_stream;
      if (s1 != GS_OK || ec != cudaSuccess) { status = s1 != GS_OK ? s1 : GS_ERR_CUDA; break; }
      if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) { status = GS_ERR_CUDA; break; }
      if (cudaGraphLaunch(exec, main_stream) != cudaSuccess) { status = GS_ERR_CUDA; break; }
    } while (false);
    ctx->stream = main_stream;
    ctx->prof.on = prof;
    if (status != GS_OK) {
      cudaGetLastError();
      set_error("gs_pcg_solve_batch: graph construction or launch failed");
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (status != GS_OK) return status;
  } else {
    int* hflag = ctx->h_pinned + 256;
    for (int it = 0; it < max_iter; ++it) {
      GS_TRY(iteration());
      if ((it + 1) % 8 == 0) {
        GS_CUDA(cudaMemcpyAsync(hflag, &h->all_conv, 4, cudaMemcpyDeviceToHost, st));
        GS_CUDA(cudaStreamSynchronize(st));
        if (*hflag) break;
      }
    }
  }
  GS_CUDA(cudaGetLastError());
  std::vector<int> hconv(n_sys), hit(n_sys);
  std::vector<double> hbn(n_sys), hrr(n_sys);
  Head hh;
  GS_CUDA(cudaMemcpyAsync(hconv.data(), a.conv, n_sys * 4, cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaMemcpyAsync(hit.data(), a.iters, n_sys * 4, cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaMemcpyAsync(hbn.data(), a.bnorm2, n_sys * 8, cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaMemcpyAsync(hrr.data(), a.rr, n_sys * 8, cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaMemcpyAsync(&hh, h, sizeof(Head), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  bool all = true;
  for (int s = 0; s < n_sys; ++s) {
    if (iters) iters[s] = hit[s];
    if (rel_res) rel_res[s] = hbn[s] > 0 ? std::sqrt(hrr[s] / hbn[s]) : 0.0;
    all = all && hconv[s];
  }
  int flags = 0;
  GS_TRY(ctx->take_flags(&flags));
  if (hh.flags) return status_from_flags(hh.flags);
  if (flags) return status_from_flags(flags);
  if (!all) {
    set_error("gs_pcg_solve_batch: not every system converged in %d iterations", max_iter);
    return GS_ERR_MAXITER;
  }
  return GS_OK;
}

}  // namespace gs
