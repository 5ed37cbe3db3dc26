// Mixed-precision MAS-PCG: FP64 iterative refinement around an FP32 inner
// MAS-PCG (this library's precision form; the paper solves in FP64).
//
// One PCG recurrence runs in FP32 (FP32 copy of the stored blocks, MAS
// inverses in FP32 with FP32 accumulation; the p.Ap and r.z reductions
// accumulate in FP64 and alpha, beta are FP64), accumulating its update d.
// Reliable updates refine it in FP64: once the FP32 residual of RHS k has
// fallen by inner_tol since its last correction (or below tol ||b_k||),
// x += d in FP64, the residual is recomputed as r = b - A x with the FP64
// SpMV, d restarts at 0, and the recurrence continues from the corrected
// residual with its search direction kept -- so Krylov information is not
// thrown away as a restarted refinement would.  RHS k stops once the true
// residual satisfies ||r_k|| <= tol ||b_k||, so the answer meets the same
// test as the FP64 solver.
//
// Inner vectors are interleaved node-major over the right-hand sides,
// v[(node * R + k) * 3 + c], so one block of the SpMV meets the R
// right-hand sides of a neighbour in one contiguous 12 R-byte run, and the
// MAS apply gathers a node's residuals in one run.  R is a compile-time 1,
// 2, 4 or 8; other counts are padded with zero right-hand sides.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "primitives.cuh"

namespace gs {

int spmv_launch(gs_ctx ctx, gs_mat m, const double* x, double* y, int nrhs, int variant);
int ensure_row_order(gs_ctx ctx, gs_mat m);

namespace mixed {

constexpr int kT = 256;
constexpr int kMaxBlocks = 512;
constexpr int kMaxR = 8;

struct Scalars {
  double rnorm2[kMaxR];   // outer: ||r||^2 (FP64 residual)
  double bnorm2[kMaxR];   // ||b||^2
  double inner_ref[kMaxR];  // inner target: inner_tol^2 ||r||^2 at the outer step
  double rz[kMaxR], alpha[kMaxR], beta[kMaxR], rr[kMaxR];
  int conv_out[kMaxR];    // RHS finished: true residual below tol
  int want[kMaxR];        // RHS asks for a reliable update
  int iters[kMaxR];       // FP32 iterations (SpMVs) per RHS
  int any_want, all_out;
  unsigned counter;
  int flags;
};

enum Op : int { kOuterNorm = 0, kInRz0, kInPAp, kInRR, kInRz };

inline int nblocks(int64_t items) {
  int64_t g = (items + kT * 4 - 1) / (kT * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxBlocks));
}

template <int R>
__device__ __forceinline__ void block_sum_r(double (&v)[R], double* __restrict__ partials) {
  __shared__ double red[kT / 32][R];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) red[w][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < R) {
    double s = 0.0;
    for (int q = 0; q < kT / 32; ++q) s += red[q][threadIdx.x];
    partials[blockIdx.x * kMaxR + threadIdx.x] = s;
  }
}

__device__ void apply_op(Scalars* s, int k, double sum, int op, double tol2, double itol2) {
  if (!isfinite(sum)) {
    atomicOr(&s->flags, kErrNonFinite);
    s->conv_out[k] = 1;
    s->alpha[k] = 0.0;
    return;
  }
  switch (op) {
    case kOuterNorm:  // sum = ||b - A x||^2 of the FP64 residual (a reliable update)
      s->rnorm2[k] = sum;
      if (!s->conv_out[k] && sum <= tol2 * s->bnorm2[k]) s->conv_out[k] = 1;
      s->inner_ref[k] = itol2 * sum;
      s->want[k] = 0;
      break;
    case kInRz0:
      s->rz[k] = sum;
      break;
    case kInPAp:
      if (s->conv_out[k]) {
        s->alpha[k] = 0.0;
      } else if (!(sum > 0.0)) {
        atomicOr(&s->flags, kErrNotSPD);
        s->conv_out[k] = 1;
        s->alpha[k] = 0.0;
      } else {
        s->alpha[k] = s->rz[k] / sum;
      }
      break;
    case kInRR:
      if (!s->conv_out[k]) {
        s->rr[k] = sum;
        s->iters[k] += 1;
        if (sum <= s->inner_ref[k] || sum <= tol2 * s->bnorm2[k]) s->want[k] = 1;
      }
      break;
    case kInRz:
      s->beta[k] = s->conv_out[k] ? 0.0 : sum / s->rz[k];
      s->rz[k] = sum;
      break;
  }
}

template <int R>
__device__ void finalize(Scalars* s, const double* __restrict__ partials, int nrhs, int op, double tol2, double itol2) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicInc(&s->counter, gridDim.x - 1) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    const int k = threadIdx.x;
    double sum = 0.0;
    if (k < R)
      for (int b = 0; b < (int)gridDim.x; ++b) sum += __ldcg(&partials[b * kMaxR + k]);
    // each lane sums its own RHS over the blocks in block order
    if (k < nrhs) {
      apply_op(s, k, sum, op, tol2, itol2);
    } else if (k < kMaxR) {  // padding right-hand sides never run
      s->conv_out[k] = 1;
      s->want[k] = 0;
    }
    const bool done = k >= nrhs || s->conv_out[k];
    const bool w = k < nrhs && !s->conv_out[k] && s->want[k];
    const bool ao = __all_sync(kFull, done), aw = __any_sync(kFull, w);
    if (k == 0) {
      s->all_out = ao;
      s->any_want = aw;
    }
  }
}

// ---------------------------------------------------------------- outer (FP64, RHS-major)
// r = b - Ax (Ax computed by the FP64 SpMV into r), ||r||^2 per RHS, and the
// FP32 interleaved copy of r that the inner solve starts from.
template <int R>
__global__ void __launch_bounds__(kT) k_outer_residual(const double* __restrict__ b, double* __restrict__ r,
                                                       float* __restrict__ rin, float* __restrict__ d, int32_t n,
                                                       int nrhs, Scalars* s, double* __restrict__ partials,
                                                       double tol2, double itol2, bool first) {
  double v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = 0.0;
  const int64_t stride = 3LL * n;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double rv = 0.0;
        if (k < nrhs) {
          const int64_t o = k * stride + 3 * node + c;
          rv = first ? b[o] : b[o] - r[o];  // r holds A x on later steps
          r[o] = rv;
        }
        v[k] += rv * rv;
        rin[(node * R + k) * 3 + c] = (float)rv;
        d[(node * R + k) * 3 + c] = 0.0f;
      }
    }
  }
  block_sum_r<R>(v, partials);
  finalize<R>(s, partials, nrhs, kOuterNorm, tol2, itol2);
}

// x += d (FP32 interleaved -> FP64 RHS-major) for RHS still running.
template <int R>
__global__ void k_outer_update(double* __restrict__ x, const float* __restrict__ d, int32_t n, int nrhs,
                               const Scalars* s) {
  const int64_t stride = 3LL * n;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (k >= nrhs || s->conv_out[k]) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) x[k * stride + 3 * node + c] += (double)d[(node * R + k) * 3 + c];
    }
  }
}

// ---------------------------------------------------------------- inner (FP32, interleaved)
template <int R, bool kCopy>
__global__ void __launch_bounds__(kT) k_in_dot(const float* __restrict__ a, const float* __restrict__ b,
                                               float* __restrict__ dst, int32_t n, int nrhs, Scalars* s,
                                               double* __restrict__ partials, int op) {
  if (s->all_out && op != kInRz0) return;
  double v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
    const float* pa = a + node * R * 3;
    const float* pb = b + node * R * 3;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float bb = pb[3 * k + c];
        acc = fmaf(pa[3 * k + c], bb, acc);
        if (kCopy) dst[node * R * 3 + 3 * k + c] = bb;
      }
      v[k] += (double)acc;
    }
  }
  block_sum_r<R>(v, partials);
  finalize<R>(s, partials, nrhs, op, 0.0, 0.0);
}

template <int R>
__global__ void __launch_bounds__(kT) k_in_update_dr(float* __restrict__ d, float* __restrict__ r,
                                                     const float* __restrict__ p, const float* __restrict__ Ap,
                                                     int32_t n, int nrhs, Scalars* s,
                                                     double* __restrict__ partials) {
  if (s->all_out) return;
  float al[R];
#pragma unroll
  for (int k = 0; k < R; ++k) al[k] = (float)s->alpha[k];
  double v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = node * R * 3;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float rk = r[o + 3 * k + c];
        if (al[k] != 0.0f) {
          d[o + 3 * k + c] = fmaf(al[k], p[o + 3 * k + c], d[o + 3 * k + c]);
          rk = fmaf(-al[k], Ap[o + 3 * k + c], rk);
          r[o + 3 * k + c] = rk;
        }
        acc = fmaf(rk, rk, acc);
      }
      v[k] += (double)acc;
    }
  }
  block_sum_r<R>(v, partials);
  finalize<R>(s, partials, nrhs, kInRR, 0.0, 0.0);
}

template <int R>
__global__ void k_in_update_p(float* __restrict__ p, const float* __restrict__ z, int32_t n, const Scalars* s) {
  if (s->all_out) return;
  float be[R];
  bool run[R];
#pragma unroll
  for (int k = 0; k < R; ++k) be[k] = (float)s->beta[k], run[k] = !s->conv_out[k];
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = node * R * 3;
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (run[k])
#pragma unroll
        for (int c = 0; c < 3; ++c) p[o + 3 * k + c] = fmaf(be[k], p[o + 3 * k + c], z[o + 3 * k + c]);
  }
}

// FP32 SpMV on the interleaved layout: kLanes lanes per block row, each
// holding the R right-hand sides of its rows in registers.
template <int R, int kLanes>
__global__ void __launch_bounds__(256) k_spmv32(const int32_t* __restrict__ row_order,
                                                const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cid,
                                                const int32_t* __restrict__ lo_ptr, const int32_t* __restrict__ lo_idx,
                                                const int32_t* __restrict__ lo_col, const float* __restrict__ au,
                                                int32_t n, const float* __restrict__ x, float* __restrict__ y,
                                                const Scalars* s) {
  if (s->all_out) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t slot = (int32_t)(t / kLanes);
  const int sub = threadIdx.x % kLanes;
  const bool in = slot < n;
  const int32_t row = in ? row_order[slot] : 0;  // longest rows first: equal lengths share a warp
  int32_t u0 = 0, u1 = 0, l0 = 0, l1 = 0;
  if (in) {
    u0 = row_ptr[row], u1 = row_ptr[row + 1];
    l0 = lo_ptr[row], l1 = lo_ptr[row + 1];
  }
  const int32_t nu = u1 - u0, total = nu + (l1 - l0);
  float acc[3 * R];
#pragma unroll
  for (int k = 0; k < 3 * R; ++k) acc[k] = 0.0f;
  for (int32_t e = sub; e < total; e += kLanes) {
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
    float H[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) H[q] = au[blk * 9 + q];
    if (!upper) {
      float t1 = H[1], t2 = H[2], t5 = H[5];
      H[1] = H[3], H[2] = H[6], H[5] = H[7];
      H[3] = t1, H[6] = t2, H[7] = t5;
    }
    const float* xc = x + (int64_t)col * R * 3;
    float xv[3 * R];
    if ((3 * R) % 4 == 0) {
#pragma unroll
      for (int q = 0; q < 3 * R / 4; ++q) {
        float4 f = reinterpret_cast<const float4*>(xc)[q];
        xv[4 * q] = f.x, xv[4 * q + 1] = f.y, xv[4 * q + 2] = f.z, xv[4 * q + 3] = f.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3 * R; ++q) xv[q] = xc[q];
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float a = acc[3 * k + c];
        a = fmaf(H[3 * c + 0], xv[3 * k + 0], a);
        a = fmaf(H[3 * c + 1], xv[3 * k + 1], a);
        acc[3 * k + c] = fmaf(H[3 * c + 2], xv[3 * k + 2], a);
      }
  }
#pragma unroll
  for (int k = 0; k < 3 * R; ++k)
#pragma unroll
    for (int o = kLanes / 2; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(kFull, acc[k], o, kLanes);
  if (in && sub == 0) {
    float* yr = y + (int64_t)row * R * 3;
    if ((3 * R) % 4 == 0) {
#pragma unroll
      for (int q = 0; q < 3 * R / 4; ++q)
        reinterpret_cast<float4*>(yr)[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    } else {
#pragma unroll
      for (int q = 0; q < 3 * R; ++q) yr[q] = acc[q];
    }
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ---------------------------------------------------------------- MAS apply, FP32 interleaved
struct Levels32 {
  const int32_t* coarse[8];
  int64_t vec_off[8];
  int L;
  int N;
};

// Restriction: one warp per level-0 domain; sums per coarse item, FP32 in, FP32 out.
template <int R>
__global__ void k_restrict32(const float* __restrict__ r, const int32_t* __restrict__ remap0, int32_t n_dom0,
                             Levels32 al, float* __restrict__ rl, const Scalars* s) {
  if (s->all_out) return;
  const int32_t d = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (d >= n_dom0) return;
  const int N = al.N;
  const int32_t node = lane < N ? remap0[(int64_t)d * N + lane] : -1;
  const bool real = node >= 0;
  float v[3 * R];
#pragma unroll
  for (int q = 0; q < 3 * R; ++q) v[q] = real ? r[(int64_t)node * R * 3 + q] : 0.0f;
  // level 1 only: its items lie inside this domain, so the warp stores each
  // item's sum; coarser levels follow from level 1 in k_restrict_up
  const int32_t c = real ? al.coarse[1][node] : -1;
  uint32_t left = __ballot_sync(kFull, real);
  while (left) {
    const int lead = __ffs(left) - 1;
    const int32_t cc = __shfl_sync(kFull, c, lead);
    const uint32_t g = __ballot_sync(kFull, real && c == cc);
    left &= ~g;
    const bool mine = (g >> lane) & 1u;
#pragma unroll
    for (int q = 0; q < 3 * R; ++q) {
      float t = warp_sum(mine ? v[q] : 0.0f);
      if (lane == 0) rl[(al.vec_off[1] + cc) * R * 3 + q] = t;
    }
  }
}

// Coarse levels: one thread per (domain row i, RHS k).  Ts: stored inverse type.
template <int R, typename Ts>
__global__ void __launch_bounds__(256) k_coarse32(const Ts* const* __restrict__ inv, const int32_t* __restrict__ jl,
                                                  const int32_t* __restrict__ jd, int n_jobs, int N, Levels32 al,
                                                  const float* __restrict__ rl, float* __restrict__ zl,
                                                  const Scalars* s) {
  if (s->all_out) return;
  const int ld = 3 * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)ld * R;
  if (t >= per * n_jobs) return;
  const int job = (int)(t / per), rem = (int)(t % per);
  const int k = rem / ld, i = rem % ld;
  const int l = jl[job];
  const int32_t d = jd[job];
  const Ts* Mi = inv[l] + (int64_t)d * ld * ld;
  const int64_t base = al.vec_off[l] + (int64_t)d * N;  // first item of the domain
  float acc = 0.0f;
#pragma unroll 8
  for (int j = 0; j < ld; ++j)
    acc = fmaf(widen(Mi[(int64_t)j * ld + i]), rl[((base + j / 3) * R + k) * 3 + j % 3], acc);
  zl[((base + i / 3) * R + k) * 3 + i % 3] = acc;
}

// Level 0 + prolongation: one CTA per domain, thread = (row i, RHS group).
template <int R, typename Ts>
__global__ void __launch_bounds__(384) k_level0_32(const Ts* __restrict__ inv0, const int32_t* __restrict__ remap0,
                                                   int N, Levels32 al, const float* __restrict__ r,
                                                   const float* __restrict__ zl, float* __restrict__ z,
                                                   const Scalars* s) {
  if (s->all_out) return;
  constexpr int kG = R >= 4 ? 4 : R;  // RHS per thread
  extern __shared__ float sr32[];     // [R][3N]
  const int ld = 3 * N;
  const int32_t d = blockIdx.x;
  const Ts* Mi = inv0 + (int64_t)d * ld * ld;
  for (int e = threadIdx.x; e < ld * R; e += blockDim.x) {
    const int slot = e / (3 * R), rem = e % (3 * R);  // coalesced over a node's 3R values
    const int k = rem / 3, c = rem % 3;
    const int32_t node = remap0[(int64_t)d * N + slot];
    sr32[k * ld + 3 * slot + c] = node >= 0 ? r[(int64_t)node * R * 3 + rem] : 0.0f;
  }
  __syncthreads();
  const int i = threadIdx.x % ld, g = threadIdx.x / ld;
  const int k0 = g * kG;
  if (k0 >= R) return;
  float acc[kG];
#pragma unroll
  for (int q = 0; q < kG; ++q) acc[q] = 0.0f;
#pragma unroll 4
  for (int j = 0; j < ld; ++j) {
    const float m = widen(Mi[(int64_t)j * ld + i]);
#pragma unroll
    for (int q = 0; q < kG; ++q) acc[q] = fmaf(m, sr32[(k0 + q) * ld + j], acc[q]);
  }
  const int32_t node = remap0[(int64_t)d * N + i / 3];
  if (node < 0) return;
  const int c = i % 3;
#pragma unroll
  for (int q = 0; q < kG; ++q) {
    const int k = k0 + q;
    float v = acc[q];
    for (int l = 1; l < al.L; ++l) v += zl[((al.vec_off[l] + al.coarse[l][node]) * R + k) * 3 + c];
    z[((int64_t)node * R + k) * 3 + c] = v;
  }
}

}  // namespace mixed

// FP32 copies of the matrix blocks and the domain inverses (built once).
static int ensure_f32(gs_ctx ctx, gs_mat m, gs_mas mas, float** au32, std::vector<float*>& inv) {
  static_assert(sizeof(float) == 4, "");
  cudaStream_t st = ctx->stream;
  if (!m->au32) {
    GS_TRY(ctx->alloc((void**)&m->au32, (size_t)std::max<int64_t>(m->nnzb, 1) * 9 * 4));
    if (m->nnzb) {
      GS_PROF(ctx, GS_K_OTHER);
      mixed::k_f64_to_f32<<<ceil_div(m->nnzb * 9, 256), 256, 0, st>>>(m->au, m->au32, m->nnzb * 9);
    }
  }
  *au32 = m->au32;
  // BF16 form: inv32 holds the FP32 coarse levels (level 0 is the BF16 factor)
  if (mas->inv32.empty()) {
    const int ld = 3 * mas->N;
    for (int l = 0; l < mas->L; ++l) {
      float* f = nullptr;
      const int64_t cnt = (int64_t)mas->n_domains[l] * ld * ld;
      GS_TRY(ctx->alloc((void**)&f, (size_t)cnt * 4));
      mas->inv32.push_back(f);
      GS_PROF(ctx, GS_K_OTHER);
      mixed::k_f64_to_f32<<<ceil_div(cnt, 256), 256, 0, st>>>(mas->inv64[l], f, cnt);
    }
  }
  inv = mas->inv32;
  if (!mas->d_inv32_tab) {
    GS_TRY(ctx->alloc((void**)&mas->d_inv32_tab, 8 * sizeof(float*)));
    std::vector<float*> hp(8, nullptr);
    for (int l = 0; l < mas->L; ++l) hp[l] = mas->inv32[l];
    GS_CUDA(cudaMemcpyAsync(mas->d_inv32_tab, hp.data(), 8 * sizeof(float*), cudaMemcpyHostToDevice, st));
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template <int R>
static int solve_mixed(gs_ctx ctx, gs_mat mat, gs_mas mas, const double* b, int nrhs, double tol, int max_iter,
                       double inner_tol, double* x, int32_t* iters_out, double* rel_out, int32_t* outer_out) {
  using namespace mixed;
  cudaStream_t st = ctx->stream;
  const int32_t n = mat->n;
  const int64_t len64 = 3LL * n;
  GS_TRY(ensure_row_order(ctx, mat));
  float* au32 = nullptr;
  std::vector<float*> inv;
  GS_TRY(ensure_f32(ctx, mat, mas, &au32, inv));
  // buffers: FP64 r (RHS-major); FP32 interleaved rin, z, p, Ap, d; coarse vectors
  const size_t v32 = (((size_t)n * R * 3 * 4 + 255) / 256) * 256 / 4;  // floats, 256-byte aligned
  const size_t coarse = (((size_t)std::max<int64_t>(mas->vec_items, 1) * R * 3 * 4 + 255) / 256) * 256 / 4;
  const size_t r64_bytes = (((size_t)nrhs * len64 * 8 + 255) / 256) * 256;
  char* buf = nullptr;
  const size_t bytes = r64_bytes + 5 * v32 * 4 + 2 * coarse * 4 + 256;
  GS_TRY(ctx->scratch_buf(kSlotPcgVectors, bytes, (void**)&buf));
  double* r64 = (double*)buf;
  float* rin = (float*)(buf + r64_bytes);
  float *z = rin + v32, *p = z + v32, *Ap = p + v32, *d = Ap + v32, *rl = d + v32, *zl = rl + coarse;
  char* sbuf = nullptr;
  GS_TRY(ctx->scratch_buf(kSlotPcgScalars, sizeof(Scalars) + kMaxBlocks * kMaxR * 8 + 512, (void**)&sbuf));
  Scalars* s = (Scalars*)sbuf;
  double* partials = (double*)(sbuf + ((sizeof(Scalars) + 255) / 256) * 256);
  GS_CUDA(cudaMemsetAsync(s, 0, sizeof(Scalars), st));
  // ||b||^2 via the outer residual kernel on x = 0 (first = true writes r = b)
  const int G = nblocks(n);
  const double tol2 = tol * tol, itol2 = inner_tol * inner_tol;
  Levels32 al{};
  al.L = mas->L;
  al.N = mas->N;
  for (int l = 0; l < mas->L; ++l) al.coarse[l] = mas->coarse[l], al.vec_off[l] = mas->vec_off[l];
  const int N = mas->N, ld = 3 * N;
  const bool bf16 = mas->precision == GS_PREC_BF16;
  const int lv0_threads = std::min(((ld * ((R + 3) / 4) + 31) / 32) * 32, 384);
  const size_t lv0_smem = (size_t)ld * R * 4;
  const int lanes32 = ctx->tune[GS_TUNE_SPMV32_LANES];
  const int spmv_grid = ceil_div((int64_t)n * lanes32, 256);
  GS_CUDA(cudaMemsetAsync(x, 0, (size_t)nrhs * len64 * 8, st));
  {
    GS_PROF(ctx, GS_K_PCG_VECTOR);
    k_outer_residual<R><<<G, kT, 0, st>>>(b, r64, rin, d, n, nrhs, s, partials, tol2, itol2, true);
  }
  // ||b||^2: the first residual is b itself (conv_out was decided against
  // bnorm2 = 0, i.e. only a zero right-hand side counts as converged)
  GS_CUDA(cudaMemcpyAsync(s->bnorm2, s->rnorm2, sizeof(double) * kMaxR, cudaMemcpyDeviceToDevice, st));
  Scalars hs;
  int outer = 0;
  auto apply = [&](const float* rr, float* zz) -> int {
    if (mas->L > 1) {
      GS_CUDA(cudaMemsetAsync(rl, 0, coarse * 4, st));
      {
        GS_PROF(ctx, GS_K_MAS_APPLY_COARSE);
        k_restrict32<R><<<ceil_div((int64_t)mas->n_domains[0] * 32, 256), 256, 0, st>>>(rr, mas->remap0,
                                                                                       mas->n_domains[0], al, rl, s);
      }
      for (int l = 1; l + 1 < mas->L; ++l) {  // levels >= 2 from the level below, in a fixed order
        GS_PROF(ctx, GS_K_MAS_APPLY_COARSE);
        k_restrict_up<float, LevelIdxNodeMajor><<<ceil_div((int64_t)mas->n_domains[l] * 32, 128), 128, 0, st>>>(
            mas->up[l], mas->n_domains[l], N, 3 * R, LevelIdxNodeMajor{mas->vec_off[l], 3 * R},
            LevelIdxNodeMajor{mas->vec_off[l + 1], 3 * R}, rl, &s->all_out);
      }
      {
        GS_PROF(ctx, GS_K_MAS_APPLY_COARSE);
        const int64_t outs = (int64_t)mas->n_coarse_jobs * ld * R;
        k_coarse32<R, float><<<ceil_div(outs, 256), 256, 0, st>>>((const float* const*)mas->d_inv32_tab,
                                                                  mas->d_coarse_jobs,
                                                                  mas->d_coarse_jobs + mas->n_coarse_jobs,
                                                                  mas->n_coarse_jobs, N, al, rl, zl, s);
      }
    }
    if (bf16) {
      GS_PROF(ctx, GS_K_MAS_APPLY_L0);
      GS_TRY(level0_bf16_launch(ctx, mas, true, R, rr, 0, zl, 0, zz, &s->all_out, &s->flags));
    } else {
      GS_PROF(ctx, GS_K_MAS_APPLY_L0);
      k_level0_32<R, float><<<mas->n_domains[0], lv0_threads, lv0_smem, st>>>(inv[0], mas->remap0, N, al, rr, zl,
                                                                              zz, s);
    }
    return GS_OK;
  };
  auto reliable_update = [&]() -> int {
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_outer_update<R><<<G, kT, 0, st>>>(x, d, n, nrhs, s); }
    GS_TRY(spmv_launch(ctx, mat, x, r64, nrhs, GS_SPMV_ROW));
    {
      GS_PROF(ctx, GS_K_PCG_VECTOR);
      k_outer_residual<R><<<G, kT, 0, st>>>(b, r64, rin, d, n, nrhs, s, partials, tol2, itol2, false);
    }
    ++outer;
    return GS_OK;
  };
  int* hflags = ctx->h_pinned + 128;  // any_want, all_out (adjacent in Scalars)
  auto poll_flags = [&]() -> int {
    GS_CUDA(cudaMemcpyAsync(hflags, &s->any_want, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
  };
  GS_TRY(poll_flags());
  if (!hflags[1]) {
    GS_TRY(apply(rin, z));
    { GS_PROF(ctx, GS_K_PCG_VECTOR); k_in_dot<R, true><<<G, kT, 0, st>>>(rin, z, p, n, nrhs, s, partials, kInRz0); }
    const int poll = 8;
    int it = 0;
    while (it < max_iter) {
      {
        GS_PROF(ctx, GS_K_SPMV);
        if (lanes32 == 4)
          k_spmv32<R, 4><<<spmv_grid, 256, 0, st>>>(mat->row_order, mat->row_ptr, mat->cid, mat->lo_ptr,
                                                    mat->lo_idx, mat->lo_col, au32, n, p, Ap, s);
        else
          k_spmv32<R, 2><<<spmv_grid, 256, 0, st>>>(mat->row_order, mat->row_ptr, mat->cid, mat->lo_ptr,
                                                    mat->lo_idx, mat->lo_col, au32, n, p, Ap, s);
      }
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_in_dot<R, false><<<G, kT, 0, st>>>(p, Ap, nullptr, n, nrhs, s, partials, kInPAp); }
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_in_update_dr<R><<<G, kT, 0, st>>>(d, rin, p, Ap, n, nrhs, s, partials); }
      ++it;
      if (it % poll == 0 || it == max_iter) {
        GS_TRY(poll_flags());
        if (hflags[0] || it == max_iter) {
          GS_TRY(reliable_update());
          GS_TRY(poll_flags());
        }
        if (hflags[1]) break;
      }
      if (it == max_iter) break;
      GS_TRY(apply(rin, z));
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_in_dot<R, false><<<G, kT, 0, st>>>(rin, z, nullptr, n, nrhs, s, partials, kInRz); }
      { GS_PROF(ctx, GS_K_PCG_VECTOR); k_in_update_p<R><<<G, kT, 0, st>>>(p, z, n, s); }
    }
  }
  GS_CUDA(cudaMemcpyAsync(&hs, s, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  GS_CUDA(cudaGetLastError());
  bool all = true;
  for (int k = 0; k < nrhs; ++k) {
    if (iters_out) iters_out[k] = hs.iters[k];
    if (rel_out) rel_out[k] = hs.bnorm2[k] > 0 ? std::sqrt(hs.rnorm2[k] / hs.bnorm2[k]) : 0.0;
    all = all && hs.conv_out[k];
  }
  if (outer_out) *outer_out = outer;
  int flags = 0;
  GS_TRY(ctx->take_flags(&flags));
  if (hs.flags) return status_from_flags(hs.flags);
  if (flags) return status_from_flags(flags);
  if (!all) {
    set_error("gs_pcg_solve_mixed: not converged within %d inner iterations", max_iter);
    return GS_ERR_MAXITER;
  }
  return GS_OK;
}

}  // namespace gs

extern "C" int gs_pcg_solve_mixed(gs_ctx ctx, gs_mat mat, gs_mas mas, const double* b, int32_t nrhs, double tol,
                                  int32_t max_iter, double inner_tol, double* x, int32_t* iters, double* rel_res,
                                  int32_t* outer_iters) {
  GS_CHECK(ctx && mat && mas && b && x && b != x, GS_ERR_INVALID, "gs_pcg_solve_mixed: null or aliased argument");
  GS_CHECK(nrhs >= 1 && nrhs <= gs::mixed::kMaxR, GS_ERR_INVALID, "gs_pcg_solve_mixed: nrhs %d (1..8)", nrhs);
  GS_CHECK(mas->n == mat->n, GS_ERR_INVALID, "gs_pcg_solve_mixed: preconditioner built for another size");
  GS_CHECK(tol >= 0.0 && max_iter >= 0 && inner_tol > 0.0 && inner_tol < 1.0, GS_ERR_INVALID,
           "gs_pcg_solve_mixed: tol %g max_iter %d inner_tol %g", tol, max_iter, inner_tol);
  GS_CHECK(3 * mas->N * ((std::min(nrhs, 8) + 3) / 4) <= 384, GS_ERR_UNSUPPORTED, "gs_pcg_solve_mixed: domain size");
  GS_CUDA(cudaSetDevice(ctx->device));
  if (nrhs == 1) return gs::solve_mixed<1>(ctx, mat, mas, b, nrhs, tol, max_iter, inner_tol, x, iters, rel_res, outer_iters);
  if (nrhs == 2) return gs::solve_mixed<2>(ctx, mat, mas, b, nrhs, tol, max_iter, inner_tol, x, iters, rel_res, outer_iters);
  if (nrhs <= 4) return gs::solve_mixed<4>(ctx, mat, mas, b, nrhs, tol, max_iter, inner_tol, x, iters, rel_res, outer_iters);
  return gs::solve_mixed<8>(ctx, mat, mas, b, nrhs, tol, max_iter, inner_tol, x, iters, rel_res, outer_iters);
}
