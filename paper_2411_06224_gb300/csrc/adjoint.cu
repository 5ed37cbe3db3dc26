// Adjoint of the linear solve x = A^{-1} b (this library's differentiation
// form; the paper does not differentiate through the solve).
//
// For a loss L(x) with g = dL/dx (one column per right-hand side):
//   lambda = A^{-1} g                      a second MAS-PCG solve (A is SPD,
//                                          so the same preconditioner serves);
//   dL/db  = lambda;
//   dL/dA  = -lambda x^T, restricted to the stored parameters: a stored
//            off-diagonal block H = A_rc also sits transposed at (c, r), so
//            dL/dH = -sum_k (lambda_r x_c^T + x_r lambda_c^T); a stored
//            diagonal block appears once: dL/dH = -sum_k lambda_r x_r^T;
//   dL/d(input block i) = dL/dH of the stored block that input was summed
//            into (assembly is a sum), 0 for inputs below the diagonal.
#include "common.cuh"

namespace gs {

// One thread per stored block; sums over the right-hand sides.
__global__ void k_outer_grad(const int32_t* __restrict__ rid, const int32_t* __restrict__ cid, int64_t nnzb,
                             const double* __restrict__ x, const double* __restrict__ lam, int64_t stride, int nrhs,
                             double* __restrict__ dH) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nnzb) return;
  const int32_t r = rid[u], c = cid[u];
  double G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < nrhs; ++k) {
    const double* xk = x + k * stride;
    const double* lk = lam + k * stride;
    const double lr[3] = {lk[3 * r], lk[3 * r + 1], lk[3 * r + 2]};
    const double xc[3] = {xk[3 * c], xk[3 * c + 1], xk[3 * c + 2]};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bq = 0; bq < 3; ++bq) G[3 * a + bq] = fma(lr[a], xc[bq], G[3 * a + bq]);
    if (r != c) {
      const double xr[3] = {xk[3 * r], xk[3 * r + 1], xk[3 * r + 2]};
      const double lc[3] = {lk[3 * c], lk[3 * c + 1], lk[3 * c + 2]};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bq = 0; bq < 3; ++bq) G[3 * a + bq] = fma(xr[a], lc[bq], G[3 * a + bq]);
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) dH[u * 9 + q] = -G[q];
}

__global__ void k_input_grad(const int32_t* __restrict__ key_of_input, int64_t nb, const double* __restrict__ dH,
                             double* __restrict__ dIn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const int32_t k = key_of_input[i];
#pragma unroll
  for (int q = 0; q < 9; ++q) dIn[i * 9 + q] = k >= 0 ? dH[(int64_t)k * 9 + q] : 0.0;
}

}  // namespace gs

extern "C" int gs_adjoint(gs_ctx ctx, gs_mat mat, gs_mas mas, const double* x, const double* g, int32_t nrhs,
                          double tol, int32_t max_iter, int32_t mixed, double* lam, double* dLdH, double* dLdinput,
                          int32_t* iters) {
  GS_CHECK(ctx && mat && mas && x && g && lam, GS_ERR_INVALID, "gs_adjoint: null argument");
  GS_CHECK(lam != g && lam != x, GS_ERR_INVALID, "gs_adjoint: lambda aliases an input");
  GS_CHECK(nrhs >= 1, GS_ERR_INVALID, "gs_adjoint: nrhs %d", nrhs);
  GS_CHECK(!dLdinput || mat->key_of_input, GS_ERR_INVALID, "gs_adjoint: matrix has no input map");
  GS_CUDA(cudaSetDevice(ctx->device));
  int s = mixed ? gs_pcg_solve_mixed(ctx, mat, mas, g, nrhs, tol, max_iter, 1e-3, lam, iters, nullptr, nullptr)
                : gs_pcg_solve(ctx, mat, mas, g, nrhs, tol, max_iter, GS_SPMV_ROW, lam, iters, nullptr);
  if (s != GS_OK) return s;
  cudaStream_t st = ctx->stream;
  if (dLdH && mat->nnzb > 0) {
    GS_PROF(ctx, GS_K_OTHER);
    gs::k_outer_grad<<<gs::ceil_div(mat->nnzb, 256), 256, 0, st>>>(mat->rid, mat->cid, mat->nnzb, x, lam,
                                                                    3LL * mat->n, nrhs, dLdH);
  }
  if (dLdinput && mat->n_input > 0) {
    GS_CHECK(dLdH, GS_ERR_INVALID, "gs_adjoint: dLdinput needs dLdH");
    GS_PROF(ctx, GS_K_OTHER);
    gs::k_input_grad<<<gs::ceil_div(mat->n_input, 256), 256, 0, st>>>(mat->key_of_input, mat->n_input, dLdH,
                                                                        dLdinput);
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}
