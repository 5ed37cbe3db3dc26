// Measurement only: a library SpMV on the full (both-triangle) BSR matrix,
// for comparing the paper's symmetric storage (Sec. 5.3) with full BSR.
#include <cusparse.h>

#include "common.cuh"

extern "C" int gs_micro_bsr_spmv_cusparse(gs_ctx ctx, int32_t n, int32_t nnzb, const int32_t* row_ptr,
                                          const int32_t* col_ind, const double* vals, const double* x, double* y,
                                          int32_t reps, float* ms) {
  using namespace gs;
  GS_CHECK(ctx && row_ptr && col_ind && vals && x && y && ms && n > 0 && nnzb > 0 && reps > 0, GS_ERR_INVALID,
           "gs_micro_bsr_spmv_cusparse: bad argument");
  GS_CUDA(cudaSetDevice(ctx->device));
  cusparseHandle_t h = nullptr;
  cusparseMatDescr_t d = nullptr;
  if (cusparseCreate(&h) != CUSPARSE_STATUS_SUCCESS) {
    set_error("cusparseCreate failed");
    return GS_ERR_CUDA;
  }
  int s = GS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const double one = 1.0, zero = 0.0;
  if (cusparseSetStream(h, ctx->stream) != CUSPARSE_STATUS_SUCCESS || cusparseCreateMatDescr(&d) != CUSPARSE_STATUS_SUCCESS ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("gs_micro_bsr_spmv_cusparse: setup failed");
    s = GS_ERR_CUDA;
  }
  if (s == GS_OK) {
    cusparseSetMatType(d, CUSPARSE_MATRIX_TYPE_GENERAL);
    cusparseSetMatIndexBase(d, CUSPARSE_INDEX_BASE_ZERO);
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < reps && s == GS_OK; ++r)
      if (cusparseDbsrmv(h, CUSPARSE_DIRECTION_ROW, CUSPARSE_OPERATION_NON_TRANSPOSE, n, n, nnzb, &one, d, vals,
                         row_ptr, col_ind, 3, x, &zero, y) != CUSPARSE_STATUS_SUCCESS) {
        set_error("cusparseDbsrmv failed");
        s = GS_ERR_CUDA;
      }
    cudaEventRecord(e1, ctx->stream);
    if (s == GS_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)) {
      set_error("gs_micro_bsr_spmv_cusparse: timing failed");
      s = GS_ERR_CUDA;
    }
    if (s == GS_OK) *ms /= reps;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d) cusparseDestroyMatDescr(d);
  cusparseDestroy(h);
  return s;
}
