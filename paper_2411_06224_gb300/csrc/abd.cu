// Two-level reduction for coupled FEM / affine-body Hessians (Sec. 5.1, Sec. 5.2).
//
// Level 1 reduces every 3x3 contact / element block per full-space node
// pair (r, c) with the FastHashReduction of assemble.cu.  Each unique pair
// is then mapped once through the Jacobians: with w(i) = [1, xbar_i] for a
// body node (x_i = A xbar_i + p, q = [p; a_1; a_2; a_3]) the product
// J_r^T C J_c consists of the 3x3 sub-blocks w_a(r) w_b(c) C, which are
// emitted on the reduced block rows (16 for body-body, 4 for body-FEM, 1
// for FEM-FEM: Sec. 5.2's unification), and level 2 reduces them again.
// Both orientations (r, c, C) and (c, r, C^T) of an off-diagonal pair are
// expanded so that every reduced sub-block lands in the upper triangle.
// Indices n_nodes + 4b + a name body b's own reduced block row a directly:
// a body's 12 x 12 Hessian (inertia, orthogonality potential) enters as its
// 16 sub-blocks, Sec. 5.2's ABD-ABD block type, and passes level 2 with
// weight 1.

#include "common.cuh"
#include "sort_scan.cuh"

namespace gs {

int reduce_blocks(gs_ctx ctx, int32_t n, const int32_t* rows, const int32_t* cols, const double* blocks,
                  int64_t nb, gs_mat* out);

struct AbdMap {
  const int32_t* body;
  const double* xbar;
  int32_t n_fem;
  int32_t n_bodies;
  int32_t n_nodes;
};

__device__ __forceinline__ int abd_targets(const AbdMap& m, int32_t node, int32_t* R, double* w) {
  if (node >= m.n_nodes) {  // a body's own reduced block row (its 12 x 12 Hessian's 3 x 3 sub-blocks)
    R[0] = m.n_fem + (node - m.n_nodes);
    w[0] = 1.0;
    return 1;
  }
  int32_t b = m.body[node];
  if (b < 0) {
    R[0] = node;
    w[0] = 1.0;
    return 1;
  }
  int32_t base = m.n_fem + 4 * b;
  R[0] = base;
  R[1] = base + 1;
  R[2] = base + 2;
  R[3] = base + 3;
  w[0] = 1.0;
  w[1] = m.xbar[3 * node + 0];
  w[2] = m.xbar[3 * node + 1];
  w[3] = m.xbar[3 * node + 2];
  return 4;
}

__global__ void k_abd_validate(AbdMap m, int32_t n_nodes, int* flags) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int32_t b = m.body[i];
  bool ok = (b < 0) ? (i < m.n_fem) : (b < m.n_bodies && i >= m.n_fem);
  if (!ok) atomicOr(flags, kErrIndex);
}

// mode 0: count the emitted sub-blocks of each stored pair; mode 1: emit.
template <int kMode>
__global__ void k_abd_expand(AbdMap m, const int32_t* __restrict__ rid, const int32_t* __restrict__ cid,
                             const double* __restrict__ au, int64_t U, const int32_t* __restrict__ off,
                             int32_t* __restrict__ cnt, int32_t* __restrict__ orow, int32_t* __restrict__ ocol,
                             double* __restrict__ oblk) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  int32_t r = rid[u], c = cid[u];
  double C[9];
  if (kMode == 1) {
#pragma unroll
    for (int k = 0; k < 9; ++k) C[k] = au[u * 9 + k];
  }
  int32_t Rr[4], Rc[4];
  double wr[4], wc[4];
  int nr = abd_targets(m, r, Rr, wr);
  int nc = abd_targets(m, c, Rc, wc);
  int64_t o = (kMode == 1) ? off[u] : 0;
  int count = 0;
  for (int orient = 0; orient < (r == c ? 1 : 2); ++orient) {
    const int32_t* RA = orient ? Rc : Rr;
    const int32_t* RB = orient ? Rr : Rc;
    const double* wa = orient ? wc : wr;
    const double* wb = orient ? wr : wc;
    int na = orient ? nc : nr, nbb = orient ? nr : nc;
    for (int a = 0; a < na; ++a)
      for (int b = 0; b < nbb; ++b) {
        if (RA[a] > RB[b]) continue;
        if (kMode == 1) {
          double s = wa[a] * wb[b];
          orow[o + count] = RA[a];
          ocol[o + count] = RB[b];
          double* dst = oblk + (o + count) * 9;
#pragma unroll
          for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = 0; y < 3; ++y) dst[3 * x + y] = s * (orient ? C[3 * y + x] : C[3 * x + y]);
        }
        ++count;
      }
  }
  if (kMode == 0) cnt[u] = count;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_assemble_abd(gs_ctx ctx, int32_t n_nodes, int32_t n_fem, int32_t n_bodies,
                               const int32_t* body_of_node, const double* xbar, const int32_t* rows,
                               const int32_t* cols, const double* blocks, int64_t n_blocks, gs_mat* out) {
  GS_CHECK(ctx && out, GS_ERR_INVALID, "gs_assemble_abd: null context or output");
  *out = nullptr;
  GS_CHECK(n_nodes > 0 && n_fem >= 0 && n_fem <= n_nodes && n_bodies >= 0, GS_ERR_INVALID,
           "gs_assemble_abd: bad sizes");
  GS_CHECK(body_of_node && (n_bodies == 0 || xbar), GS_ERR_INVALID, "gs_assemble_abd: null body map");
  int64_t n_red = (int64_t)n_fem + 4LL * n_bodies;
  GS_CHECK(n_red > 0 && n_red < (1 << 30), GS_ERR_INVALID, "gs_assemble_abd: reduced size out of range");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  AbdMap m{body_of_node, xbar, n_fem, n_bodies, n_nodes};
  { GS_PROF(ctx, GS_K_OTHER); k_abd_validate<<<ceil_div(n_nodes, 256), 256, 0, st>>>(m, n_nodes, ctx->d_flags); }
  int flags = 0;
  GS_TRY(ctx->take_flags(&flags));
  if (flags) return status_from_flags(flags);
  gs_mat lvl1 = nullptr;
  GS_CHECK((int64_t)n_nodes + 4LL * n_bodies < (1LL << 30), GS_ERR_INVALID, "gs_assemble_abd: too many rows");
  GS_TRY(gs_assemble(ctx, n_nodes + 4 * n_bodies, rows, cols, blocks, n_blocks, &lvl1));
  int64_t U = lvl1->nnzb;
  int32_t *cnt = nullptr, *off = nullptr, *orow = nullptr, *ocol = nullptr;
  double* oblk = nullptr;
  void* temp = nullptr;
  size_t tb = 0;
  int s = GS_OK;
  int64_t total = 0;
  if ((s = ctx->alloc((void**)&cnt, (size_t)(U + 1) * 4)) || (s = ctx->alloc((void**)&off, (size_t)(U + 1) * 4)))
    goto done;
  if (U > 0) {
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_abd_expand<0><<<ceil_div(U, 256), 256, 0, st>>>(m, lvl1->rid, lvl1->cid, lvl1->au, U, nullptr, cnt, nullptr,
                                                      nullptr, nullptr); }
  }
  cudaMemsetAsync(cnt + U, 0, 4, st);
  tb = scan_temp_bytes(U + 1);
  if ((s = ctx->alloc(&temp, tb))) goto done;
  {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    if ((s = exclusive_scan_i32(st, cnt, off, U + 1, temp, tb))) goto done;
  }
  if (cudaMemcpyAsync(ctx->h_pinned, off + U, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("gs_assemble_abd: readback failed");
    s = GS_ERR_CUDA;
    goto done;
  }
  total = ctx->h_pinned[0];
  if ((s = ctx->alloc((void**)&orow, (size_t)total * 4)) || (s = ctx->alloc((void**)&ocol, (size_t)total * 4)) ||
      (s = ctx->alloc((void**)&oblk, (size_t)total * 72)))
    goto done;
  if (U > 0) {
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_abd_expand<1><<<ceil_div(U, 256), 256, 0, st>>>(m, lvl1->rid, lvl1->cid, lvl1->au, U, off, nullptr, orow,
                                                      ocol, oblk); }
  }
  s = gs_assemble(ctx, (int32_t)n_red, orow, ocol, oblk, total, out);
done:
  ctx->release(cnt);
  ctx->release(off);
  ctx->release(temp);
  ctx->release(orow);
  ctx->release(ocol);
  ctx->release(oblk);
  gs_mat_destroy(lvl1);
  return s;
}
