// Element Hessians of a stiff-cloth sheet on the device, emitted as
// (row, col, 3x3) triplets for the hash assembly: the membrane with the
// cubic strain-limiting energy of Sec. 4 (its analytic PSD Hessian,
// Eq. Stretch_Hessian), Baraff-Witkin stretching (the negative eigenvalue of
// its Hessian clamped), Gauss-Newton shearing, Gauss-Newton hinge bending
// and lumped masses; the system is scaled as K + M / dt^2.
//
// Per triangle (vertices 0, 1, 2): F = sum_a x_a w_a^T (3 x 2, w from the
// in-plane rest edge matrix, evaluated from the edges), and per direction d with f = F e_d, s = |f|,
// P = f f^T / s^2, the 3 x 3 F-Hessian block
//   2 lam (max(1 - 1/s, 0) I + (1 - max(1 - 1/s, 0)) P)
//   + [s > 1] 3 E ((1 - 1/s)(s - 1) I + (s^2 - 1) / s^3 f f^T),
// plus the shear term 2 (0.3 lam) g g^T with g = [f_1; f_0], all times the
// rest area times the thickness.  Vertex block (a, b) = sum_{i,j} w_a[i]
// w_b[j] H_ij.  Per hinge (e_0, e_1, o_1, o_2): the dihedral-angle gradient in
// closed form (q_i = n_i / |n_i|^2, n_1 = e x (o_1 - e_0), n_2 = (o_2 - e_0)
// x e) and the blocks 2 k_b g_a g_b^T, k_b = E t^3 / 12 |e_rest|^2 / (A_1 + A_2).
//
// Emission order: 6 blocks per triangle (pairs (0,0) (0,1) (0,2) (1,1) (1,2)
// (2,2)), 10 per hinge (pairs a <= b of (e_0, e_1, o_1, o_2)), each at (min,
// max) of its two vertices, transposed when the first is the larger; then
// one m_v / dt^2 I block per vertex, m_v summed over the vertex's triangle
// corners in ascending order (rho t A / 3 each).
#include <algorithm>
#include <vector>

#include "common.cuh"

struct gs_cloth_s {
  int32_t V = 0;
  int64_t T = 0, H = 0;
  int32_t* tris = nullptr;    // 3 T
  int32_t* hinges = nullptr;  // 4 H
  double* w = nullptr;        // 6 T: w_a[j] at [6 t + 2 a + j]
  double* at = nullptr;       // T: rest area times thickness
  double* kb = nullptr;       // H: bending stiffness
  double* mdt = nullptr;      // V: m_v / dt^2
  double E = 0, lam = 0;
  gs_ctx owner = nullptr;
};

namespace gs {
namespace cloth {

constexpr double kShear = 0.3;  // shear stiffness relative to lam
constexpr int kMemThreads = 64;  // membrane kernel block: 27 KB of staged blocks
constexpr int kBendThreads = 128;
constexpr int kBendStage = 25;  // doubles staged per hinge (24 used; odd stride)

// Rest data per triangle: w and a_t; flags a repeated or out-of-range vertex
// and a degenerate rest triangle.
__global__ void k_cloth_rest(const double* __restrict__ X, const int32_t* __restrict__ tris, int64_t T, int32_t V,
                             double thickness, double* __restrict__ w, double* __restrict__ at,
                             int* __restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int32_t a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
  if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V || a == b || b == c || a == c) {
    atomicOr(flags, kErrIndex);
    for (int k = 0; k < 6; ++k) w[6 * t + k] = 0.0;
    at[t] = 0.0;
    return;
  }
  // Dm columns: X_b - X_a, X_c - X_a (in-plane coordinates)
  const double d00 = X[3 * b] - X[3 * a], d10 = X[3 * b + 1] - X[3 * a + 1];
  const double d01 = X[3 * c] - X[3 * a], d11 = X[3 * c + 1] - X[3 * a + 1];
  const double det = d00 * d11 - d01 * d10;
  if (!(fabs(det) > 0.0) || !isfinite(det)) {
    atomicOr(flags, kErrNonFinite);
    for (int k = 0; k < 6; ++k) w[6 * t + k] = 0.0;
    at[t] = 0.0;
    return;
  }
  // B = Dm^-1; w_1 = row 0 of B, w_2 = row 1, w_0 = -(w_1 + w_2)
  const double b00 = d11 / det, b01 = -d01 / det, b10 = -d10 / det, b11 = d00 / det;
  w[6 * t + 2] = b00;
  w[6 * t + 3] = b01;
  w[6 * t + 4] = b10;
  w[6 * t + 5] = b11;
  w[6 * t + 0] = -(b00 + b10);
  w[6 * t + 1] = -(b01 + b11);
  at[t] = 0.5 * fabs(det) * thickness;
}

// k_b per hinge from the rest positions; flags bad indices.
__global__ void k_hinge_rest(const double* __restrict__ X, const int32_t* __restrict__ hg, int64_t H, int32_t V,
                             double coef, double* __restrict__ kb, int* __restrict__ flags) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  int32_t v[4];
  for (int k = 0; k < 4; ++k) {
    v[k] = hg[4 * h + k];
    if (v[k] < 0 || v[k] >= V) {
      atomicOr(flags, kErrIndex);
      kb[h] = 0.0;
      return;
    }
  }
  double e[3], p1[3], p2[3];
  for (int k = 0; k < 3; ++k) {
    e[k] = X[3 * v[1] + k] - X[3 * v[0] + k];
    p1[k] = X[3 * v[2] + k] - X[3 * v[0] + k];
    p2[k] = X[3 * v[3] + k] - X[3 * v[0] + k];
  }
  auto cross_norm = [](const double* u, const double* q) {
    const double c0 = u[1] * q[2] - u[2] * q[1], c1 = u[2] * q[0] - u[0] * q[2], c2 = u[0] * q[1] - u[1] * q[0];
    return sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  };
  const double a12 = 0.5 * cross_norm(e, p1) + 0.5 * cross_norm(e, p2);
  if (!(a12 > 0.0)) {
    atomicOr(flags, kErrNonFinite);
    kb[h] = 0.0;
    return;
  }
  kb[h] = coef * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) / a12;
}

// m_v / dt^2 from the vertex's triangle corners in ascending order.
__global__ void k_cloth_mass(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_tri,
                             const double* __restrict__ at, double rho_3, double inv_dt2, int32_t V,
                             double* __restrict__ mdt) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  double m = 0.0;  // at = A t, so rho t A / 3 = (rho / 3) at
  for (int32_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) m += rho_3 * at[inc_tri[k]];
  mdt[v] = m * inv_dt2;
}

// One 3x3 block at (min, max) of vertices (va, vb): B (row-major) or its
// transpose when va > vb.
__device__ __forceinline__ void emit(int64_t k, int32_t va, int32_t vb, const double (&B)[9], int32_t* __restrict__ rows,
                                     int32_t* __restrict__ cols, double* __restrict__ out) {
  const bool sw = va > vb;
  if (rows) rows[k] = sw ? vb : va;
  if (cols) cols[k] = sw ? va : vb;
  double* o = out + 9 * k;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) o[3 * x + y] = sw ? B[3 * y + x] : B[3 * x + y];
}

// Membrane blocks: one thread per triangle, 6 blocks at 6 t.  The owner
// thread forms its 6 blocks and stages them, already in emission layout, for
// the warp's coalesced write.  The kernel is bound by the FP64 pipe, not by
// its bytes, so the F-Hessian is kept in its structured form (symmetric
// direction blocks, the shear cross block) and scaled by a_t through its
// coefficients.
__global__ void __launch_bounds__(kMemThreads) k_cloth_membrane(const double* __restrict__ x, const int32_t* __restrict__ tris,
                                                        const double* __restrict__ w, const double* __restrict__ at,
                                                        int64_t T, double E, double lam, int32_t* __restrict__ rows,
                                                        int32_t* __restrict__ cols, double* __restrict__ out) {
  // per warp: the lanes' triangles' blocks back to back (54 doubles each) and
  // their vertices; the warp then writes them as one contiguous run,
  // consecutive lanes on consecutive doubles (a thread writing its own
  // 432-byte run left the stores uncoalesced)
  __shared__ double st[kMemThreads / 32][32 * 54];
  __shared__ int32_t sv[kMemThreads / 32][32][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t0 = t - lane;  // the warp's first triangle
  if (t0 >= T) return;          // whole warps only: the lanes below meet at __syncwarp
  const bool valid = t < T;
  const int64_t tc = valid ? t : t0;  // an idle lane computes its warp's first triangle again, unused
  const int32_t v[3] = {tris[3 * tc], tris[3 * tc + 1], tris[3 * tc + 2]};
  const double w10 = w[6 * tc + 2], w11 = w[6 * tc + 3], w20 = w[6 * tc + 4], w21 = w[6 * tc + 5];
  // F = (x_1 - x_0) w_1^T + (x_2 - x_0) w_2^T (w_0 = -(w_1 + w_2)): no
  // cancellation of absolute coordinates against the 1/h-sized weights
  double F[3][2];  // F[x][j]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double x0 = x[3 * (int64_t)v[0] + c];
    const double e1 = x[3 * (int64_t)v[1] + c] - x0, e2 = x[3 * (int64_t)v[2] + c] - x0;
    F[c][0] = e1 * w10 + e2 * w20;
    F[c][1] = e1 * w11 + e2 * w21;
  }
  const double s_at = at[tc];
  // the F-Hessian times a_t: symmetric direction blocks H_00, H_11 (upper
  // triangles, index u(p, q)) and the shear cross block H_01 = mu2 f_1 f_0^T
  constexpr int kU[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  const double mu2 = 2.0 * kShear * lam * s_at;
  double Hd[2][6];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const double f[3] = {F[0][d], F[1][d], F[2][d]};
    const double s2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
    const double is = rsqrt(s2), is2 = is * is, s = s2 * is;
    const double across = fmax(1.0 - is, 0.0);
    double ci = 2.0 * lam * across;                // coefficient of I
    double cf = 2.0 * lam * (1.0 - across) * is2;  // coefficient of f f^T
    if (s > 1.0) {                                 // strain limit, Sec. 4
      ci += 3.0 * E * (1.0 - is) * (s - 1.0);
      cf += 3.0 * E * (s2 - 1.0) * is2 * is;
    }
    ci *= s_at;
    cf *= s_at;
    const double g[3] = {F[0][1 - d], F[1][1 - d], F[2][1 - d]};  // shear: g = [f_1; f_0]
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const double cfp = cf * f[p], mgp = mu2 * g[p];
#pragma unroll
      for (int q = p; q < 3; ++q) Hd[d][kU[p][q]] = fma(cfp, f[q], fma(mgp, g[q], p == q ? ci : 0.0));
    }
  }
  double H01[3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const double mgp = mu2 * F[p][1];
#pragma unroll
    for (int q = 0; q < 3; ++q) H01[p][q] = mgp * F[q][0];
  }
  // block (a, b) = sum_{i,j} w_a[i] w_b[j] H_ij (H_10 = H_01^T), each block
  // from its own weights: forming some blocks from the others through
  // w_0 = -(w_1 + w_2) cancels when the two directions' stiffnesses differ
  // by orders of magnitude (the strain limit against the stretching)
  double* my = st[warp] + 54 * lane;
  double hx[6];  // H_01 + H_01^T, upper triangle
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = p; q < 3; ++q) hx[kU[p][q]] = H01[p][q] + H01[q][p];
  auto diag = [&](int k, double wa0, double wa1) {  // symmetric (a, a)
    const double c00 = wa0 * wa0, c11 = wa1 * wa1, c01 = wa0 * wa1;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = p; q < 3; ++q)
        my[9 * k + 3 * p + q] = my[9 * k + 3 * q + p] =
            fma(c00, Hd[0][kU[p][q]], fma(c11, Hd[1][kU[p][q]], c01 * hx[kU[p][q]]));
  };
  // (a, b), a < b, stored transposed when v_a > v_b
  auto off = [&](int k, double wa0, double wa1, double wb0, double wb1, bool sw) {
    const double c00 = wa0 * wb0, c11 = wa1 * wb1, c01 = wa0 * wb1, c10 = wa1 * wb0;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double bpq =
            fma(c00, Hd[0][kU[p][q]], fma(c11, Hd[1][kU[p][q]], fma(c01, H01[p][q], c10 * H01[q][p])));
        my[9 * k + (sw ? 3 * q + p : 3 * p + q)] = bpq;
      }
  };
  const double w00 = w[6 * tc], w01 = w[6 * tc + 1];
  diag(0, w00, w01);
  off(1, w00, w01, w10, w11, v[0] > v[1]);
  off(2, w00, w01, w20, w21, v[0] > v[2]);
  diag(3, w10, w11);
  off(4, w10, w11, w20, w21, v[1] > v[2]);
  diag(5, w20, w21);
#pragma unroll
  for (int a = 0; a < 3; ++a) sv[warp][lane][a] = v[a];
  __syncwarp();
  const int nv = (int)(T - t0 < 32 ? T - t0 : 32);
  for (int i = lane; i < 54 * nv; i += 32) out[54 * t0 + i] = st[warp][i];
  for (int j = lane; j < 6 * nv; j += 32) {
    const int tri = j / 6, k = j - 6 * tri;
    const int a = k < 3 ? 0 : (k < 5 ? 1 : 2), b = k < 3 ? k : (k < 5 ? k - 2 : 2);
    const int32_t va = sv[warp][tri][a], vb = sv[warp][tri][b];
    if (rows) rows[6 * t0 + j] = min(va, vb);
    if (cols) cols[6 * t0 + j] = max(va, vb);
  }
}

// Bending blocks: one thread per hinge, 10 blocks at base + 10 h.
__global__ void __launch_bounds__(kBendThreads) k_cloth_bending(const double* __restrict__ x, const int32_t* __restrict__ hg,
                                                       const double* __restrict__ kb, int64_t H, int64_t base,
                                                       int32_t* __restrict__ rows, int32_t* __restrict__ cols,
                                                       double* __restrict__ out) {
  // per warp: each lane's hinge gradient g and 2 k_b g and its vertices,
  // then the warp writes its hinges' blocks as one contiguous run (see the
  // membrane kernel); an entry costs one DMUL
  __shared__ double sg[kBendThreads / 32][32][kBendStage];
  __shared__ int32_t sv[kBendThreads / 32][32][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t hh = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t h0 = hh - lane;
  if (h0 >= H) return;  // whole warps only
  const int64_t h = hh < H ? hh : h0;
  int32_t v[4];
  double P[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    v[a] = hg[4 * h + a];
#pragma unroll
    for (int c = 0; c < 3; ++c) P[a][c] = x[3 * (int64_t)v[a] + c];
  }
  double e[3], u1[3], u2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) e[c] = P[1][c] - P[0][c], u1[c] = P[2][c] - P[0][c], u2[c] = P[3][c] - P[0][c];
  // n_1 = e x u1, n_2 = u2 x e
  const double n1[3] = {e[1] * u1[2] - e[2] * u1[1], e[2] * u1[0] - e[0] * u1[2], e[0] * u1[1] - e[1] * u1[0]};
  const double n2[3] = {u2[1] * e[2] - u2[2] * e[1], u2[2] * e[0] - u2[0] * e[2], u2[0] * e[1] - u2[1] * e[0]};
  // one reciprocal square root and one division (each expands into several
  // FP64-pipe instructions): 1/|e| and 1/(|n_1|^2 |n_2|^2)
  const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  const double ile = rsqrt(ee), le = ee * ile;
  const double m1 = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
  const double m2 = n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2];
  const double im = 1.0 / (m1 * m2);
  const double r1 = m2 * im, r2 = m1 * im;  // 1 / |n_i|^2
  // projections onto e / |e|: (o_i - e_1) . e = u_i . e - |e|^2, (o_i - e_0) . e = u_i . e
  const double p1 = (u1[0] * e[0] + u1[1] * e[1] + u1[2] * e[2]) * ile;
  const double p2 = (u2[0] * e[0] + u2[1] * e[1] + u2[2] * e[2]) * ile;
  const double a1 = -(p1 - le) * r1, a2 = -(p2 - le) * r2;  // d theta / d e_0 = a1 n1 + a2 n2
  const double b1 = p1 * r1, b2 = p2 * r2;                  // d theta / d e_1 = b1 n1 + b2 n2
  double g[4][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g[0][c] = a1 * n1[c] + a2 * n2[c];
    g[1][c] = b1 * n1[c] + b2 * n2[c];
    g[2][c] = -le * r1 * n1[c];
    g[3][c] = -le * r2 * n2[c];
  }
  double* my = sg[warp][lane];
  const double k2 = 2.0 * kb[h];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) my[3 * a + c] = k2 * g[a][c], my[12 + 3 * a + c] = g[a][c];
#pragma unroll
  for (int a = 0; a < 4; ++a) sv[warp][lane][a] = v[a];
  __syncwarp();
  const int nv = (int)(H - h0 < 32 ? H - h0 : 32);
  // block k of a hinge is the vertex pair (a, b), a <= b, in the order
  // (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3)
  for (int i = lane; i < 90 * nv; i += 32) {
    const int hi = i / 90, rem = i - 90 * hi, k = rem / 9, e = rem - 9 * k;
    const int a = k < 4 ? 0 : (k < 7 ? 1 : (k < 9 ? 2 : 3));
    const int b = k < 4 ? k : (k < 7 ? k - 3 : (k < 9 ? k - 5 : 3));
    const double* d = sg[warp][hi];
    int p = e / 3, q = e - 3 * (e / 3);
    if (sv[warp][hi][a] > sv[warp][hi][b]) {  // stored at (min, max): the transpose
      const int tmp = p;
      p = q;
      q = tmp;
    }
    out[9 * base + 90 * h0 + i] = d[3 * a + p] * d[12 + 3 * b + q];
  }
  for (int j = lane; j < 10 * nv; j += 32) {
    const int hi = j / 10, k = j - 10 * hi;
    const int a = k < 4 ? 0 : (k < 7 ? 1 : (k < 9 ? 2 : 3));
    const int b = k < 4 ? k : (k < 7 ? k - 3 : (k < 9 ? k - 5 : 3));
    const int32_t va = sv[warp][hi][a], vb = sv[warp][hi][b];
    if (rows) rows[base + 10 * h0 + j] = min(va, vb);
    if (cols) cols[base + 10 * h0 + j] = max(va, vb);
  }
}

// Mass blocks at base + v.
__global__ void k_cloth_mass_blocks(const double* __restrict__ mdt, int32_t V, int64_t base, int32_t* __restrict__ rows,
                                    int32_t* __restrict__ cols, double* __restrict__ out) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double m = mdt[v];
  const double B[9] = {m, 0, 0, 0, m, 0, 0, 0, m};
  emit(base + v, v, v, B, rows, cols, out);
}

}  // namespace cloth
}  // namespace gs

using namespace gs;

extern "C" {

int gs_cloth_destroy(gs_cloth c) {
  if (!c) return GS_OK;
  gs_ctx ctx = c->owner;
  ctx->release(c->tris);
  ctx->release(c->hinges);
  ctx->release(c->w);
  ctx->release(c->at);
  ctx->release(c->kb);
  ctx->release(c->mdt);
  delete c;
  return GS_OK;
}

int gs_cloth_create(gs_ctx ctx, int32_t n_vertices, const double* X, int64_t n_tris, const int32_t* tris,
                    int64_t n_hinges, const int32_t* hinges, double E, double lam, double thickness, double rho,
                    double dt, gs_cloth* out) {
  GS_CHECK(ctx && out, GS_ERR_INVALID, "gs_cloth_create: null context or output");
  *out = nullptr;
  const int32_t V = n_vertices;
  const int64_t T = n_tris, H = n_hinges;
  GS_CHECK(V > 0 && T >= 0 && H >= 0 && 6 * T + 10 * H + V < (1LL << 31), GS_ERR_INVALID,
           "gs_cloth_create: sizes V=%d T=%lld H=%lld", V, (long long)T, (long long)H);
  GS_CHECK(X && (T == 0 || tris) && (H == 0 || hinges), GS_ERR_INVALID, "gs_cloth_create: null array");
  GS_CHECK(E >= 0 && lam >= 0 && thickness > 0 && rho > 0 && dt > 0, GS_ERR_INVALID,
           "gs_cloth_create: parameters");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  gs_cloth c = new gs_cloth_s();
  c->V = V, c->T = T, c->H = H, c->E = E, c->lam = lam, c->owner = ctx;
  auto fail = [&](int s) {
    gs_cloth_destroy(c);
    return s;
  };
  int s;
  if ((s = ctx->alloc((void**)&c->tris, std::max<int64_t>(T, 1) * 12)) ||
      (s = ctx->alloc((void**)&c->hinges, std::max<int64_t>(H, 1) * 16)) ||
      (s = ctx->alloc((void**)&c->w, std::max<int64_t>(T, 1) * 48)) ||
      (s = ctx->alloc((void**)&c->at, std::max<int64_t>(T, 1) * 8)) ||
      (s = ctx->alloc((void**)&c->kb, std::max<int64_t>(H, 1) * 8)) ||
      (s = ctx->alloc((void**)&c->mdt, (size_t)V * 8)))
    return fail(s);
  if (T && cudaMemcpyAsync(c->tris, tris, T * 12, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return fail(GS_ERR_CUDA);
  if (H && cudaMemcpyAsync(c->hinges, hinges, H * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return fail(GS_ERR_CUDA);
  if (T) {
    GS_PROF(ctx, GS_K_ELEMENT);
    cloth::k_cloth_rest<<<ceil_div(T, 256), 256, 0, st>>>(X, c->tris, T, V, thickness, c->w, c->at, ctx->d_flags);
  }
  if (H) {
    GS_PROF(ctx, GS_K_ELEMENT);
    cloth::k_hinge_rest<<<ceil_div(H, 256), 256, 0, st>>>(X, c->hinges, H, V, E * thickness * thickness * thickness / 12.0,
                                                       c->kb, ctx->d_flags);
  }
  // vertex -> triangle incidence in ascending (triangle, corner) order, built
  // on the host once per mesh (a counting sort of the corners)
  std::vector<int32_t> ht(3 * T), ptr(V + 1, 0), idx(3 * T);
  if (T && cudaMemcpyAsync(ht.data(), c->tris, T * 12, cudaMemcpyDeviceToHost, st) != cudaSuccess) return fail(GS_ERR_CUDA);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(GS_ERR_CUDA);
  int flags = 0;
  if ((s = ctx->take_flags(&flags))) return fail(s);
  if (flags) {
    set_error("gs_cloth_create: %s", flags & kErrIndex ? "a vertex index out of range or repeated in a triangle"
                                                       : "a degenerate rest triangle or hinge");
    return fail(status_from_flags(flags));
  }
  for (int64_t k = 0; k < 3 * T; ++k) ++ptr[ht[k] + 1];
  for (int32_t v = 0; v < V; ++v) ptr[v + 1] += ptr[v];
  {
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t k = 0; k < 3 * T; ++k) idx[fill[ht[k]]++] = (int32_t)(k / 3);
  }
  int32_t *d_ptr = nullptr, *d_idx = nullptr;
  if ((s = ctx->alloc((void**)&d_ptr, (size_t)(V + 1) * 4)) || (s = ctx->alloc((void**)&d_idx, std::max<int64_t>(3 * T, 1) * 4)))
    return fail(s);
  if (cudaMemcpyAsync(d_ptr, ptr.data(), (size_t)(V + 1) * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (T && cudaMemcpyAsync(d_idx, idx.data(), (size_t)3 * T * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)) {
    ctx->release(d_ptr);
    ctx->release(d_idx);
    return fail(GS_ERR_CUDA);
  }
  {
    GS_PROF(ctx, GS_K_ELEMENT);
    cloth::k_cloth_mass<<<ceil_div(V, 256), 256, 0, st>>>(d_ptr, d_idx, c->at, rho / 3.0, 1.0 / (dt * dt), V, c->mdt);
  }
  const bool sync_ok = cudaStreamSynchronize(st) == cudaSuccess;  // the host vectors must outlive the copies
  ctx->release(d_ptr);
  ctx->release(d_idx);
  if (!sync_ok || cudaGetLastError() != cudaSuccess) return fail(GS_ERR_CUDA);
  *out = c;
  return GS_OK;
}

int gs_cloth_triplets(gs_ctx ctx, gs_cloth c, const double* x, int32_t* rows, int32_t* cols, double* blocks) {
  GS_CHECK(ctx && c && x && blocks, GS_ERR_INVALID, "gs_cloth_triplets: null argument");
  GS_CHECK(c->owner == ctx, GS_ERR_INVALID, "gs_cloth_triplets: cloth of another context");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  if (c->T) {
    GS_PROF(ctx, GS_K_ELEMENT);
    cloth::k_cloth_membrane<<<ceil_div(c->T, cloth::kMemThreads), cloth::kMemThreads, 0, st>>>(x, c->tris, c->w, c->at, c->T, c->E, c->lam, rows, cols,
                                                                blocks);
  }
  if (c->H) {
    GS_PROF(ctx, GS_K_ELEMENT);
    cloth::k_cloth_bending<<<ceil_div(c->H, cloth::kBendThreads), cloth::kBendThreads, 0, st>>>(x, c->hinges, c->kb, c->H, 6 * c->T, rows, cols, blocks);
  }
  {
    GS_PROF(ctx, GS_K_ELEMENT);
    cloth::k_cloth_mass_blocks<<<ceil_div(c->V, 256), 256, 0, st>>>(c->mdt, c->V, 6 * c->T + 10 * c->H, rows, cols,
                                                                    blocks);
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

int gs_cloth_info(gs_cloth c, int64_t* n_triplets) {
  GS_CHECK(c && n_triplets, GS_ERR_INVALID, "gs_cloth_info: null argument");
  *n_triplets = 6 * c->T + 10 * c->H + c->V;
  return GS_OK;
}

}  // extern "C"
