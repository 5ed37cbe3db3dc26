// Elastic tet bodies on the device: the local Hessians of the implicit-Euler
// incremental potential (Sec. 3.1: elastic energy, PSD-projected element
// Hessians) emitted straight into the hash-key assembly (Sec. 5.1-5.2), the
// energy and gradient, and the Newton loop around the MAS-PCG solve
// (Fig. framework; supplement Eq. 1, T_nt = T_ga + T_pa + N_pcg T_pcg).
//
// Energy of an element (stable Neo-Hookean, Smith, de Goes and Kim 2018,
// without the log term), F the deformation gradient:
//   Psi(F) = mu/2 (|F|^2 - 3) + lam/2 (det F - alpha)^2,   alpha = 1 + mu/lam,
// mu, lam Lame parameters re-parameterised from (E, nu) as mu = 4/3 mu_L,
// lam = lam_L + 5/6 mu_L.  F = sum_a x_a w_a^T over the tet's four nodes,
// w_1..w_3 the rows of Dm^-1 (Dm the rest edge matrix) and w_0 = -(w_1 + w_2 + w_3).
//
// PSD projection by the analytic eigensystem of isotropic energies (Smith,
// de Goes and Kim 2019).  With F = U diag(s) V^T (U, V rotations, s_2 carrying
// the sign of det F) and D = U^T dF V, the F-Hessian is block diagonal in
// the entries of D: for each pair i < j (k the third index) a 2x2 block on
// (D_ij, D_ji) with the twist mode (1, -1)/sqrt2 at mu + lam (J - alpha) s_k
// and the flip mode (1, 1)/sqrt2 at mu - lam (J - alpha) s_k; and a 3x3 block
// on (D_00, D_11, D_22), mu I + lam g g^T + lam (J - alpha) S with
// g = (s1 s2, s0 s2, s0 s1) and S = [[0, s2, s1], [s2, 0, s0], [s1, s0, 0]].
// Each block's negative eigenvalues are set to zero.  The element Hessian
// follows by the chain rule in the rotated frame: with z_a = V^T w_a, block
// (a, b) is vol U Hy U^T, Hy[i][i'] = sum_{j,j'} z_a[j] z_b[j'] H_D+[(i,j),(i',j')].
// The SVD: cyclic Jacobi on F^T F gives V (sorted, det V = +1), Givens QR of
// F V gives U and the signed singular values (McAdams et al. 2011, with
// exact rotations in FP64).
//
// Assembly pattern (symbolic / numeric split).  Every element emits its ten
// upper node-pair blocks in the pair order (0,0) (0,1) (0,2) (0,3) (1,1)
// (1,2) (1,3) (2,2) (2,3) (3,3), stored at (min, max) of the two nodes
// (transposed when the first node is the larger); then every vertex its mass
// block m_v / dt^2 I.  Their keys are sorted once when the body is created;
// contact springs are sorted on their own whenever they change and merged
// into the element pattern.  Each Newton iteration then only writes values
// and reduces them through the stored order: no sort.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "common.cuh"
#include "primitives.cuh"

namespace gs {
int reduce_blocks(gs_ctx ctx, int32_t n, const int32_t* rows, const int32_t* cols, const double* blocks, int64_t nb,
                  gs_mat* out);
}  // namespace gs

struct gs_fem_s {
  gs_ctx owner = nullptr;
  int32_t V = 0;
  int64_t T = 0;
  double mu = 0, lam = 0, rho = 0, dt = 0;
  double* X = nullptr;       // V * 3 rest positions
  int32_t* tets = nullptr;   // T * 4
  double* w = nullptr;       // T * 12: w[t][a][j]
  double* vol = nullptr;     // T
  double* mass = nullptr;    // V lumped masses
  int32_t* inc_ptr = nullptr;  // V + 1: the (tet, node) entries t * 4 + a of each vertex, ascending
  int32_t* inc_idx = nullptr;  // 4T
  int shift = 0;             // key = (row << shift) | col
  int64_t n_in = 0;          // element inputs: 10 T + V
  uint32_t* e_sidx = nullptr;  // element inputs in key order
  int32_t* e_O = nullptr;      // unique element key of each sorted input
  int64_t U_e = 0;
  uint64_t* e_keys = nullptr;  // U_e unique element keys, ascending
  double* e_vals = nullptr;    // n_in * 9 input blocks (numeric scratch)
  double* forces = nullptr;    // T * 12 node forces of the elements
  double* energy = nullptr;    // T + nc + V energy terms
  // contact springs
  int64_t nc = 0;
  int32_t* c_pairs = nullptr;  // 2 nc
  double* c_K = nullptr;       // 9 nc
  double* c_rest = nullptr;    // 3 nc
  double* c_forces = nullptr;  // 6 nc
  int32_t* cinc_ptr = nullptr; // V + 1: entries 2p + s of each vertex
  int32_t* cinc_idx = nullptr; // 2 nc
  gs_mat c_mat = nullptr;      // reduced spring blocks (their own sort)
  int32_t* pos_c = nullptr;    // U_c: merged position of each spring block
  // merged pattern
  int64_t U = 0;
  int32_t* rid = nullptr;
  int32_t* cid = nullptr;
  int32_t* row_ptr = nullptr;
  int32_t* O_m = nullptr;      // n_in: merged position of each sorted element input
  uint64_t version = 0;        // changes with the merged pattern
};

namespace gs {
namespace fem {

// ------------------------------------------------------------------ 3x3 math
// One cyclic-Jacobi rotation in the (p, q) plane: A <- J^T A J, Q <- Q J.
// With th = (A_qq - A_pp) / 2 the rotation tangent is the smaller root of
// t^2 + 2 (th / A_pq) t - 1 = 0, written as sgn(th) A_pq / (|th| + hypot(th, A_pq))
// (one division, no overflow of th / A_pq); c = 1 / sqrt(1 + t^2), s = t c.
template <int p, int q>
__device__ __forceinline__ void jacobi_rotate(double (&A)[3][3], double (&Q)[3][3]) {
  constexpr int r = 3 - p - q;
  const double apq = A[p][q];
  const double th = 0.5 * (A[q][q] - A[p][p]);
  const double h = sqrt(th * th + apq * apq);
  if (apq == 0.0 || h == 0.0) return;
  const double t = (th >= 0.0 ? apq : -apq) / (fabs(th) + h);
  const double c = rsqrt(1.0 + t * t);
  const double s = t * c;
  A[p][p] -= t * apq;
  A[q][q] += t * apq;
  A[p][q] = A[q][p] = 0.0;
  const double arp = A[r][p], arq = A[r][q];
  A[r][p] = A[p][r] = c * arp - s * arq;
  A[r][q] = A[q][r] = s * arp + c * arq;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double qp = Q[i][p], qq = Q[i][q];
    Q[i][p] = c * qp - s * qq;
    Q[i][q] = s * qp + c * qq;
  }
}

// Symmetric A = Q diag(A) Q^T on return (A diagonal, Q orthogonal).
__device__ __forceinline__ void sym_eig3(double (&A)[3][3], double (&Q)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 16; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double dg = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (!(off > 1e-34 * dg)) break;  // converged (or a NaN: leave)
    jacobi_rotate<0, 1>(A, Q);
    jacobi_rotate<0, 2>(A, Q);
    jacobi_rotate<1, 2>(A, Q);
  }
}

template <int i, int j>
__device__ __forceinline__ void swap_pair(double (&A)[3][3], double (&Q)[3][3]) {
  if (A[i][i] < A[j][j]) {
    const double d = A[i][i];
    A[i][i] = A[j][j];
    A[j][j] = d;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double q = Q[r][i];
      Q[r][i] = Q[r][j];
      Q[r][j] = q;
    }
  }
}

// Rows p, q of B rotated so that B[q][p] = 0 and B[p][p] >= 0; U <- U G^T.
template <int p, int q>
__device__ __forceinline__ void givens(double (&B)[3][3], double (&U)[3][3]) {
  const double a = B[p][p], b = B[q][p];
  const double n2 = a * a + b * b;
  if (n2 == 0.0) return;
  const double inv = rsqrt(n2);
  const double c = a * inv, s = b * inv;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double bp = B[p][k], bq = B[q][k];
    B[p][k] = c * bp + s * bq;
    B[q][k] = -s * bp + c * bq;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double up = U[i][p], uq = U[i][q];
    U[i][p] = c * up + s * uq;
    U[i][q] = -s * up + c * uq;
  }
}

// F = U diag(s) V^T with U, V rotations, s0 >= s1 >= |s2| up to rounding.
__device__ __forceinline__ void svd3(const double (&F)[3][3], double (&U)[3][3], double (&s)[3],
                                     double (&V)[3][3]) {
  double A[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
  sym_eig3(A, V);
  swap_pair<0, 1>(A, V);
  swap_pair<0, 2>(A, V);
  swap_pair<1, 2>(A, V);
  const double detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                      V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                      V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (detV < 0.0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) V[i][2] = -V[i][2];
  }
  double B[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) B[i][j] = F[i][0] * V[0][j] + F[i][1] * V[1][j] + F[i][2] * V[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) U[i][j] = i == j ? 1.0 : 0.0;
  givens<0, 1>(B, U);
  givens<0, 2>(B, U);
  givens<1, 2>(B, U);
  s[0] = B[0][0];
  s[1] = B[1][1];
  s[2] = B[2][2];
}

__device__ __forceinline__ double pos(double v) { return v > 0.0 ? v : 0.0; }

// The node pair of each of an element's ten upper blocks.
__device__ __forceinline__ void pair_nodes(int p, int& a, int& b) {
  // (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3)
  a = p < 4 ? 0 : p < 7 ? 1 : p < 9 ? 2 : 3;
  const int first = a == 0 ? 0 : a == 1 ? 4 : a == 2 ? 7 : 9;
  b = a + (p - first);
}

__device__ __forceinline__ void load_F(const double* __restrict__ x, const int32_t (&v)[4],
                                       const double (&w)[4][3], double (&F)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[i][j] = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double xa[3] = {x[3 * (int64_t)v[a]], x[3 * (int64_t)v[a] + 1], x[3 * (int64_t)v[a] + 2]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = fma(xa[i], w[a][j], F[i][j]);
  }
}

// ------------------------------------------------------------------ kernels
// Rest shape: w (rows of Dm^-1, w_0 = -sum) and volume |det Dm| / 6.
__global__ void k_rest(const double* __restrict__ X, const int32_t* __restrict__ tets, int64_t T, int32_t V,
                       double* __restrict__ w, double* __restrict__ vol, int* flags) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  int32_t v[4];
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    v[a] = tets[4 * t + a];
    if (v[a] < 0 || v[a] >= V) bad = true;
  }
  if (bad || v[0] == v[1] || v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3] || v[2] == v[3]) {
    atomicOr(flags, kErrIndex);
    return;
  }
  double D[3][3];  // columns: X_a - X_0
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) D[i][a - 1] = X[3 * (int64_t)v[a] + i] - X[3 * (int64_t)v[0] + i];
  const double c00 = D[1][1] * D[2][2] - D[1][2] * D[2][1];
  const double c01 = D[1][2] * D[2][0] - D[1][0] * D[2][2];
  const double c02 = D[1][0] * D[2][1] - D[1][1] * D[2][0];
  const double det = D[0][0] * c00 + D[0][1] * c01 + D[0][2] * c02;
  if (!(fabs(det) > 0.0) || !isfinite(det)) {
    atomicOr(flags, kErrNonFinite);
    return;
  }
  // B = Dm^-1 = adj(Dm) / det; B[r][i] = cofactor(i, r) / det
  double B[3][3];
  B[0][0] = c00 / det;
  B[1][0] = c01 / det;
  B[2][0] = c02 / det;
  B[0][1] = (D[0][2] * D[2][1] - D[0][1] * D[2][2]) / det;
  B[1][1] = (D[0][0] * D[2][2] - D[0][2] * D[2][0]) / det;
  B[2][1] = (D[0][1] * D[2][0] - D[0][0] * D[2][1]) / det;
  B[0][2] = (D[0][1] * D[1][2] - D[0][2] * D[1][1]) / det;
  B[1][2] = (D[0][2] * D[1][0] - D[0][0] * D[1][2]) / det;
  B[2][2] = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) / det;
  double* wt = w + 12 * t;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    wt[j] = -(B[0][j] + B[1][j] + B[2][j]);
#pragma unroll
    for (int a = 1; a < 4; ++a) wt[3 * a + j] = B[a - 1][j];
  }
  vol[t] = fabs(det) / 6.0;
}

__global__ void k_iota(uint32_t* __restrict__ a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (uint32_t)i;
}

// ptr[v] = first sorted entry with key >= v, ptr[V] = n (keys ascending, 0..V-1).
__global__ void k_seg_ptr(const uint32_t* __restrict__ skey, int64_t n, int32_t V, int32_t* __restrict__ ptr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int32_t here = i < n ? (int32_t)skey[i] : V;
  const int32_t prev = i > 0 ? (int32_t)skey[i - 1] : -1;
  for (int32_t v = prev + 1; v <= here; ++v) ptr[v] = (int32_t)i;
}

// m_v = sum over the vertex's (tet, node) entries, ascending, of rho vol / 4.
__global__ void k_mass(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_idx,
                       const double* __restrict__ vol, double rho, int32_t V, double* __restrict__ mass) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  double m = 0.0;
  for (int32_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) m += rho * vol[inc_idx[k] >> 2] / 4.0;
  mass[v] = m;
}

// Keys of the element inputs: ten pair blocks per tet, then one mass block per vertex.
__global__ void k_element_keys(const int32_t* __restrict__ tets, int64_t T, int32_t V, int shift,
                               uint64_t* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 10 * T + V) return;
  uint64_t r, c;
  if (i < 10 * T) {
    const int64_t t = i / 10;
    int a, b;
    pair_nodes((int)(i - 10 * t), a, b);
    const uint32_t va = (uint32_t)tets[4 * t + a], vb = (uint32_t)tets[4 * t + b];
    r = va < vb ? va : vb;
    c = va < vb ? vb : va;
  } else {
    r = c = (uint64_t)(i - 10 * T);
  }
  keys[i] = (r << shift) | c;
}

// P[i] = K[i] != K[i+1] (1 at the end of every run).
__global__ void k_run_ends(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ P) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) P[i] = (i + 1 == n) ? 1 : (keys[i] != keys[i + 1]);
}

__global__ void k_unique_keys(const uint64_t* __restrict__ skeys, const int32_t* __restrict__ O, int64_t n,
                              uint64_t* __restrict__ ukeys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (i == 0 || O[i] != O[i - 1])) ukeys[O[i]] = skeys[i];
}

// Element Hessians: per tet, its ten projected 3x3 blocks (the pair order
// above), transposed where the first node is the larger.
__global__ void __launch_bounds__(128) k_element_hessians(const double* __restrict__ x,
                                                          const int32_t* __restrict__ tets,
                                                          const double* __restrict__ w,
                                                          const double* __restrict__ vol, int64_t T, double mu,
                                                          double lam, double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  int32_t v[4];
  double wl[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    v[a] = tets[4 * t + a];
#pragma unroll
    for (int j = 0; j < 3; ++j) wl[a][j] = w[12 * t + 3 * a + j];
  }
  double F[3][3];
  load_F(x, v, wl, F);
  double U[3][3], s[3], Vm[3][3];
  svd3(F, U, s, Vm);
  const double alpha = 1.0 + mu / lam;
  const double J = s[0] * s[1] * s[2];
  const double c1 = lam * (J - alpha);
  // 3x3 block on the diagonal entries of D, projected
  const double g[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
  double As[3][3], Es[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) As[i][j] = lam * g[i] * g[j] + (i == j ? mu : c1 * s[3 - i - j]);
  sym_eig3(As, Es);
  double Ps[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Ps[i][j] = pos(As[0][0]) * Es[i][0] * Es[j][0] + pos(As[1][1]) * Es[i][1] * Es[j][1] +
                 pos(As[2][2]) * Es[i][2] * Es[j][2];
  // 2x2 blocks: pair (i, j) = (1, 2), (0, 2), (0, 1) for k = 0, 1, 2
  double dk[3], ok[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double tw = pos(mu + c1 * s[k]), fl = pos(mu - c1 * s[k]);
    dk[k] = 0.5 * (tw + fl);
    ok[k] = 0.5 * (fl - tw);
  }
  // z_a = vol^(1/2) V^T w_a (the volume split over both factors of each block)
  const double sv = sqrt(vol[t]);
  double z[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      z[a][j] = sv * (wl[a][0] * Vm[0][j] + wl[a][1] * Vm[1][j] + wl[a][2] * Vm[2][j]);
  // The projected F-Hessian rotated back by U, kept per pair of D-columns:
  // G[c][c'][r][r'] = sum_{i,i'} U[r][i] H_D+[(i,c),(i',c')] U[r'][i'].
  // Diagonal (c = c'): U diag(e) U^T with e_i = Ps[c][c] for i = c, else the
  // pair block's diagonal dk; off-diagonal: Ps[c][c'] u_c u_c'^T +
  // ok u_c' u_c^T, and G[c'][c] = G[c][c']^T.
  double Gd[3][3][3], Go[3][3][3];  // Gd[c] (symmetric); Go[0] = G[0][1], Go[1] = G[0][2], Go[2] = G[1][2]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double e[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) e[i] = i == c ? Ps[c][c] : dk[3 - i - c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = r; q < 3; ++q) {
        const double g = e[0] * U[r][0] * U[q][0] + e[1] * U[r][1] * U[q][1] + e[2] * U[r][2] * U[q][2];
        Gd[c][r][q] = g;
        Gd[c][q][r] = g;
      }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int c = m == 2 ? 1 : 0, c2 = m == 0 ? 1 : 2;
    const double ps = Ps[c][c2], o = ok[3 - c - c2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) Go[m][r][q] = ps * U[r][c] * U[q][c2] + o * U[r][c2] * U[q][c];
  }
  double* dst = out + (size_t)t * 90;
  int p = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    // Ma[c'] = sum_c z_a[c] G[c][c']
    double Ma[3][3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        Ma[0][r][q] = z[a][0] * Gd[0][r][q] + z[a][1] * Go[0][q][r] + z[a][2] * Go[1][q][r];
        Ma[1][r][q] = z[a][0] * Go[0][r][q] + z[a][1] * Gd[1][r][q] + z[a][2] * Go[2][q][r];
        Ma[2][r][q] = z[a][0] * Go[1][r][q] + z[a][1] * Go[2][r][q] + z[a][2] * Gd[2][r][q];
      }
#pragma unroll
    for (int b = a; b < 4; ++b, ++p) {
      const bool tr = v[a] > v[b];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const double h = z[b][0] * Ma[0][r][q] + z[b][1] * Ma[1][r][q] + z[b][2] * Ma[2][r][q];
          dst[9 * p + (tr ? 3 * q + r : 3 * r + q)] = h;
        }
    }
  }
}

__global__ void k_mass_blocks(const double* __restrict__ mass, int32_t V, double inv_dt2, double* __restrict__ out) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double m = mass[v] * inv_dt2;
  double* d = out + (size_t)v * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) d[k] = (k % 4 == 0) ? m : 0.0;
}

// Numeric assembly through the stored order: sorted entry i carries input
// sidx[i] into stored block O[i] (ascending).  Warp head-segmented sums
// (Sec. 5.2 FastSegmentReduction); runs shared between warps finish with
// atomics on the zeroed output.
__global__ void k_reduce_sorted(const uint32_t* __restrict__ sidx, const int32_t* __restrict__ O, int64_t n,
                                const double* __restrict__ vals, double* __restrict__ R) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool in = i < n;
  const int32_t b = in ? O[i] : -1;
  const int32_t b_prev = (in && i > 0) ? O[i - 1] : -1;
  const bool head = lane == 0 || b_prev != b;
  double v[9];
  if (in) {
    const double* src = vals + (size_t)sidx[i] * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = src[k];
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = 0.0;
  }
  const unsigned hm = __ballot_sync(kFull, head);
  const int send = segment_end(hm, lane);
  head_segmented_reduce<9>(v, lane, send);
  if (!in || !head) return;
  const bool cont_prev = lane == 0 && b_prev == b;
  bool cont_next = false;
  if (send == 32) {
    const int64_t nxt = i - lane + 32;
    cont_next = nxt < n && O[nxt] == b;
  }
  double* d = R + (size_t)b * 9;
  if (cont_prev || cont_next) {
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(d + k, v[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = v[k];
  }
}

__global__ void k_add_blocks(const int32_t* __restrict__ pos, const double* __restrict__ src, int64_t n,
                             double* __restrict__ R) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 9) return;
  const int64_t u = i / 9;
  R[(size_t)pos[u] * 9 + (i - u * 9)] += src[i];
}

// ------------------------------------------------------------------ contact springs
__global__ void k_spring_triplets(const int32_t* __restrict__ pairs, const double* __restrict__ K, int64_t nc,
                                  int32_t V, int32_t* __restrict__ rows, int32_t* __restrict__ cols,
                                  double* __restrict__ blocks, uint32_t* __restrict__ inc_key, int* flags) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc) return;
  int32_t i = pairs[2 * p], j = pairs[2 * p + 1];
  if (i < 0 || i >= V || j < 0 || j >= V || i == j) {
    atomicOr(flags, kErrIndex);
    i = 0, j = V > 1 ? 1 : 0;
  }
  rows[3 * p] = cols[3 * p] = i;
  rows[3 * p + 1] = cols[3 * p + 1] = j;
  rows[3 * p + 2] = i < j ? i : j;
  cols[3 * p + 2] = i < j ? j : i;
  const double* k = K + 9 * p;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      blocks[27 * p + 3 * a + b] = k[3 * a + b];
      blocks[27 * p + 9 + 3 * a + b] = k[3 * a + b];
      blocks[27 * p + 18 + 3 * a + b] = -(i < j ? k[3 * a + b] : k[3 * b + a]);
    }
  inc_key[2 * p] = (uint32_t)i;
  inc_key[2 * p + 1] = (uint32_t)j;
}

__global__ void k_keys_of(const int32_t* __restrict__ rid, const int32_t* __restrict__ cid, int64_t n, int shift,
                          uint64_t* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = ((uint64_t)(uint32_t)rid[i] << shift) | (uint32_t)cid[i];
}

// First index of a (ascending, n entries) with a[k] >= key.
__device__ __forceinline__ int64_t lower_bound(const uint64_t* __restrict__ a, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Merge of two ascending unique key lists E (elements) and C (springs).  A
// key's merged position is the number of merged keys below it: the element
// keys below it plus the spring keys below it that are not element keys.
// is_new[c] marks spring keys absent from E (lb[c] = their place in E);
// new_below = ExclusiveSum(is_new) over Uc + 1 entries.
__global__ void k_merge_flags(const uint64_t* __restrict__ ck, int64_t Uc, const uint64_t* __restrict__ ek,
                              int64_t Ue, int32_t* __restrict__ lb, int32_t* __restrict__ is_new) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > Uc) return;
  if (c == Uc) {
    is_new[c] = 0;
    return;
  }
  const int64_t l = lower_bound(ek, Ue, ck[c]);
  lb[c] = (int32_t)l;
  is_new[c] = (l == Ue || ek[l] != ck[c]) ? 1 : 0;
}

__global__ void k_merge_springs(const uint64_t* __restrict__ ck, int64_t Uc, const int32_t* __restrict__ lb,
                                const int32_t* __restrict__ new_below, uint64_t* __restrict__ mk,
                                int32_t* __restrict__ pos_c) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Uc) return;
  const int32_t p = lb[c] + new_below[c];
  pos_c[c] = p;
  mk[p] = ck[c];
}

__global__ void k_merge_elements(const uint64_t* __restrict__ ek, int64_t Ue, const uint64_t* __restrict__ ck,
                                 int64_t Uc, const int32_t* __restrict__ new_below, uint64_t* __restrict__ mk,
                                 int32_t* __restrict__ pos_e) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Ue) return;
  const int64_t p = a + new_below[lower_bound(ck, Uc, ek[a])];
  pos_e[a] = (int32_t)p;
  mk[p] = ek[a];
}

__global__ void k_decode(const uint64_t* __restrict__ mk, int64_t U, int shift, int32_t* __restrict__ rid,
                         int32_t* __restrict__ cid) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  rid[u] = (int32_t)(mk[u] >> shift);
  cid[u] = (int32_t)(mk[u] & ((1ull << shift) - 1));
}

__global__ void k_row_ptr(const int32_t* __restrict__ rid, int64_t U, int32_t n, int32_t* __restrict__ row_ptr) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u > U) return;
  const int32_t here = (u < U) ? rid[u] : n;
  const int32_t prev = (u > 0) ? rid[u - 1] : -1;
  for (int32_t r = prev + 1; r <= here; ++r) row_ptr[r] = (int32_t)u;
}

__global__ void k_compose(const int32_t* __restrict__ O, int64_t n, const int32_t* __restrict__ pos_e,
                          int32_t* __restrict__ Om) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Om[i] = pos_e[O[i]];
}

// ------------------------------------------------------------------ energy and gradient
// Per tet: vol Psi(F) and the node forces vol sum_j w[a][j] dPsi/df_j.
__global__ void __launch_bounds__(128) k_element_forces(const double* __restrict__ x,
                                                        const int32_t* __restrict__ tets,
                                                        const double* __restrict__ w,
                                                        const double* __restrict__ vol, int64_t T, double mu,
                                                        double lam, double* __restrict__ forces,
                                                        double* __restrict__ energy) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  int32_t v[4];
  double wl[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    v[a] = tets[4 * t + a];
#pragma unroll
    for (int j = 0; j < 3; ++j) wl[a][j] = w[12 * t + 3 * a + j];
  }
  double F[3][3];
  load_F(x, v, wl, F);
  // columns f_j, cofactor columns g_0 = f_1 x f_2, g_1 = f_2 x f_0, g_2 = f_0 x f_1
  double G[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    G[0][j] = F[1][j1] * F[2][j2] - F[2][j1] * F[1][j2];
    G[1][j] = F[2][j1] * F[0][j2] - F[0][j1] * F[2][j2];
    G[2][j] = F[0][j1] * F[1][j2] - F[1][j1] * F[0][j2];
  }
  const double J = F[0][0] * G[0][0] + F[1][0] * G[1][0] + F[2][0] * G[2][0];
  double Ic = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Ic += F[i][j] * F[i][j];
  const double alpha = 1.0 + mu / lam;
  const double vt = vol[t];
  energy[t] = vt * (0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - alpha) * (J - alpha));
  const double c1 = lam * (J - alpha);
  double P[3][3];  // dPsi/dF
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) P[i][j] = mu * F[i][j] + c1 * G[i][j];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      forces[12 * t + 3 * a + i] = vt * (P[i][0] * wl[a][0] + P[i][1] * wl[a][1] + P[i][2] * wl[a][2]);
}

__global__ void k_spring_forces(const int32_t* __restrict__ pairs, const double* __restrict__ K,
                                const double* __restrict__ rest, int64_t nc, const double* __restrict__ x,
                                double* __restrict__ cf, double* __restrict__ energy) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc) return;
  const int64_t i = pairs[2 * p], j = pairs[2 * p + 1];
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = x[3 * i + a] - x[3 * j + a] - rest[3 * p + a];
  double e = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double f = K[9 * p + 3 * a] * d[0] + K[9 * p + 3 * a + 1] * d[1] + K[9 * p + 3 * a + 2] * d[2];
    cf[6 * p + a] = f;
    cf[6 * p + 3 + a] = -f;
    e += d[a] * f;
  }
  energy[p] = 0.5 * e;
}

// Per vertex: the gathered element and spring forces plus the inertia term;
// energy m / (2 dt^2) |x - xt|^2.
__global__ void k_vertex_gradient(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_idx,
                                  const double* __restrict__ forces, const int32_t* __restrict__ cinc_ptr,
                                  const int32_t* __restrict__ cinc_idx, const double* __restrict__ cf,
                                  const double* __restrict__ mass, const double* __restrict__ x,
                                  const double* __restrict__ xt, int32_t V, double inv_dt2,
                                  double* __restrict__ grad, double* __restrict__ energy) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  double g[3] = {0.0, 0.0, 0.0};
  for (int32_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
    const int64_t e = inc_idx[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] += forces[3 * e + a];
  }
  if (cinc_ptr)
    for (int32_t k = cinc_ptr[v]; k < cinc_ptr[v + 1]; ++k) {
      const int64_t e = cinc_idx[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) g[a] += cf[3 * e + a];
    }
  const double m = mass[v] * inv_dt2;
  double e2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double dx = x[3 * (int64_t)v + a] - xt[3 * (int64_t)v + a];
    e2 += dx * dx;
    if (grad) grad[3 * (int64_t)v + a] = g[a] + m * dx;
  }
  energy[v] = 0.5 * m * e2;
}

// Deterministic sums: a fixed grid of strided partial sums, then one block.
constexpr int kSumBlocks = 304;
__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  return sh[0];
}

// part[b] = (sum of a over the block's stride), for kind 0; for kind 1 the
// pair (sum a_i b_i, max |b_i|) of a, b.
__global__ void __launch_bounds__(256) k_partials(const double* __restrict__ a, const double* __restrict__ b,
                                                  int64_t n, double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0, m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    if (b) {
      s += a[i] * b[i];
      m = fmax(m, fabs(b[i]));
    } else {
      s += a[i];
    }
  }
  const double ts = block_sum(s, sh);
  __syncthreads();
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ts;
    part[2 * blockIdx.x + 1] = sh[0];
  }
}

__global__ void __launch_bounds__(256) k_finish(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0, m = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) {
    s += part[2 * i];
    m = fmax(m, part[2 * i + 1]);
  }
  const double ts = block_sum(s, sh);
  __syncthreads();
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = ts;
    out[1] = sh[0];
  }
}

__global__ void k_axpy_to(const double* __restrict__ x, const double* __restrict__ d, double alpha, int64_t n,
                          double* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] + alpha * d[i];
}

__global__ void k_negate(const double* __restrict__ a, int64_t n, double* __restrict__ b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = -a[i];
}

}  // namespace fem
}  // namespace gs

namespace gs {
namespace fem {
__global__ void k_element_rows_cols(const int32_t* __restrict__ tets, int64_t T, int32_t V, int32_t* __restrict__ rows,
                                    int32_t* __restrict__ cols) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 10 * T + V) return;
  if (i < 10 * T) {
    const int64_t t = i / 10;
    int a, b;
    pair_nodes((int)(i - 10 * t), a, b);
    const int32_t va = tets[4 * t + a], vb = tets[4 * t + b];
    rows[i] = va < vb ? va : vb;
    cols[i] = va < vb ? vb : va;
  } else {
    rows[i] = cols[i] = (int32_t)(i - 10 * T);
  }
}

}  // namespace fem
}  // namespace gs

// ====================================================================== host
namespace gs {
namespace fem {
namespace {

// Device buffers of one call, freed on every return.
struct Tmp {
  gs_ctx ctx;
  std::vector<void*> ptrs;
  ~Tmp() {
    for (void* p : ptrs) ctx->release(p);
  }
  template <typename T>
  int get(T** out, size_t count) {
    void* p = nullptr;
    GS_TRY(ctx->alloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
    ptrs.push_back(p);
    *out = (T*)p;
    return GS_OK;
  }
};

template <typename K, typename Vt>
int sort_pairs(gs_ctx ctx, Tmp& tmp, const K* kin, K* kout, const Vt* vin, Vt* vout, int64_t n, int end_bit) {
  size_t tb = 0;
  GS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, kin, kout, vin, vout, n, 0, end_bit, ctx->stream));
  void* t;
  GS_TRY(tmp.get((char**)&t, tb));
  GS_PROF(ctx, GS_K_LIBPRIM);
  GS_CUDA(cub::DeviceRadixSort::SortPairs(t, tb, kin, kout, vin, vout, n, 0, end_bit, ctx->stream));
  return GS_OK;
}

int exclusive_sum(gs_ctx ctx, Tmp& tmp, const int32_t* in, int32_t* out, int64_t n) {
  size_t tb = 0;
  GS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, n, ctx->stream));
  void* t;
  GS_TRY(tmp.get((char**)&t, tb));
  GS_PROF(ctx, GS_K_LIBPRIM);
  GS_CUDA(cub::DeviceScan::ExclusiveSum(t, tb, in, out, n, ctx->stream));
  return GS_OK;
}

int read_i32(gs_ctx ctx, const int32_t* d, int32_t* h) {
  GS_CUDA(cudaMemcpyAsync(ctx->h_pinned + 12, d, 4, cudaMemcpyDeviceToHost, ctx->stream));
  GS_CUDA(cudaStreamSynchronize(ctx->stream));
  *h = ctx->h_pinned[12];
  return GS_OK;
}

int check_flags(gs_ctx ctx, const char* what) {
  int flags = 0;
  GS_TRY(ctx->take_flags(&flags));
  if (flags) {
    int s = status_from_flags(flags);
    set_error("%s: %s", what, flags & kErrIndex ? "an index out of range or a repeated node"
                               : flags & kErrNonFinite ? "a degenerate or non-finite rest element"
                                                       : "device error");
    return s;
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// Vertex -> entries CSR: keys (vertex of each entry, uint32), sorted stably.
int incidence(gs_ctx ctx, Tmp& tmp, const uint32_t* keys, int64_t n, int32_t V, int32_t* ptr, int32_t* idx) {
  uint32_t *skeys, *iota;
  GS_TRY(tmp.get(&skeys, n));
  GS_TRY(tmp.get(&iota, n));
  cudaStream_t st = ctx->stream;
  if (n > 0) {
    { GS_PROF(ctx, GS_K_OTHER); k_iota<<<ceil_div(n, 256), 256, 0, st>>>(iota, n); }
    GS_TRY(sort_pairs(ctx, tmp, keys, skeys, iota, (uint32_t*)idx, n, bits_for(V)));
  }
  { GS_PROF(ctx, GS_K_OTHER); k_seg_ptr<<<ceil_div(n + 1, 256), 256, 0, st>>>(skeys, n, V, ptr); }
  return GS_OK;
}

// Merged pattern of the element keys and the current spring blocks.
int merge_pattern(gs_ctx ctx, gs_fem f) {
  cudaStream_t st = ctx->stream;
  Tmp tmp{ctx};
  const int64_t Uc = f->c_mat ? f->c_mat->nnzb : 0;
  uint64_t *ck, *mk;
  int32_t *pos_e, *lb, *is_new, *new_below;
  GS_TRY(tmp.get(&ck, Uc));
  GS_TRY(tmp.get(&mk, f->U_e + Uc));
  GS_TRY(tmp.get(&pos_e, f->U_e));
  GS_TRY(tmp.get(&lb, Uc));
  GS_TRY(tmp.get(&is_new, Uc + 1));
  GS_TRY(tmp.get(&new_below, Uc + 1));
  ctx->release(f->pos_c);
  f->pos_c = nullptr;
  GS_TRY(ctx->alloc((void**)&f->pos_c, std::max<int64_t>(Uc, 1) * 4));
  {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    if (Uc) k_keys_of<<<ceil_div(Uc, 256), 256, 0, st>>>(f->c_mat->rid, f->c_mat->cid, Uc, f->shift, ck);
  }
  { GS_PROF(ctx, GS_K_ASSEMBLE); k_merge_flags<<<ceil_div(Uc + 1, 256), 256, 0, st>>>(ck, Uc, f->e_keys, f->U_e, lb, is_new); }
  GS_TRY(exclusive_sum(ctx, tmp, is_new, new_below, Uc + 1));
  {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    if (Uc) k_merge_springs<<<ceil_div(Uc, 256), 256, 0, st>>>(ck, Uc, lb, new_below, mk, f->pos_c);
  }
  {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    if (f->U_e) k_merge_elements<<<ceil_div(f->U_e, 256), 256, 0, st>>>(f->e_keys, f->U_e, ck, Uc, new_below, mk, pos_e);
  }
  int32_t added = 0;
  GS_TRY(read_i32(ctx, new_below + Uc, &added));
  const int64_t U = f->U_e + added;
  ctx->release(f->rid);
  ctx->release(f->cid);
  f->rid = f->cid = nullptr;
  GS_TRY(ctx->alloc((void**)&f->rid, std::max<int64_t>(U, 1) * 4));
  GS_TRY(ctx->alloc((void**)&f->cid, std::max<int64_t>(U, 1) * 4));
  {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    if (U) k_decode<<<ceil_div(U, 256), 256, 0, st>>>(mk, U, f->shift, f->rid, f->cid);
  }
  { GS_PROF(ctx, GS_K_ASSEMBLE); k_row_ptr<<<ceil_div(U + 1, 256), 256, 0, st>>>(f->rid, U, f->V, f->row_ptr); }
  {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    if (f->n_in) k_compose<<<ceil_div(f->n_in, 256), 256, 0, st>>>(f->e_O, f->n_in, pos_e, f->O_m);
  }
  f->U = U;
  ++f->version;
  return check_flags(ctx, "fem pattern");
}

void release_springs(gs_fem f) {
  gs_ctx c = f->owner;
  for (void* p : {(void*)f->c_pairs, (void*)f->c_K, (void*)f->c_rest, (void*)f->c_forces, (void*)f->cinc_ptr,
                  (void*)f->cinc_idx})
    c->release(p);
  f->c_pairs = f->cinc_ptr = f->cinc_idx = nullptr;
  f->c_K = f->c_rest = f->c_forces = nullptr;
  gs_mat_destroy(f->c_mat);
  f->c_mat = nullptr;
  f->nc = 0;
}

// Energy terms and (optionally) the gradient at x; *E the total on the host.
int energy_grad(gs_ctx ctx, gs_fem f, const double* x, const double* xt, double* grad, double* part, double* E) {
  cudaStream_t st = ctx->stream;
  const double inv_dt2 = 1.0 / (f->dt * f->dt);
  {
    GS_PROF(ctx, GS_K_ELEMENT);
    if (f->T) k_element_forces<<<ceil_div(f->T, 128), 128, 0, st>>>(x, f->tets, f->w, f->vol, f->T, f->mu, f->lam,
                                                                    f->forces, f->energy);
  }
  {
    GS_PROF(ctx, GS_K_ELEMENT);
    if (f->nc) k_spring_forces<<<ceil_div(f->nc, 256), 256, 0, st>>>(f->c_pairs, f->c_K, f->c_rest, f->nc, x,
                                                                     f->c_forces, f->energy + f->T);
  }
  {
    GS_PROF(ctx, GS_K_ELEMENT);
    k_vertex_gradient<<<ceil_div(f->V, 256), 256, 0, st>>>(f->inc_ptr, f->inc_idx, f->forces, f->cinc_ptr,
                                                           f->cinc_idx, f->c_forces, f->mass, x, xt, f->V, inv_dt2,
                                                           grad, f->energy + f->T + f->nc);
  }
  const int64_t n = f->T + f->nc + f->V;
  {
    GS_PROF(ctx, GS_K_PCG_VECTOR);
    k_partials<<<kSumBlocks, 256, 0, st>>>(f->energy, nullptr, n, part);
  }
  {
    GS_PROF(ctx, GS_K_PCG_VECTOR);
    k_finish<<<1, 256, 0, st>>>(part, kSumBlocks, part + 2 * kSumBlocks);
  }
  double* h = (double*)(ctx->h_pinned + 128);
  GS_CUDA(cudaMemcpyAsync(h, part + 2 * kSumBlocks, 8, cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  GS_CUDA(cudaGetLastError());
  *E = h[0];
  return GS_OK;
}

// (sum a_i b_i, max |b_i|) on the host.
int dot_max(gs_ctx ctx, const double* a, const double* b, int64_t n, double* part, double* out2) {
  cudaStream_t st = ctx->stream;
  {
    GS_PROF(ctx, GS_K_PCG_VECTOR);
    k_partials<<<kSumBlocks, 256, 0, st>>>(a, b, n, part);
  }
  {
    GS_PROF(ctx, GS_K_PCG_VECTOR);
    k_finish<<<1, 256, 0, st>>>(part, kSumBlocks, part + 2 * kSumBlocks);
  }
  double* h = (double*)(ctx->h_pinned + 128);
  GS_CUDA(cudaMemcpyAsync(h, part + 2 * kSumBlocks, 16, cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  out2[0] = h[0];
  out2[1] = h[1];
  return GS_OK;
}

int hessian_values(gs_ctx ctx, gs_fem f, const double* x) {
  cudaStream_t st = ctx->stream;
  if (f->T) {
    GS_PROF(ctx, GS_K_ELEMENT);
    k_element_hessians<<<ceil_div(f->T, 128), 128, 0, st>>>(x, f->tets, f->w, f->vol, f->T, f->mu, f->lam,
                                                            f->e_vals);
  }
  {
    GS_PROF(ctx, GS_K_ELEMENT);
    k_mass_blocks<<<ceil_div(f->V, 256), 256, 0, st>>>(f->mass, f->V, 1.0 / (f->dt * f->dt), f->e_vals + 90 * f->T);
  }
  return GS_OK;
}

int refill(gs_ctx ctx, gs_fem f, const double* x, gs_mat m) {
  cudaStream_t st = ctx->stream;
  GS_TRY(hessian_values(ctx, f, x));
  GS_CUDA(cudaMemsetAsync(m->au, 0, (size_t)f->U * 72, st));
  {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    if (f->n_in) k_reduce_sorted<<<ceil_div(f->n_in, 256), 256, 0, st>>>(f->e_sidx, f->O_m, f->n_in, f->e_vals, m->au);
  }
  if (f->c_mat && f->c_mat->nnzb) {
    GS_PROF(ctx, GS_K_ASSEMBLE);
    k_add_blocks<<<ceil_div(f->c_mat->nnzb * 9, 256), 256, 0, st>>>(f->pos_c, f->c_mat->au, f->c_mat->nnzb, m->au);
  }
  // copies derived from the values are rebuilt on their next use
  ctx->release(m->au32);
  ctx->release(m->au_ff);
  ctx->release(m->ff_k);
  m->au32 = nullptr;
  m->au_ff = nullptr;
  m->ff_k = nullptr;
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace
}  // namespace fem
}  // namespace gs

using namespace gs;
using namespace gs::fem;

extern "C" {

int gs_fem_destroy(gs_fem f) {
  if (!f) return GS_OK;
  gs_ctx c = f->owner;
  release_springs(f);
  for (void* p : {(void*)f->X, (void*)f->tets, (void*)f->w, (void*)f->vol, (void*)f->mass, (void*)f->inc_ptr,
                  (void*)f->inc_idx, (void*)f->e_sidx, (void*)f->e_O, (void*)f->e_keys, (void*)f->e_vals,
                  (void*)f->forces, (void*)f->energy, (void*)f->pos_c, (void*)f->rid, (void*)f->cid,
                  (void*)f->row_ptr, (void*)f->O_m})
    c->release(p);
  delete f;
  return GS_OK;
}

int gs_fem_create(gs_ctx ctx, int32_t n_vertices, int64_t n_tets, const double* X, const int32_t* tets, double E,
                  double nu, double rho, double dt, gs_fem* out) {
  GS_CHECK(ctx && out, GS_ERR_INVALID, "gs_fem_create: null context or output");
  *out = nullptr;
  const int32_t V = n_vertices;
  const int64_t T = n_tets;
  GS_CHECK(V > 0 && V < (1 << 30) && T >= 0 && 10 * T + V < (1LL << 31), GS_ERR_INVALID,
           "gs_fem_create: %d vertices, %lld tets out of range", V, (long long)T);
  GS_CHECK(X && (T == 0 || tets), GS_ERR_INVALID, "gs_fem_create: null positions or tets");
  GS_CHECK(E > 0 && nu >= 0 && nu < 0.5 && rho > 0 && dt > 0, GS_ERR_INVALID,
           "gs_fem_create: E %g, nu %g, rho %g, dt %g out of range", E, nu, rho, dt);
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  gs_fem f = new gs_fem_s();
  f->owner = ctx;
  f->V = V;
  f->T = T;
  const double mu_l = E / (2.0 * (1.0 + nu)), lam_l = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  f->mu = 4.0 / 3.0 * mu_l;
  f->lam = lam_l + 5.0 / 6.0 * mu_l;
  f->rho = rho;
  f->dt = dt;
  f->shift = bits_for(V);
  f->n_in = 10 * T + V;
  auto fail = [&](int s) {
    gs_fem_destroy(f);
    return s;
  };
  int s;
  if ((s = ctx->alloc((void**)&f->X, (size_t)V * 24)) || (s = ctx->alloc((void**)&f->tets, std::max<int64_t>(T, 1) * 16)) ||
      (s = ctx->alloc((void**)&f->w, std::max<int64_t>(T, 1) * 96)) ||
      (s = ctx->alloc((void**)&f->vol, std::max<int64_t>(T, 1) * 8)) || (s = ctx->alloc((void**)&f->mass, (size_t)V * 8)) ||
      (s = ctx->alloc((void**)&f->inc_ptr, (size_t)(V + 1) * 4)) ||
      (s = ctx->alloc((void**)&f->inc_idx, std::max<int64_t>(4 * T, 1) * 4)) ||
      (s = ctx->alloc((void**)&f->e_sidx, (size_t)f->n_in * 4)) || (s = ctx->alloc((void**)&f->e_O, (size_t)f->n_in * 4)) ||
      (s = ctx->alloc((void**)&f->O_m, (size_t)f->n_in * 4)) ||
      (s = ctx->alloc((void**)&f->e_vals, (size_t)f->n_in * 72)) ||
      (s = ctx->alloc((void**)&f->forces, std::max<int64_t>(T, 1) * 96)) ||
      (s = ctx->alloc((void**)&f->energy, (size_t)(T + V) * 8)) ||
      (s = ctx->alloc((void**)&f->row_ptr, (size_t)(V + 1) * 4)))
    return fail(s);
  if (cudaMemcpyAsync(f->X, X, (size_t)V * 24, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      (T && cudaMemcpyAsync(f->tets, tets, (size_t)T * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
    return fail(GS_ERR_CUDA);
  {
    GS_PROF(ctx, GS_K_ELEMENT);
    if (T) k_rest<<<ceil_div(T, 256), 256, 0, st>>>(f->X, f->tets, T, V, f->w, f->vol, ctx->d_flags);
  }
  if ((s = check_flags(ctx, "gs_fem_create"))) return fail(s);
  {
    Tmp tmp{ctx};
    if ((s = incidence(ctx, tmp, (const uint32_t*)f->tets, 4 * T, V, f->inc_ptr, f->inc_idx))) return fail(s);
    { GS_PROF(ctx, GS_K_ELEMENT); k_mass<<<ceil_div(V, 256), 256, 0, st>>>(f->inc_ptr, f->inc_idx, f->vol, rho, V, f->mass); }
    // element keys, sorted once
    uint64_t *keys, *skeys;
    uint32_t* iota;
    int32_t* P;
    const int64_t n = f->n_in;
    if ((s = tmp.get(&keys, n)) || (s = tmp.get(&skeys, n)) || (s = tmp.get(&iota, n)) || (s = tmp.get(&P, n)))
      return fail(s);
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_element_keys<<<ceil_div(n, 256), 256, 0, st>>>(f->tets, T, V, f->shift, keys); }
    { GS_PROF(ctx, GS_K_OTHER); k_iota<<<ceil_div(n, 256), 256, 0, st>>>(iota, n); }
    if ((s = sort_pairs(ctx, tmp, keys, skeys, iota, f->e_sidx, n, 2 * f->shift))) return fail(s);
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_run_ends<<<ceil_div(n, 256), 256, 0, st>>>(skeys, n, P); }
    if ((s = exclusive_sum(ctx, tmp, P, f->e_O, n))) return fail(s);
    int32_t last = 0;
    if ((s = read_i32(ctx, f->e_O + n - 1, &last))) return fail(s);
    f->U_e = (int64_t)last + 1;
    if ((s = ctx->alloc((void**)&f->e_keys, (size_t)f->U_e * 8))) return fail(s);
    { GS_PROF(ctx, GS_K_ASSEMBLE); k_unique_keys<<<ceil_div(n, 256), 256, 0, st>>>(skeys, f->e_O, n, f->e_keys); }
    if ((s = check_flags(ctx, "gs_fem_create"))) return fail(s);
  }
  if ((s = merge_pattern(ctx, f))) return fail(s);
  *out = f;
  return GS_OK;
}

int gs_fem_set_springs(gs_ctx ctx, gs_fem f, const int32_t* pairs, const double* K, const double* rest,
                       int64_t n_springs) {
  GS_CHECK(ctx && f && f->owner == ctx, GS_ERR_INVALID, "gs_fem_set_springs: null or foreign body");
  GS_CHECK(n_springs >= 0 && 3 * n_springs < (1LL << 31) && (n_springs == 0 || (pairs && K && rest)),
           GS_ERR_INVALID, "gs_fem_set_springs: bad springs");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int64_t nc = n_springs;
  // the new springs are built aside; the body keeps its old ones if that fails
  gs_fem_s next;
  next.owner = ctx;
  next.V = f->V;
  auto fail = [&](int s) {
    release_springs(&next);
    return s;
  };
  int s;
  if (nc) {
    if ((s = ctx->alloc((void**)&next.c_pairs, (size_t)nc * 8)) || (s = ctx->alloc((void**)&next.c_K, (size_t)nc * 72)) ||
        (s = ctx->alloc((void**)&next.c_rest, (size_t)nc * 24)) ||
        (s = ctx->alloc((void**)&next.c_forces, (size_t)nc * 48)) ||
        (s = ctx->alloc((void**)&next.cinc_ptr, (size_t)(f->V + 1) * 4)) ||
        (s = ctx->alloc((void**)&next.cinc_idx, (size_t)nc * 8)))
      return fail(s);
    next.nc = nc;
    if (cudaMemcpyAsync(next.c_pairs, pairs, (size_t)nc * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(next.c_K, K, (size_t)nc * 72, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(next.c_rest, rest, (size_t)nc * 24, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return fail(GS_ERR_CUDA);
    Tmp tmp{ctx};
    int32_t *rows, *cols;
    double* blocks;
    uint32_t* ikey;
    if ((s = tmp.get(&rows, 3 * nc)) || (s = tmp.get(&cols, 3 * nc)) || (s = tmp.get(&blocks, 27 * nc)) ||
        (s = tmp.get(&ikey, 2 * nc)))
      return fail(s);
    {
      GS_PROF(ctx, GS_K_ELEMENT);
      k_spring_triplets<<<ceil_div(nc, 256), 256, 0, st>>>(next.c_pairs, next.c_K, nc, f->V, rows, cols, blocks, ikey,
                                                           ctx->d_flags);
    }
    if ((s = check_flags(ctx, "gs_fem_set_springs"))) return fail(s);
    // only the spring keys are sorted: their own reduction, then a merge
    if ((s = reduce_blocks(ctx, f->V, rows, cols, blocks, 3 * nc, &next.c_mat))) return fail(s);
    if ((s = incidence(ctx, tmp, ikey, 2 * nc, f->V, next.cinc_ptr, next.cinc_idx))) return fail(s);
  }
  double* energy = nullptr;
  if ((s = ctx->alloc((void**)&energy, (size_t)(f->T + nc + f->V) * 8))) return fail(s);
  release_springs(f);
  ctx->release(f->energy);
  f->energy = energy;
  f->nc = next.nc;
  f->c_pairs = next.c_pairs;
  f->c_K = next.c_K;
  f->c_rest = next.c_rest;
  f->c_forces = next.c_forces;
  f->cinc_ptr = next.cinc_ptr;
  f->cinc_idx = next.cinc_idx;
  f->c_mat = next.c_mat;
  return merge_pattern(ctx, f);
}

int gs_fem_info(gs_fem f, int64_t* n_stored, int64_t* n_element_stored, double* lame_mu, double* lame_lambda) {
  GS_CHECK(f, GS_ERR_INVALID, "gs_fem_info: null body");
  if (n_stored) *n_stored = f->U;
  if (n_element_stored) *n_element_stored = f->U_e;
  if (lame_mu) *lame_mu = f->mu;
  if (lame_lambda) *lame_lambda = f->lam;
  return GS_OK;
}

int gs_fem_export_rest(gs_ctx ctx, gs_fem f, double* w, double* vol, double* mass) {
  GS_CHECK(ctx && f, GS_ERR_INVALID, "gs_fem_export_rest: null argument");
  cudaStream_t st = ctx->stream;
  if (w && f->T) GS_CUDA(cudaMemcpyAsync(w, f->w, (size_t)f->T * 96, cudaMemcpyDeviceToDevice, st));
  if (vol && f->T) GS_CUDA(cudaMemcpyAsync(vol, f->vol, (size_t)f->T * 8, cudaMemcpyDeviceToDevice, st));
  if (mass) GS_CUDA(cudaMemcpyAsync(mass, f->mass, (size_t)f->V * 8, cudaMemcpyDeviceToDevice, st));
  return GS_OK;
}

int gs_fem_energy(gs_ctx ctx, gs_fem f, const double* x, const double* xt, double* energy, double* grad) {
  GS_CHECK(ctx && f && f->owner == ctx && x && xt && energy, GS_ERR_INVALID, "gs_fem_energy: null argument");
  GS_CUDA(cudaSetDevice(ctx->device));
  Tmp tmp{ctx};
  double* part;
  GS_TRY(tmp.get(&part, 2 * kSumBlocks + 2));
  return energy_grad(ctx, f, x, xt, grad, part, energy);
}

int gs_fem_triplets(gs_ctx ctx, gs_fem f, const double* x, int32_t* rows, int32_t* cols, double* blocks) {
  GS_CHECK(ctx && f && f->owner == ctx && x && blocks, GS_ERR_INVALID, "gs_fem_triplets: null argument");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  GS_TRY(hessian_values(ctx, f, x));
  GS_CUDA(cudaMemcpyAsync(blocks, f->e_vals, (size_t)f->n_in * 72, cudaMemcpyDeviceToDevice, st));
  Tmp tmp{ctx};
  int32_t *r = rows, *c = cols;
  if (!r) GS_TRY(tmp.get(&r, f->n_in + 3 * f->nc));
  if (!c) GS_TRY(tmp.get(&c, f->n_in + 3 * f->nc));
  { GS_PROF(ctx, GS_K_ELEMENT); k_element_rows_cols<<<ceil_div(f->n_in, 256), 256, 0, st>>>(f->tets, f->T, f->V, r, c); }
  if (f->nc) {
    uint32_t* ikey;
    GS_TRY(tmp.get(&ikey, 2 * f->nc));
    GS_PROF(ctx, GS_K_ELEMENT);
    k_spring_triplets<<<ceil_div(f->nc, 256), 256, 0, st>>>(f->c_pairs, f->c_K, f->nc, f->V, r + f->n_in,
                                                            c + f->n_in, blocks + 9 * f->n_in, ikey, ctx->d_flags);
  }
  return check_flags(ctx, "gs_fem_triplets");
}

int gs_fem_assemble(gs_ctx ctx, gs_fem f, const double* x, gs_mat* out) {
  GS_CHECK(ctx && f && f->owner == ctx && x && out, GS_ERR_INVALID, "gs_fem_assemble: null argument");
  *out = nullptr;
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  gs_mat m = new gs_mat_s();
  m->n = f->V;
  m->owner = ctx;
  m->nnzb = f->U;
  m->pattern_owner = f;
  m->pattern_version = f->version;
  auto fail = [&](int s) {
    gs_mat_destroy(m);
    return s;
  };
  int s;
  const size_t U = std::max<int64_t>(f->U, 1);
  if ((s = ctx->alloc((void**)&m->rid, U * 4)) || (s = ctx->alloc((void**)&m->cid, U * 4)) ||
      (s = ctx->alloc((void**)&m->au, U * 72)) || (s = ctx->alloc((void**)&m->row_ptr, (size_t)(f->V + 1) * 4)))
    return fail(s);
  if (cudaMemcpyAsync(m->rid, f->rid, (size_t)f->U * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m->cid, f->cid, (size_t)f->U * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m->row_ptr, f->row_ptr, (size_t)(f->V + 1) * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return fail(GS_ERR_CUDA);
  if ((s = refill(ctx, f, x, m))) return fail(s);
  *out = m;
  return GS_OK;
}

int gs_fem_refill(gs_ctx ctx, gs_fem f, const double* x, gs_mat m) {
  GS_CHECK(ctx && f && f->owner == ctx && x && m, GS_ERR_INVALID, "gs_fem_refill: null argument");
  GS_CHECK(m->pattern_owner == f && m->pattern_version == f->version, GS_ERR_INVALID,
           "gs_fem_refill: the matrix was not assembled from this body's current pattern");
  GS_CUDA(cudaSetDevice(ctx->device));
  return refill(ctx, f, x, m);
}

int gs_fem_newton(gs_ctx ctx, gs_fem f, const double* xt, double* x, const int32_t* adj_ptr, const int32_t* adj,
                  const gs_newton_opts* o, gs_newton_stats* stats, double* energies) {
  GS_CHECK(ctx && f && f->owner == ctx && xt && x && adj_ptr && o && stats, GS_ERR_INVALID,
           "gs_fem_newton: null argument");
  GS_CHECK(o->max_newton >= 0 && o->tol >= 0 && o->armijo >= 0 && o->armijo < 1 && o->max_halvings >= 0,
           GS_ERR_INVALID, "gs_fem_newton: options out of range");
  GS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  memset(stats, 0, sizeof(*stats));
  const int64_t n3 = 3LL * f->V;
  Tmp tmp{ctx};
  double *grad, *d, *b, *xtry, *part;
  GS_TRY(tmp.get(&grad, n3));
  GS_TRY(tmp.get(&d, n3));
  GS_TRY(tmp.get(&b, n3));
  GS_TRY(tmp.get(&xtry, n3));
  GS_TRY(tmp.get(&part, 2 * kSumBlocks + 2));
  cudaEvent_t ev[2];
  GS_CUDA(cudaEventCreate(&ev[0]));
  GS_CUDA(cudaEventCreate(&ev[1]));
  gs_mat mat = nullptr;
  gs_mas mas = nullptr;
  int status = GS_OK;
  // time one phase on the stream into stats->ms[k]
  auto phase = [&](int k, auto&& fn) -> int {
    if (cudaEventRecord(ev[0], st) != cudaSuccess) return GS_ERR_CUDA;
    int s = fn();
    if (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess) return GS_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    stats->ms[k] += ms;
    stats->ms[5] += ms;
    return s;
  };
  double E = 0.0;
  status = phase(0, [&] { return energy_grad(ctx, f, x, xt, grad, part, &E); });
  stats->energy0 = E;
  if (energies && status == GS_OK) energies[0] = E;
  gs_mas_opts mo{o->domain_size, o->max_levels, o->precision};
  for (int it = 0; status == GS_OK && it <= o->max_newton; ++it) {
    // Hessian values into the fixed pattern (the first call makes the matrix)
    status = phase(1, [&] { return mat ? refill(ctx, f, x, mat) : gs_fem_assemble(ctx, f, x, &mat); });
    if (status) break;
    status = phase(2, [&] {
      return mas ? gs_mas_refresh(ctx, mas, mat)
                 : gs_build_mas_mesh(ctx, mat, f->X, o->part_rule, adj_ptr, adj, f->c_pairs, f->nc, &mo, &mas);
    });
    if (status) break;
    int32_t pit = 0;
    double rr = 0.0;
    status = phase(3, [&] {
      {
        GS_PROF(ctx, GS_K_PCG_VECTOR);
        k_negate<<<ceil_div(n3, 256), 256, 0, st>>>(grad, n3, b);
      }
      int s = gs_pcg_solve(ctx, mat, mas, b, 1, o->pcg_tol, o->pcg_max_iter, o->spmv_variant, d, &pit, &rr);
      return s == GS_ERR_MAXITER ? GS_OK : s;  // an inexact direction is still a descent direction
    });
    stats->pcg_iterations += pit;
    if (status) break;
    double gd_dinf[2];
    if ((status = dot_max(ctx, grad, d, n3, part, gd_dinf))) break;
    stats->step_inf = gd_dinf[1];
    if (gd_dinf[1] <= o->tol * f->dt) {
      stats->converged = 1;
      break;
    }
    if (it == o->max_newton) break;  // out of steps
    if (!(gd_dinf[0] < 0.0)) {
      set_error("gs_fem_newton: the direction is not a descent direction (g.d = %g)", gd_dinf[0]);
      status = GS_ERR_NOT_SPD;
      break;
    }
    double alpha = 1.0, Et = 0.0;
    int h = 0;
    status = phase(4, [&] {
      for (;;) {
        {
          GS_PROF(ctx, GS_K_PCG_VECTOR);
          k_axpy_to<<<ceil_div(n3, 256), 256, 0, st>>>(x, d, alpha, n3, xtry);
        }
        GS_TRY(energy_grad(ctx, f, xtry, xt, nullptr, part, &Et));
        if (Et <= E + o->armijo * alpha * gd_dinf[0] || h >= o->max_halvings) return GS_OK;
        alpha *= 0.5;
        ++h;
      }
    });
    if (status) break;
    stats->halvings += h;
    if (cudaMemcpyAsync(x, xtry, (size_t)n3 * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      status = GS_ERR_CUDA;
      break;
    }
    ++stats->iterations;
    status = phase(0, [&] { return energy_grad(ctx, f, x, xt, grad, part, &E); });
    if (energies && status == GS_OK) energies[stats->iterations] = E;
  }
  stats->energy = E;
  gs_mas_destroy(mas);
  gs_mat_destroy(mat);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (status == GS_OK && !stats->converged) {
    set_error("gs_fem_newton: not converged in %d steps", o->max_newton);
    status = GS_ERR_MAXITER;
  }
  return status;
}

}  // extern "C"
