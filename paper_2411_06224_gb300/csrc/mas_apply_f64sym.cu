// Every level's MAS product z_d = M_d^{-1} r_d (Eq. 6) in FP64 accuracy on
// the BF16 tensor cores, streaming only the block lower triangle of each
// symmetric inverse, one byte per digit.
//
// The inverses are symmetric, so a symmetric scaling keeps them symmetric:
// with R_i = max_k |M_ik| < 2^e_i and c_i = ceil(e_i / 2),
//   |M_ik| <= sqrt(R_i R_k) < 2^(c_i + c_k),
// so X~ = D^-1 M D^-1 (D = diag 2^c_i) has every entry below 1 and
//   z_i = 2^c_i sum_k X~_ik (2^c_k r_k).
// Build time: X_ik = rint(X~_ik 2^55) (|X| <= 2^55) is cut into 8 balanced
// base-128 digits m_0..m_7 (m_0 in [-64, 64], the others in [-64, 63]),
// X = sum_p m_p 128^(7-p); only the 8x8 core blocks (I, K) with K <= I are
// stored, each digit as the byte m + 64: 40 KB per 96 x 96 domain, 1.07x the
// bytes of the packed FP64 lower triangle.
//
// Apply, one CTA per domain (128 threads):
//   * r~ = 2^c_j r_j, column exponent b_k with |r~_jk| < 2^(b_k - 1) and
//     Y_jk = rint(r~_jk 2^(56 - b_k)) -> 8 balanced base-128 digits n_q,
//     written as BF16 into the B operand (column 8 q + k, N = 64);
//   * each digit matrix p is bulk-copied into a staging ring and expanded by
//     all four warps into the BF16 A operand: the byte u becomes the BF16
//     with bits 0x43uu, the exact value 128 + u = 192 + m (one byte permute
//     for two entries); a stored block goes to (I, K) and, transposed by
//     movmatrix, to (K, I);
//   * one MMA per digit matrix and K step writes the digit-pair groups
//     t = p + q at TMEM columns 8 t .. 8 t + 7 (the B columns of digit q sit
//     8 q columns further), so G'_t = sum_{p+q=t} (192 + m_p) n_q collects in
//     place; only q <= 9 - p is issued (N rounded up to a multiple of 16);
//   * every |(192 + m) n| <= 256 * 64, 96 terms, <= 8 pairs: |G'_t| < 2^24, so
//     the FP32 accumulator is exact; the bias is removed in the epilogue,
//     G_t = G'_t - 192 sum_{q in pair range of t} sum_j n_q(j, k);
//   * z_ik = 2^(c_i + b_k - 76) sum_{t=0..9} G_t 128^(9-t), combined in 128-bit
//     integers and rounded once to a double.
// Per output the dropped groups (t >= 10) and the two roundings give
//   |dz_ik| <= 2^(c_i - 56) sum_j 2^c_j |r_jk| + 2^(b_k - 57) sum_j |M_ij| 2^-c_j
//              + 2^(c_i + b_k - 61),
// FP64's own rounding level relative to the symmetric scale of M.
// All waits are bounded (kErrTimeout); TMEM is always freed.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "fp64split.cuh"
#include "umma.cuh"

namespace gs {
namespace f64sym {

constexpr int kDigits = 8;   // base-128 digits per entry, both operands
constexpr int kGroups = 10;  // digit-pair groups t = p + q kept (t = 0..9)
constexpr int kStage = 4;    // staging slots, one digit matrix of a domain each
constexpr int kThreads = 128;
constexpr int kM = 128;
constexpr int kTmemCols = 128;
constexpr int kBias = 192;           // an expanded A entry holds 192 + m
constexpr int kNoScale = -1000000;   // scale of an all-zero row
constexpr int kNoExp = -(1 << 30);   // column exponent of an all-zero right-hand side

__host__ __device__ constexpr int n_cores(int ld) { return (ld / 8) * (ld / 8 + 1) / 2; }
// bytes of one digit of one domain: the stored core blocks, 64 bytes each
__host__ __device__ constexpr uint32_t digit_bytes(int ld) { return (uint32_t)n_cores(ld) * 64u; }
__host__ __device__ constexpr uint32_t stage_bytes(int ld) { return (digit_bytes(ld) + 127u) & ~127u; }
// K-major A operand with M = 128 rows read (rows >= ld land in TMEM lanes that are not read)
__host__ __device__ constexpr uint32_t a_bytes(int ld) {
  return ((uint32_t)(ld * ld * 2 - ld * 16 + kM * 16) + 127u) & ~127u;
}
__host__ __device__ constexpr uint32_t b_bytes(int ld) { return (uint32_t)(ld / 8) * 1024u; }
__host__ inline size_t smem_bytes(int ld) {
  return 128 + 2 * (size_t)a_bytes(ld) + kStage * (size_t)stage_bytes(ld) + b_bytes(ld) + (kStage + 3) * 8 + 8 +
         4 * (8 + kGroups * 8 + 64 + 128 + 32);
}

struct Levels {
  const int32_t* coarse[8];
  int64_t vec_off[8];
  int L;
};

// Balanced base-128 digits of x (|x| <= 2^55): x = sum_p d[p] 128^(7-p),
// d[0] the most significant, in [-64, 64]; d[1..7] in [-64, 63].
__device__ __forceinline__ void digits128(long long x, int (&d)[kDigits]) {
#pragma unroll
  for (int p = kDigits - 1; p >= 1; --p) {
    int t = (int)(x & 127);
    if (t >= 64) t -= 128;
    d[p] = t;
    x = (x - t) >> 7;
  }
  d[0] = (int)x;
}

// Build time: scales and digit bytes of the inverses of one level.  One CTA
// per domain, thread i = row i.  Output per domain: kDigits blocks of
// n_cores(ld) core blocks of 64 bytes (core I (I + 1) / 2 + K holds rows
// 8 I .. 8 I + 7, columns 8 K .. 8 K + 7, row-major), and the row scales c_i.
__global__ void k_split_sym(const double* __restrict__ inv, int ld, uint8_t* __restrict__ out,
                            int32_t* __restrict__ cexp) {
  __shared__ int sc[kM];
  const int64_t d = blockIdx.x;
  const int i = threadIdx.x;
  const double* Mi = inv + d * ld * ld + (int64_t)i * ld;
  if (i < ld) {
    int emax = 0;
    for (int k = 0; k < ld; ++k) emax = max(emax, biased_exp(Mi[k]));
    const int c = emax ? (emax - 1022 + 1) >> 1 : kNoScale;  // ceil(e_i / 2), |M_ik| < 2^(emax - 1022)
    sc[i] = c;
    cexp[d * ld + i] = c;
  }
  __syncthreads();
  if (i >= ld) return;
  const int I = i >> 3, row = i & 7;
  uint8_t* base = out + d * kDigits * (int64_t)digit_bytes(ld);
  for (int K = 0; K <= I; ++K) {
    uint32_t w[kDigits][2];  // the row's 8 bytes of every digit
#pragma unroll
    for (int p = 0; p < kDigits; ++p) w[p][0] = w[p][1] = 0;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const int k = 8 * K + c8;
      long long x = 0;
      if (sc[i] != kNoScale && sc[k] != kNoScale) x = scaled_rint(Mi[k], sc[i] + sc[k] + 1);  // rint(M 2^(55-c_i-c_k))
      int dg[kDigits];
      digits128(x, dg);
#pragma unroll
      for (int p = 0; p < kDigits; ++p) w[p][c8 >> 2] |= (uint32_t)(dg[p] + 64) << (8 * (c8 & 3));
    }
    const int64_t core = I * (I + 1) / 2 + K;
#pragma unroll
    for (int p = 0; p < kDigits; ++p)
      *(uint2*)(base + p * (int64_t)digit_bytes(ld) + core * 64 + row * 8) = make_uint2(w[p][0], w[p][1]);
  }
}

// Expansion of one digit matrix by warp W: every stored core block c with
// c % 4 == W, from the staging slot into the BF16 A operand (K-major, core
// (I, K) at (K nb + I) 128 bytes; 8 rows of 16 bytes).
template <int LD, int W>
__device__ __forceinline__ void expand_digit(const unsigned char* __restrict__ stage, unsigned char* __restrict__ A,
                                             int lane) {
  constexpr int nb = LD / 8;
  const unsigned char* src = stage + lane * 2;
  unsigned char* dst = A + lane * 4;
#pragma unroll
  for (int I = 0; I < nb; ++I) {
#pragma unroll
    for (int K = 0; K <= I; ++K) {
      const int c = I * (I + 1) / 2 + K;
      if (c % 4 != W) continue;
      const uint32_t u = *(const uint16_t*)(src + c * 64);  // row lane / 4, columns 2 (lane % 4) + {0, 1}
      const uint32_t v = __byte_perm(u, 0x43434343u, 0x4140);  // two BF16 of value 128 + byte
      *(uint32_t*)(dst + (K * nb + I) * 128) = v;
      if (I != K) *(uint32_t*)(dst + (I * nb + K) * 128) = umma::movmatrix_trans(v);
    }
  }
}

template <int LD>
__device__ __forceinline__ void expand(const unsigned char* stage, unsigned char* A, int warp, int lane) {
  switch (warp) {
    case 0: expand_digit<LD, 0>(stage, A, lane); break;
    case 1: expand_digit<LD, 1>(stage, A, lane); break;
    case 2: expand_digit<LD, 2>(stage, A, lane); break;
    default: expand_digit<LD, 3>(stage, A, lane); break;
  }
}

// kCoarse = false: level 0, CTA = level-0 domain, r gathered through remap0,
//   z = level-0 product + prolongated coarse results, written per node;
// kCoarse = true: one coarse-level domain per CTA (job tables), r and z are the
//   level's contiguous multilevel vectors rl, zl.
template <bool kCoarse, int LD>
__global__ void __launch_bounds__(kThreads) k_f64sym(const uint8_t* const* __restrict__ dig_tab,
                                                     const int32_t* const* __restrict__ scale_tab,
                                                     const int32_t* __restrict__ job_level,
                                                     const int32_t* __restrict__ job_dom,
                                                     const int32_t* __restrict__ remap0, int N, int nrhs, Levels al,
                                                     const double* __restrict__ r, int64_t stride,
                                                     const double* __restrict__ zl, int64_t lstride,
                                                     double* __restrict__ z, int* __restrict__ flags,
                                                     const int* __restrict__ skip) {
  using namespace umma;
  if (skip && *skip) return;  // whole CTA, before any barrier or TMEM use
  extern __shared__ unsigned char smem_raw[];
  constexpr int ld = LD;
  constexpr uint32_t ab = a_bytes(LD), sb = stage_bytes(LD), bb = b_bytes(LD), db = digit_bytes(LD);
  unsigned char* sA = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);  // [2] expanded digit matrices
  unsigned char* stage = sA + 2 * ab;                                              // [kStage] digit bytes
  unsigned char* sB = stage + kStage * sb;                                         // digits of r, N = 64
  uint64_t* full = (uint64_t*)(sB + bb);
  uint64_t* aempty = full + kStage;
  uint64_t* done = aempty + 2;
  uint32_t* tslot = (uint32_t*)(done + 1);
  int* sfail = (int*)(tslot + 1);
  int* sexp = sfail + 1;       // [8] column exponent keys (biased exponent + c_j) of the RHS
  int* ct = sexp + 8;          // bias corrections folded per RHS (16 int64, 8-byte aligned)
  int* csum = ct + kGroups * 8;  // [8 digits][8 RHS] column sums of the digits of r
  int* sc = csum + 64;         // [128] row scales c_i of the domain
  int* snode = sc + kM;        // [32] node of every slot of the domain (-1: padding)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lvl = kCoarse ? job_level[blockIdx.x] : 0;
  const int32_t d = kCoarse ? job_dom[blockIdx.x] : (int32_t)blockIdx.x;
  const uint8_t* dd = dig_tab[lvl] + (int64_t)d * kDigits * db;
  const int64_t cbase = kCoarse ? 3 * (al.vec_off[lvl] + (int64_t)d * N) : 0;  // coarse: first entry of the domain

  if (tid == 0) {
    for (int s = 0; s < kStage; ++s) mbar_init(&full[s], 1);
    mbar_init(&aempty[0], 1);
    mbar_init(&aempty[1], 1);
    mbar_init(done, 1);
    *sfail = 0;
    fence_mbar_init();
  }
  if (tid < 8) sexp[tid] = kNoExp;
  if (tid < 64) csum[tid] = 0;
  sc[tid] = tid < ld ? scale_tab[lvl][(int64_t)d * ld + tid] : kNoScale;
  if (tid < 32) snode[tid] = tid < N ? (kCoarse ? 0 : remap0[(int64_t)d * N + tid]) : -1;
  if (warp == 0) {
    tmem_alloc(tslot, kTmemCols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  int loads[kStage];  // copies issued into each staging slot (thread 0)
  if (tid == 0) {
    for (int p = 0; p < kStage; ++p) {
      mbar_arrive_expect_tx(&full[p], db);
      bulk_g2s(stage + p * sb, dd + (int64_t)p * db, db, &full[p]);
      loads[p] = 1;
    }
  }
  // the epilogue's row: node, scale and the coarse items it prolongates from
  const int i_row = warp * 32 + lane;
  const int32_t node_row = (warp * 32 < ld && i_row < ld) ? snode[i_row / 3] : -1;
  const int ci = i_row < ld ? sc[i_row] : kNoScale;
  int64_t item1 = 0, item2 = 0;
  if (!kCoarse && node_row >= 0) {
    if (al.L > 1) item1 = al.vec_off[1] + al.coarse[1][node_row];
    if (al.L > 2) item2 = al.vec_off[2] + al.coarse[2][node_row];
  }
  // r_d once into registers (entry e = k * ld + j), the column exponent keys
  // of r~ = 2^c_j r by shared-memory atomics, then the digits into B
  constexpr int kPer = 8 * kM / kThreads;
  double rv[kPer];
#pragma unroll
  for (int m = 0; m < kPer; ++m) {
    const int e = tid + m * kThreads;
    const int k = e / ld, j = e - k * ld;
    rv[m] = 0.0;
    if (k < nrhs && k < 8) {
      const int32_t node = snode[j / 3];
      if (kCoarse)
        rv[m] = r[k * lstride + cbase + j];
      else if (node >= 0)
        rv[m] = r[k * stride + 3 * (int64_t)node + j % 3];
      const int eb = biased_exp(rv[m]);  // integer test: no FP64 compare
      if (eb && sc[j] != kNoScale) atomicMax(&sexp[k], eb + sc[j]);
    }
  }
  // TMEM columns 64..79 (groups 8, 9) are first reached by accumulating MMAs
  tmem_zero_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16) + 64u);
  __syncthreads();
  // element (n, j) of B at (j / 8) 1024 + (n / 8) 128 + (n % 8) 16 + (j % 8) 2, n = 8 q + k
#pragma unroll
  for (int m = 0; m < kPer; ++m) {
    const int e = tid + m * kThreads;
    if (e >= 8 * ld) break;
    const int k = e / ld, j = e - k * ld;
    long long y = 0;
    if (sexp[k] != kNoExp && sc[j] != kNoScale) y = scaled_rint(rv[m], sexp[k] - 1021 - sc[j]);
    int dg[kDigits];
    digits128_fast(y, dg);
    unsigned char* col = sB + (j >> 3) * 1024 + (j & 7) * 2 + k * 16;
    // k of the warp's first entry; with ld a multiple of 32 every lane has it
    const int k0 = (e - lane) / ld;
#pragma unroll
    for (int q = 0; q < kDigits; ++q) {
      *(uint16_t*)(col + q * 128) = small_int_bf16_bits(dg[q]);
      // column sums of the digits (bias corrections), a warp reduction per k
      const int v0 = k == k0 ? dg[q] : 0;
      const int r0 = __reduce_add_sync(0xffffffffu, v0);
      if (lane == 0) atomicAdd(&csum[q * 8 + k0], r0);
      if constexpr (LD % 32 != 0) {
        const int r1 = __reduce_add_sync(0xffffffffu, dg[q] - v0);
        if (lane == 0 && k0 + 1 < 8) atomicAdd(&csum[q * 8 + k0 + 1], r1);
      }
    }
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();

  // epilogue operands that do not depend on the MMAs: the prolongated coarse
  // results, loaded now (their items were fetched with r) and summed only in
  // the epilogue, so their latency overlaps the digit loop
  double cs1[8], cs2[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) cs1[k] = cs2[k] = 0.0;
  if (!kCoarse && node_row >= 0) {
    const int c = i_row % 3;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < nrhs) {
        if (al.L > 1) cs1[k] = zl[k * lstride + 3 * item1 + c];
        if (al.L > 2) cs2[k] = zl[k * lstride + 3 * item2 + c];
      }
    for (int l = 3; l < al.L && l < 8; ++l) {  // deeper hierarchies: summed here
      const int64_t item = al.vec_off[l] + al.coarse[l][node_row];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < nrhs) cs2[k] += zl[k * lstride + 3 * item + c];
    }
  }
  // Digit loop: expand digit p into A slot p % 2 (after the MMAs of digit
  // p - 2 have read it), then one thread refills the staging slot with digit
  // p + kStage and issues digit p's MMAs.
  const uint32_t lbo = (uint32_t)ld * 16;
  bool ok = true;
  for (int p = 0; p < kDigits; ++p) {
    const int slot = p % kStage, as = p & 1;
    if (ok) ok = mbar_wait(&full[slot], (uint32_t)(p / kStage) & 1u);
    if (ok && p >= 2) ok = mbar_wait(&aempty[as], (uint32_t)((p - 2) >> 1) & 1u);
    if (ok) expand<LD>(stage + slot * sb, sA + as * ab, warp, lane);
    fence_proxy_async();  // the expanded operand for the tensor core; the staging reads before the refill
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      if (p + kStage < kDigits) {
        mbar_arrive_expect_tx(&full[slot], db);
        bulk_g2s(stage + slot * sb, dd + (int64_t)(p + kStage) * db, db, &full[slot]);
        ++loads[slot];
      }
      fence_after_sync();
      const int qn = min(kDigits, (kGroups - p + 1) & ~1);  // digit columns of r that reach groups <= 9
      const uint32_t idesc = idesc_bf16_f32(kM, 8 * qn);
      const uint64_t da = smem_desc(smem_u32(sA + as * ab), lbo, 128);
      const uint64_t db0 = smem_desc(smem_u32(sB), 1024, 128);
#pragma unroll
      for (int ks = 0; ks < ld / 16; ++ks)
        mma_bf16(tmem + 8u * p, da + ((uint64_t)ks * 2u * lbo >> 4), db0 + ((uint64_t)ks * 2048u >> 4), idesc,
                 (p > 0 || ks > 0) ? 1u : 0u);
      mma_commit(&aempty[as]);
    }
  }
  if (tid == 0) {
    if (!ok) {
      *sfail = 1;
      atomicOr(flags, kErrTimeout);
      for (int s = 0; s < kStage; ++s)  // let the last copy into each slot land before the CTA leaves
        mbar_wait(&full[s], (uint32_t)(loads[s] - 1) & 1u);
    }
    mma_commit(done);  // every MMA issued (none on an early failure) has completed
  }
  // bias corrections, folded per RHS: sum_t 192 (sum over the pair range of t
  // of the digit column sums) 128^(9-t), as hi 2^35 + lo like the products
  long long* cfold = (long long*)ct;  // [0..7] hi part, [8..15] lo part
  if (tid < 8) {
    long long chi = 0, clo = 0;
#pragma unroll
    for (int t = 0; t < kGroups; ++t) {
      int s = 0;
      for (int q = max(0, t - (kDigits - 1)); q <= min(kDigits - 1, t); ++q) s += csum[q * 8 + tid];
      if (t < 5)
        chi = chi * 128 + (long long)kBias * s;
      else
        clo = clo * 128 + (long long)kBias * s;
    }
    cfold[tid] = chi;
    cfold[8 + tid] = clo;
  }
  __syncthreads();
  bool fin = mbar_wait(done, 0);
  if (!fin) atomicOr(flags, kErrTimeout);
  fin = __all_sync(0xffffffffu, fin) && ok && !*sfail;
  fence_after_sync();
  if (fin && warp * 32 < ld) {
    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
    float g[kGroups * 8];  // g[8 t + k]
    tmem_ld_32x32b_x16(ta + 0, g);
    tmem_ld_32x32b_x16(ta + 16, g + 16);
    tmem_ld_32x32b_x16(ta + 32, g + 32);
    tmem_ld_32x32b_x16(ta + 48, g + 48);
    tmem_ld_32x32b_x16(ta + 64, g + 64);
    if (node_row >= 0) {
      const int c = i_row % 3;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k >= nrhs) break;
        double v = 0.0;
        if (sexp[k] != kNoExp && ci != kNoScale) {
          // T = hi 2^35 + lo, hi = sum_{t=0..4} G_t 128^(4-t), lo = sum_{t=5..9} G_t 128^(9-t)
          long long hi = 0, lo = 0;
#pragma unroll
          for (int t = 0; t < 5; ++t) hi = hi * 128 + (long long)__float2int_rn(g[8 * t + k]);
#pragma unroll
          for (int t = 5; t < kGroups; ++t) lo = lo * 128 + (long long)__float2int_rn(g[8 * t + k]);
          hi -= cfold[k];
          lo -= cfold[8 + k];
          const int e = ci + (sexp[k] - 1021) - 76;  // z = T 2^e
          if (e < 900) v = combine_to_double(hi, lo, 35, e);
        }
        if (kCoarse)
          z[k * lstride + cbase + i_row] = v;
        else
          z[k * stride + 3 * (int64_t)node_row + c] = v + (cs1[k] + cs2[k]);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <bool kCoarse>
static int launch(gs_ctx ctx, gs_mas mas, int grid, int nrhs, const int32_t* jl, const int32_t* jd,
                  const double* r, int64_t stride, const double* zl, int64_t lstride, double* z, const int* skip) {
  Levels al{};
  al.L = mas->L;
  for (int l = 0; l < mas->L; ++l) al.coarse[l] = mas->coarse[l], al.vec_off[l] = mas->vec_off[l];
  const auto dt = (const uint8_t* const*)mas->d_sym_tab;
  const auto st = (const int32_t* const*)(mas->d_sym_tab + 8);
  const int ld = 3 * mas->N;
  const size_t smem = smem_bytes(ld);
  if (ld == 96) {
    GS_CUDA(cudaFuncSetAttribute(k_f64sym<kCoarse, 96>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_f64sym<kCoarse, 96><<<grid, kThreads, smem, ctx->stream>>>(dt, st, jl, jd, mas->remap0, mas->N, nrhs, al, r,
                                                                 stride, zl, lstride, z, ctx->d_flags, skip);
  } else {
    GS_CUDA(cudaFuncSetAttribute(k_f64sym<kCoarse, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_f64sym<kCoarse, 48><<<grid, kThreads, smem, ctx->stream>>>(dt, st, jl, jd, mas->remap0, mas->N, nrhs, al, r,
                                                                 stride, zl, lstride, z, ctx->d_flags, skip);
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace f64sym

// 3N = 48 or 96 (N = 16, 32): the expansion is unrolled for those shapes
bool f64sym_shape_ok(int N) { return N == 16 || N == 32; }

int f64sym_prepare(gs_ctx ctx, gs_mas mas) {
  const int ld = 3 * mas->N;
  if (!mas->dig8.empty()) return GS_OK;
  for (int l = 0; l < mas->L; ++l) {  // every level: level 0 and the coarse levels
    const int64_t n_dom = mas->n_domains[l];
    void* dg = nullptr;
    int32_t* ex = nullptr;
    GS_TRY(ctx->alloc(&dg, (size_t)std::max<int64_t>(n_dom, 1) * f64sym::kDigits * f64sym::digit_bytes(ld)));
    mas->dig8.push_back(dg);
    GS_TRY(ctx->alloc((void**)&ex, (size_t)std::max<int64_t>(n_dom, 1) * ld * 4));
    mas->dig8_scale.push_back(ex);
    if (n_dom) {
      GS_PROF(ctx, GS_K_MAS_INVERT);
      f64sym::k_split_sym<<<n_dom, ((ld + 31) / 32) * 32, 0, ctx->stream>>>(mas->inv64[l], ld, (uint8_t*)dg, ex);
    }
  }
  GS_TRY(ctx->alloc((void**)&mas->d_sym_tab, 16 * sizeof(void*)));
  std::vector<void*> hp(16, nullptr);
  for (int l = 0; l < mas->L; ++l) hp[l] = mas->dig8[l], hp[8 + l] = mas->dig8_scale[l];
  GS_CUDA(cudaMemcpyAsync(mas->d_sym_tab, hp.data(), 16 * sizeof(void*), cudaMemcpyHostToDevice, ctx->stream));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

int f64sym_level0_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* r, int64_t stride, const double* zl,
                         int64_t lstride, double* z, const int* skip) {
  if (mas->n_domains[0] == 0) return GS_OK;
  return f64sym::launch<false>(ctx, mas, mas->n_domains[0], nrhs, nullptr, nullptr, r, stride, zl, lstride, z, skip);
}

int f64sym_coarse_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* rl, double* zl, int64_t lstride,
                         const int* skip) {
  if (mas->n_coarse_jobs == 0) return GS_OK;
  return f64sym::launch<true>(ctx, mas, mas->n_coarse_jobs, nrhs, mas->d_coarse_jobs,
                              mas->d_coarse_jobs + mas->n_coarse_jobs, rl, 0, nullptr, lstride, zl, skip);
}

}  // namespace gs
