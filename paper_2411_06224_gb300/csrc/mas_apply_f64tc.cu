// Level-0 MAS product in FP64 accuracy on the BF16 tensor cores (Eq. 6 at
// level 0), by exact integer splitting of both operands (the Ozaki scheme).
//
// FP64 FMA runs at 2 per clock per SM on this part, so the FP64 dense
// product z_d = M_d^{-1} r_d is bound by the FP64 pipe.  Here both operands
// become sums of small integers times powers of two, every partial product
// is exact in the tensor core's FP32 accumulator, and only a short integer
// combination remains per output:
//   * build time: row i of M_d^{-1} gets an exponent a_i with |M_ik| < 2^(a_i-1);
//     X_ik = rint(M_ik 2^(56-a_i)) (|X| < 2^55) is cut into 7 balanced base-256
//     digits m^(1..7) in [-128, 128] (X = sum_p m^(p) 256^(7-p)), each digit
//     matrix stored as BF16 (exact) in the K-major operand layout;
//   * apply: column k of r_d gets b_k with |r_jk| < 2^(b_k-1), likewise
//     Y_jk = rint(r_jk 2^(56-b_k)) -> digits n^(1..7);
//   * G_s = sum_{p+q=s} m^(p) n^(q) for s = 2..9 (products of digits <= 2^14,
//     96 terms, <= 7 pairs: |G_s| < 2^24, exact in FP32): the B operand holds
//     all 7 digit columns of r (plus a zero one, N = 64), so one MMA per digit
//     matrix and K step writes the groups p+2 .. p+9 into TMEM columns
//     8p .. 8p+63; each G_s collects in its own 8 columns (groups above 9 are
//     not read);
//   * z_ik = 2^(a_i + b_k - 72) sum_{s=2..9} G_s 256^(9-s), combined in
//     64-bit integers (two halves) and rounded once to a double in integer
//     arithmetic, so the epilogue spends one FP64 add (the coarse levels).
// Dropped terms (p + q > 9) and the roundings of X, Y are below 2^-55 of the
// row and column maxima, the level of FP64's own rounding.
//
// One CTA per domain, 128 threads; the 7 digit matrices (18 KB each) stream
// through a shared-memory ring filled by bulk asynchronous copies: 2 slots at
// level 0 (50 KB per CTA, four CTAs share an SM and hide each other's
// latency), 4 for the few coarse-level domains.  All waits are bounded
// (kErrTimeout); TMEM is always freed.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "fp64split.cuh"
#include "umma.cuh"

namespace gs {
namespace f64tc {

constexpr int kDigits = 7;
constexpr int kSlots = 2;        // ring slots of the level-0 kernel (4 CTAs per SM; 3 slots and
                                 // 3 CTAs per SM measured 15 % slower)
constexpr int kSlotsCoarse = 4;  // coarse levels: few CTAs, so a deeper ring per CTA
constexpr int kThreads = 128;
constexpr int kM = 128;
constexpr int kTmemCols = 128;  // groups s = 2..10, 8 columns each (72 used)

struct Levels {
  const int32_t* coarse[8];
  int64_t vec_off[8];
  int L;
};

__host__ __device__ inline uint32_t slot_bytes(int ld) {  // K-major M = 128 span of one digit matrix
  return ((uint32_t)(ld * ld * 2 - ld * 16 + kM * 16) + 127u) & ~127u;
}
__host__ __device__ inline uint32_t b_bytes(int ld) { return (uint32_t)(ld / 8) * 256; }
template <int kS>
__host__ inline size_t smem_bytes(int ld) {
  return 128 + (size_t)kS * slot_bytes(ld) + 4 * (size_t)b_bytes(ld) + (2 * kS + 1) * 8 + 8 + 8 * 4 + 32 * 4;
}

// T 2^e as the nearest double (ties to even), T = hi 2^32 + lo with
// |hi|, |lo| < 2^49.
__device__ __forceinline__ double scaled_to_double(long long hi, long long lo, int e) {
  return combine_to_double(hi, lo, 32, e);
}

// Balanced base-256 digits of x (|x| < 2^55): x = sum_p d[p] 256^(6-p), d[0] the
// most significant; d[1..6] in [-128, 127], |d[0]| <= 128.
__device__ __forceinline__ void digits(long long x, int (&d)[kDigits]) {
#pragma unroll
  for (int p = kDigits - 1; p >= 1; --p) {
    int t = (int)(x & 255);
    if (t >= 128) t -= 256;
    d[p] = t;
    x = (x - t) >> 8;
  }
  d[0] = (int)x;
}

// Build time: digit matrices of the level-0 inverses.  One CTA per domain,
// thread i = row i.  Output per domain: kDigits matrices of ld*ld BF16 in the
// K-major operand layout [k/8][i/8][i%8][k%8], then the row exponents.
__global__ void k_split_inverse(const double* __restrict__ inv, int ld, __nv_bfloat16* __restrict__ out,
                                int32_t* __restrict__ row_exp) {
  const int64_t d = blockIdx.x;
  const int i = threadIdx.x;
  if (i >= ld) return;
  const double* Mi = inv + d * ld * ld + (int64_t)i * ld;
  int emax = 0;
  for (int k = 0; k < ld; ++k) emax = max(emax, biased_exp(Mi[k]));
  const int a = emax - 1021;  // |M_ik| < 2^(emax - 1022) = 2^(a - 1)
  row_exp[d * ld + i] = emax ? a : -100000;
  __nv_bfloat16* base = out + d * kDigits * ld * ld;
  const int groups = ld / 8;
  for (int k = 0; k < ld; ++k) {
    int dg[kDigits];
    digits(emax ? scaled_rint(Mi[k], a) : 0, dg);
    const int64_t pos = (int64_t)(k >> 3) * (groups * 64) + (i >> 3) * 64 + (i & 7) * 8 + (k & 7);
#pragma unroll
    for (int p = 0; p < kDigits; ++p) base[(int64_t)p * ld * ld + pos] = __int2bfloat16_rn(dg[p]);
  }
}


// kCoarse = false: level 0, CTA = level-0 domain, r gathered through remap0,
//   z = level-0 product + prolongated coarse results, written per node;
// kCoarse = true: one coarse-level domain per CTA (job tables), r and z are the
//   level's contiguous multilevel vectors rl, zl.
template <bool kCoarse, int kS, int LD, int kT>
__global__ void __launch_bounds__(kT) k_level0_f64tc(const __nv_bfloat16* const* __restrict__ dig_tab,
                                                           const int32_t* const* __restrict__ exp_tab,
                                                           const int32_t* __restrict__ job_level,
                                                           const int32_t* __restrict__ job_dom,
                                                           const int32_t* __restrict__ remap0, int N, int nrhs,
                                                           Levels al, const double* __restrict__ r, int64_t stride,
                                                           const double* __restrict__ zl, int64_t lstride,
                                                           double* __restrict__ z, int* __restrict__ flags,
                                                           const int* __restrict__ skip) {
  using namespace umma;
  if (skip && *skip) return;  // whole CTA, before any barrier or TMEM use
  extern __shared__ unsigned char smem_raw[];
  constexpr int ld = LD;  // 3 N
  const uint32_t sbytes = slot_bytes(ld), bb = b_bytes(ld);
  const uint32_t dig_bytes = (uint32_t)ld * ld * 2;
  unsigned char* ring = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* sB = ring + kS * sbytes;  // 4 pair operands [n^(2j+1) | n^(2j+2)]
  uint64_t* full = (uint64_t*)(sB + 4 * bb);
  uint64_t* empty = full + kS;
  uint64_t* done = empty + kS;
  uint32_t* tslot = (uint32_t*)(done + 1);
  int* sfail = (int*)(tslot + 1);
  int* sexp = sfail + 1;   // [8] biased exponent maxima of the RHS columns
  int* snode = sexp + 8;   // [32] node of every slot of the domain (-1: padding)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lvl = kCoarse ? job_level[blockIdx.x] : 0;
  const int32_t d = kCoarse ? job_dom[blockIdx.x] : (int32_t)blockIdx.x;
  const __nv_bfloat16* dd = dig_tab[lvl] + (int64_t)d * kDigits * ld * ld;
  const int32_t* row_exp = exp_tab[lvl];
  const int64_t cbase = kCoarse ? 3 * (al.vec_off[lvl] + (int64_t)d * N) : 0;  // coarse: first entry of the domain

  if (tid == 0) {
    for (int s = 0; s < kS; ++s) mbar_init(&full[s], 1), mbar_init(&empty[s], 1);
    mbar_init(done, 1);
    *sfail = 0;
    fence_mbar_init();
  }
  if (tid < 8) sexp[tid] = 0;
  if (tid < 32) snode[tid] = tid < N ? (kCoarse ? 0 : remap0[(int64_t)d * N + tid]) : -1;
  if (warp == 0) {
    tmem_alloc(tslot, kTmemCols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    for (int p = 0; p < kS; ++p) {
      mbar_arrive_expect_tx(&full[p], dig_bytes);
      bulk_g2s(ring + p * sbytes, dd + (int64_t)p * ld * ld, dig_bytes, &full[p]);
    }
  }
  // r_d once into registers (entry e = k * ld + j), column exponents by
  // shared-memory atomics, then the digits into the four pair operands
  constexpr int kPer = 8 * 128 / kT;  // entries per thread for ld <= 128
  double rv[kPer];
#pragma unroll
  for (int m = 0; m < kPer; ++m) {
    const int e = tid + m * kT;
    const int k = e / ld, j = e - k * ld;
    rv[m] = 0.0;
    if (k < nrhs && k < 8) {
      const int32_t node = snode[j / 3];
      if (kCoarse)
        rv[m] = r[k * lstride + cbase + j];
      else if (node >= 0)
        rv[m] = r[k * stride + 3 * (int64_t)node + j % 3];
      const int eb = biased_exp(rv[m]);  // integer test: no FP64 compare
      if (eb) atomicMax(&sexp[k], eb);
    }
  }
  __syncthreads();
  // element (n, kk) of a pair operand at (kk/8)*256 + (n/8)*128 + (n%8)*16 + (kk%8)*2
#pragma unroll
  for (int m = 0; m < kPer; ++m) {
    const int e = tid + m * kT;
    if (e >= 8 * ld) break;
    const int k = e / ld, j = e - k * ld;
    const long long y = scaled_rint(rv[m], sexp[k] - 1021);  // 0 for zero entries
    // column n = 8 q + k; q = 7: the missing 8th digit, zero
    write_digits256_bf16(y, sB + (j >> 3) * 1024 + (j & 7) * 2 + k * 16);
  }
  fence_proxy_async();
  __syncthreads();
  // Epilogue operands that do not depend on the MMAs, loaded now so that their
  // latency overlaps the tensor-core work: row exponent and the prolongated
  // coarse-level sum per RHS.
  // With 256 threads, warps w and w + 4 share TMEM lane quarter w % 4 and
  // take the right-hand sides 0..3 and 4..7 of its rows.
  constexpr int kRpt = 8 * 128 / kT;  // right-hand sides per epilogue thread
  const int q4 = warp & 3, k0 = (warp >> 2) * kRpt;
  const int i_row = q4 * 32 + lane;
  const int32_t node_row = (q4 * 32 < ld && i_row < ld) ? snode[i_row / 3] : -1;
  int a_row = -100000;
  double coarse_sum[kRpt];
#pragma unroll
  for (int k = 0; k < kRpt; ++k) coarse_sum[k] = 0.0;
  if (node_row >= 0) {
    a_row = row_exp[(int64_t)d * ld + i_row];
  }
  if (!kCoarse && node_row >= 0) {
    const int c = i_row % 3;
#pragma unroll
    for (int l = 1; l < 8; ++l) {
      if (l >= al.L) break;
      const int64_t item = al.vec_off[l] + al.coarse[l][node_row];
#pragma unroll
      for (int k = 0; k < kRpt; ++k)
        if (k0 + k < nrhs) {  // the first coarse level assigns: one FP64 add fewer per output
          const double v = zl[(k0 + k) * lstride + 3 * item + c];
          coarse_sum[k] = l == 1 ? v : coarse_sum[k] + v;
        }
    }
  }
  // MMA issue and ring refills (one thread).  A slot is refilled as soon as
  // the MMAs reading it have completed (a wait of a few hundred cycles, while
  // the next digit's copy is still in flight), so two copies stay in flight
  // per CTA.  Descriptors are built once; their 14-bit address fields are
  // advanced by adding byte offsets / 16 (all addresses stay below 256 KB).
  if (tid == 0) {
    bool ok = true;
    int loads[kS];  // copies issued into each slot
    for (int s = 0; s < kS; ++s) loads[s] = 1;
    const uint32_t lbo = (uint32_t)ld * 16;
    const uint32_t idesc = idesc_bf16_f32(kM, 64);
    const uint64_t da0 = smem_desc(smem_u32(ring), lbo, 128);
    const uint64_t db0 = smem_desc(smem_u32(sB), 1024, 128);
    const uint64_t da_ks = (2u * lbo) >> 4, db_ks = 2048u >> 4;
    for (int p = 0; p < kDigits && ok; ++p) {
      const int slot = p % kS;
      if (!mbar_wait(&full[slot], (uint32_t)(p / kS) & 1u)) {
        ok = false;
        break;
      }
      fence_after_sync();
      const uint64_t da = da0 + ((uint64_t)slot * sbytes >> 4);
      // digit p times all digit columns of r: groups s = p + 2 .. p + 9 at TMEM
      // columns 8 p .. 8 p + 63 (group s at column 8 (s - 2))
#pragma unroll 6
      for (int ks = 0; ks < ld / 16; ++ks)
        mma_bf16(tmem + 8u * p, da + ks * da_ks, db0 + ks * db_ks, idesc, (p > 0 || ks > 0) ? 1u : 0u);
      if (p + kS < kDigits) {  // this slot takes digit p + kS once its MMAs are done
        mma_commit(&empty[slot]);
        if (!mbar_wait(&empty[slot], (uint32_t)(p / kS) & 1u)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[slot], dig_bytes);
        bulk_g2s(ring + slot * sbytes, dd + (int64_t)(p + kS) * ld * ld, dig_bytes, &full[slot]);
        ++loads[slot];
      }
    }
    if (ok) {
      mma_commit(done);
    } else {
      *sfail = 1;
      atomicOr(flags, kErrTimeout);
      for (int s = 0; s < kS; ++s)  // let the last copy into each slot land before the CTA leaves
        mbar_wait(&full[s], (uint32_t)(loads[s] - 1) & 1u);
      mbar_arrive(done);
    }
  }
  // warp 0 waits for the MMAs; the other warps wait at the barrier, where they
  // take no issue slots
  if (warp == 0) {
    __syncwarp();
    bool fin = mbar_wait(done, 0);
    if (!fin) atomicOr(flags, kErrTimeout);
    fin = __all_sync(0xffffffffu, fin);
    if (lane == 0 && !fin) *sfail = 1;
  }
  __syncthreads();
  const bool ok = !*sfail;
  fence_after_sync();
  if (ok && q4 * 32 < ld) {
    const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16);
    float g[8 * kRpt];  // groups s = 2..9 of this thread's RHS: g[kRpt (s - 2) + k]
    if constexpr (kRpt == 8) {
      tmem_ld_32x32b_x16(ta + 0, g);
      tmem_ld_32x32b_x16(ta + 16, g + 16);
      tmem_ld_32x32b_x16(ta + 32, g + 32);
      tmem_ld_32x32b_x16(ta + 48, g + 48);
    } else {
#pragma unroll
      for (int s = 0; s < 8; ++s) tmem_ld_32x32b_x4(ta + 8 * s + k0, g + 4 * s);
    }
    const int32_t node = node_row;
    if (node >= 0) {
      const int a = a_row;
      const int c = i_row % 3;
#pragma unroll
      for (int k = 0; k < kRpt; ++k) {
        const int kk = k0 + k;
        if (kk >= nrhs) break;
        double v = 0.0;
        if (sexp[kk] && a > -100000) {
          // T = hi 2^32 + lo, hi = sum_{s=2..5} G_s 256^(5-s), lo = sum_{s=6..9} G_s 256^(9-s)
          long long hi = 0, lo = 0;
#pragma unroll
          for (int s = 0; s < 4; ++s) hi = (hi << 8) + (long long)__float2int_rn(g[kRpt * s + k]);
#pragma unroll
          for (int s = 4; s < 8; ++s) lo = (lo << 8) + (long long)__float2int_rn(g[kRpt * s + k]);
          const int e = a + (sexp[kk] - 1021) - 72;  // z = T 2^e, T = hi 2^32 + lo
          if (e < 900) v = scaled_to_double(hi, lo, e);
        }
        if (kCoarse)
          z[kk * lstride + cbase + i_row] = v;
        else
          z[kk * stride + 3 * (int64_t)node + c] = v + coarse_sum[k];
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


// ---------------------------------------------------------------- persistent form
// One CTA per SM walks domains d = blockIdx.x, + gridDim.x, ...  Warp roles:
//   warp 0 (one lane)  producer: streams the 7 digit matrices of domain after
//                      domain through a kRing-slot shared-memory ring;
//   warp 1 (one lane)  MMA issuer: group sums of domain n into TMEM buffer n%2;
//   warps 2-3          stagers: r of domain n -> column exponents and digits
//                      into B-operand buffer n%2;
//   warps 4-7          epilogue: TMEM lane quarter (warp % 4), rounding to
//                      FP64, prolongated coarse sums, z.
// Barriers (phase parity = use count & 1): ring full/empty per slot, B-buffer
// full/empty (empty needs the MMAs and the epilogue), TMEM full/empty.  Copies,
// MMAs, staging and epilogue of consecutive domains overlap.  Every wait is
// bounded; a timeout sets an abort word that every role checks, so all roles
// leave their loops, wait (bounded) for their asynchronous work and meet at
// the final barrier that precedes the TMEM release.
constexpr int kRing = 10;
constexpr int kPThreads = 256;

// Layout after the 128-byte alignment slack: ring, B buffers [2][4], barriers
// (full, empty [kRing]; bfull, bempty, tfull, tempty [2]; drain), a 64-byte
// word area (TMEM address, abort word), exponents [2][8], node map [2][32].
__host__ inline size_t psmem_bytes(int ld) {
  return 128 + (size_t)kRing * slot_bytes(ld) + 2 * 4 * (size_t)b_bytes(ld) + (2 * kRing + 9) * 8 + 64 + 2 * 8 * 4 +
         2 * 32 * 4;
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads, so
// that a decision to leave a loop is the same in every one of them.
__device__ __forceinline__ bool named_sync_or(int id, int count, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return out != 0;
}

__global__ void __launch_bounds__(kPThreads, 1) k_level0_f64tc_persistent(
    const __nv_bfloat16* __restrict__ dig, const int32_t* __restrict__ row_exp, const int32_t* __restrict__ remap0,
    int32_t n_dom, int N, int nrhs, Levels al, const double* __restrict__ r, int64_t stride,
    const double* __restrict__ zl, int64_t lstride, double* __restrict__ z, int* __restrict__ flags) {
  using namespace umma;
  extern __shared__ unsigned char smem_raw[];
  const int ld = 3 * N;
  const uint32_t sbytes = slot_bytes(ld), bb = b_bytes(ld);
  const uint32_t dig_bytes = (uint32_t)ld * ld * 2;
  unsigned char* ring = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* sBbuf = ring + kRing * sbytes;  // [2][4 pair operands]
  uint64_t* full = (uint64_t*)(sBbuf + 2 * 4 * bb);
  uint64_t* empty = full + kRing;
  uint64_t* bfull = empty + kRing;  // [2]
  uint64_t* bempty = bfull + 2;     // [2]
  uint64_t* tfull = bempty + 2;     // [2]
  uint64_t* tempty = tfull + 2;     // [2]
  uint64_t* drain = tempty + 2;     // [1]
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort_word = (volatile int*)(tslot + 1);
  int* sexp = (int*)(tslot + 16);  // [2][8]
  int* snode = sexp + 16;          // [2][32]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_local = n_dom > (int)blockIdx.x ? (n_dom - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int s = 0; s < kRing; ++s) mbar_init(&full[s], 1), mbar_init(&empty[s], 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bfull[b], 1);
      mbar_init(&bempty[b], 2);  // the MMAs (commit) and the epilogue
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 1);
    }
    mbar_init(drain, 1);
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 256);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int seq = 0;
      for (int n = 0; n < n_local && !*abort_word; ++n) {
        const __nv_bfloat16* dd = dig + (int64_t)(blockIdx.x + (int64_t)n * gridDim.x) * kDigits * ld * ld;
        for (int p = 0; p < kDigits; ++p) {
          const int slot = seq % kRing, use = seq / kRing;
          if (use > 0 && !mbar_wait(&empty[slot], (uint32_t)(use - 1) & 1u)) {
            *abort_word = 1;
            atomicOr(flags, kErrTimeout);
          }
          if (*abort_word) break;
          mbar_arrive_expect_tx(&full[slot], dig_bytes);
          bulk_g2s(ring + slot * sbytes, dd + (int64_t)p * ld * ld, dig_bytes, &full[slot]);
          ++seq;
        }
      }
      // every copy issued lands before the CTA can leave (the last use of each slot)
      for (int s = 0; s < kRing && s < seq; ++s) mbar_wait(&full[s], (uint32_t)((seq - 1 - s) / kRing) & 1u);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t lbo = (uint32_t)ld * 16;
      const uint32_t idesc = idesc_bf16_f32(kM, 64);
      const uint64_t da0 = smem_desc(smem_u32(ring), lbo, 128);
      const uint64_t db0 = smem_desc(smem_u32(sBbuf), 1024, 128);
      const uint64_t da_ks = (2u * lbo) >> 4, db_ks = 2048u >> 4, db_buf = (4u * bb) >> 4;
      int seq = 0;
      bool issued = false;
      for (int n = 0; n < n_local && !*abort_word; ++n) {
        const int b = n & 1, use = n >> 1;
        bool ok = (use == 0 || mbar_wait(&tempty[b], (uint32_t)(use - 1) & 1u)) &&
                  mbar_wait(&bfull[b], (uint32_t)use & 1u);
        if (ok) {
          fence_after_sync();
          const uint32_t tbase = tmem + 128u * b;
          for (int p = 0; p < kDigits && ok; ++p, ++seq) {
            const int slot = seq % kRing;
            if (!mbar_wait(&full[slot], (uint32_t)(seq / kRing) & 1u)) {
              ok = false;
              break;
            }
            fence_after_sync();
            const uint64_t da = da0 + ((uint64_t)slot * sbytes >> 4);
            const uint64_t db = db0 + b * db_buf;
#pragma unroll 6
            for (int ks = 0; ks < ld / 16; ++ks)
              mma_bf16(tbase + 8u * p, da + ks * da_ks, db + ks * db_ks, idesc, (p > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&empty[slot]);
            issued = true;
          }
        }
        if (!ok) {
          *abort_word = 1;
          atomicOr(flags, kErrTimeout);
          break;
        }
        mma_commit(&tfull[b]);
        mma_commit(&bempty[b]);
      }
      if (issued) {  // every MMA issued finishes before TMEM can be released
        mma_commit(drain);
        mbar_wait(drain, 0);
      }
    }
  } else if (warp < 4) {
    // ------------------------------------------------------------ stagers (64 threads)
    const int st = tid - 64;
    for (int n = 0; n < n_local; ++n) {
      const int b = n & 1, use = n >> 1;
      const int32_t d = blockIdx.x + n * gridDim.x;
      bool bad = *abort_word != 0;
      if (!bad && use > 0 && !mbar_wait(&bempty[b], (uint32_t)(use - 1) & 1u)) {
        bad = true;
        *abort_word = 1;
        atomicOr(flags, kErrTimeout);
      }
      if (named_sync_or(1, 64, bad)) break;
      int* se = sexp + 8 * b;
      int* sn = snode + 32 * b;
      if (st < 8) se[st] = 0;
      if (st < 32) sn[st] = st < N ? remap0[(int64_t)d * N + st] : -1;
      named_sync(1, 64);
      constexpr int kSPer = 8 * 128 / 64;
      double rv[kSPer];
#pragma unroll
      for (int m = 0; m < kSPer; ++m) {
        const int e = st + m * 64;
        const int k = e / ld, j = e - k * ld;
        rv[m] = 0.0;
        if (k < nrhs && k < 8) {
          const int32_t node = sn[j / 3];
          if (node >= 0) rv[m] = r[k * stride + 3 * (int64_t)node + j % 3];
          const int eb = biased_exp(rv[m]);
          if (eb) atomicMax(&se[k], eb);
        }
      }
      named_sync(1, 64);
      unsigned char* sB = sBbuf + b * 4 * bb;
#pragma unroll
      for (int m = 0; m < kSPer; ++m) {
        const int e = st + m * 64;
        if (e >= 8 * ld) break;
        const int k = e / ld, j = e - k * ld;
        const long long y = scaled_rint(rv[m], se[k] - 1021);
        write_digits256_bf16(y, sB + (j >> 3) * 1024 + (j & 7) * 2 + k * 16);
      }
      fence_proxy_async();
      named_sync(1, 64);
      if (st == 0) mbar_arrive(&bfull[b]);
    }
  } else {
    // ------------------------------------------------------------ epilogue (128 threads)
    const int q4 = warp & 3;  // TMEM lane quarter
    const int i_row = q4 * 32 + lane;
    for (int n = 0; n < n_local; ++n) {
      const int b = n & 1, use = n >> 1;
      const int32_t d = blockIdx.x + n * gridDim.x;
      bool bad = *abort_word != 0;
      if (!bad && !mbar_wait(&bfull[b], (uint32_t)use & 1u)) {  // this domain's node map and exponents
        bad = true;
        *abort_word = 1;
        atomicOr(flags, kErrTimeout);
      }
      if (named_sync_or(2, 128, bad)) break;
      const int* se = sexp + 8 * b;
      const int32_t node = i_row < ld ? snode[32 * b + i_row / 3] : -1;
      int a = -100000;
      double coarse_sum[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) coarse_sum[k] = 0.0;
      const int c = i_row % 3;
      if (node >= 0) {
        a = row_exp[(int64_t)d * ld + i_row];
#pragma unroll
        for (int l = 1; l < 8; ++l) {
          if (l >= al.L) break;
          const int64_t item = al.vec_off[l] + al.coarse[l][node];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (k < nrhs) {  // the first coarse level assigns: one FP64 add fewer per output
          const double v = zl[k * lstride + 3 * item + c];
          coarse_sum[k] = l == 1 ? v : coarse_sum[k] + v;
        }
        }
      }
      bad = !mbar_wait(&tfull[b], (uint32_t)use & 1u);
      if (bad) {
        *abort_word = 1;
        atomicOr(flags, kErrTimeout);
      }
      if (named_sync_or(2, 128, bad)) break;
      fence_after_sync();
      if (q4 * 32 < ld) {
        const uint32_t ta = tmem + 128u * b + ((uint32_t)(q4 * 32) << 16);
        float g[64];
        tmem_ld_32x32b_x16(ta + 0, g);
        tmem_ld_32x32b_x16(ta + 16, g + 16);
        tmem_ld_32x32b_x16(ta + 32, g + 32);
        tmem_ld_32x32b_x16(ta + 48, g + 48);
        if (node >= 0) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            if (k >= nrhs) break;
            double v = 0.0;
            if (se[k] && a > -100000) {
              long long hi = 0, lo = 0;
#pragma unroll
              for (int s = 0; s < 4; ++s) hi = (hi << 8) + (long long)__float2int_rn(g[8 * s + k]);
#pragma unroll
              for (int s = 4; s < 8; ++s) lo = (lo << 8) + (long long)__float2int_rn(g[8 * s + k]);
              const int e = a + (se[k] - 1021) - 72;
              if (e < 900) v = scaled_to_double(hi, lo, e);
            }
            z[k * stride + 3 * (int64_t)node + c] = v + coarse_sum[k];
          }
        }
      }
      fence_before_sync();
      named_sync(2, 128);
      if (tid == 128) {
        mbar_arrive(&tempty[b]);
        mbar_arrive(&bempty[b]);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, 256);
  }
}

}  // namespace f64tc

// GS_TUNE_F64_TC: 1 / 2 / 4 stream the BF16 digit matrices of this file, 3 the
// symmetric digit bytes of mas_apply_f64sym.cu; the storage is made when the
// preconditioner is built for the value set then.
bool level0_f64tc_usable(gs_ctx ctx, gs_mas mas, int nrhs) {
  if (mas->precision != GS_PREC_FP64 || nrhs < 1 || nrhs > 8) return false;
  const int t = ctx->tune[GS_TUNE_F64_TC];
  if (t == 3) return !mas->dig8.empty();
  return (t == 1 || t == 2 || t == 4) && !mas->dig64.empty();
}

int level0_f64tc_prepare(gs_ctx ctx, gs_mas mas) {
  const int ld = 3 * mas->N;
  const int t = ctx->tune[GS_TUNE_F64_TC];
  if (mas->precision != GS_PREC_FP64 || t == 0) return GS_OK;
  if (t == 3) return f64sym_shape_ok(mas->N) ? f64sym_prepare(ctx, mas) : GS_OK;  // 1, 2, 4: BF16 digits
  if (ld % 16 != 0 || ld > f64tc::kM || !mas->dig64.empty()) return GS_OK;
  for (int l = 0; l < mas->L; ++l) {  // every level: level 0 and the coarse levels
    const int64_t n_dom = mas->n_domains[l];
    void* dg = nullptr;
    int32_t* ex = nullptr;
    GS_TRY(ctx->alloc(&dg, (size_t)std::max<int64_t>(n_dom, 1) * f64tc::kDigits * ld * ld * 2));
    mas->dig64.push_back(dg);
    GS_TRY(ctx->alloc((void**)&ex, (size_t)std::max<int64_t>(n_dom, 1) * ld * 4));
    mas->dig64_exp.push_back(ex);
    if (n_dom) {
      GS_PROF(ctx, GS_K_MAS_INVERT);
      f64tc::k_split_inverse<<<n_dom, ((ld + 31) / 32) * 32, 0, ctx->stream>>>(mas->inv64[l], ld,
                                                                               (__nv_bfloat16*)dg, ex);
    }
  }
  GS_TRY(ctx->alloc((void**)&mas->d_dig_tab, 16 * sizeof(void*)));
  std::vector<void*> hp(16, nullptr);
  for (int l = 0; l < mas->L; ++l) hp[l] = mas->dig64[l], hp[8 + l] = mas->dig64_exp[l];
  GS_CUDA(cudaMemcpyAsync(mas->d_dig_tab, hp.data(), 16 * sizeof(void*), cudaMemcpyHostToDevice, ctx->stream));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

static f64tc::Levels f64tc_levels(gs_mas mas) {
  f64tc::Levels al{};
  al.L = mas->L;
  for (int l = 0; l < mas->L; ++l) al.coarse[l] = mas->coarse[l], al.vec_off[l] = mas->vec_off[l];
  return al;
}

int level0_f64tc_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* r, int64_t stride, const double* zl,
                        int64_t lstride, double* z, const int* skip) {
  GS_CHECK(level0_f64tc_usable(ctx, mas, nrhs), GS_ERR_UNSUPPORTED, "FP64 tensor-core apply: not available");
  if (ctx->tune[GS_TUNE_F64_TC] == 3) return f64sym_level0_launch(ctx, mas, nrhs, r, stride, zl, lstride, z, skip);
  if (mas->n_domains[0] == 0) return GS_OK;
  if (ctx->tune[GS_TUNE_F64_TC] == 2) {  // persistent, warp-specialised: one CTA per SM
    const size_t psmem = f64tc::psmem_bytes(3 * mas->N);
    GS_CUDA(cudaFuncSetAttribute(f64tc::k_level0_f64tc_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)psmem));
    const int grid = std::min<int>(mas->n_domains[0], std::max(ctx->sm_count, 1));
    f64tc::k_level0_f64tc_persistent<<<grid, f64tc::kPThreads, psmem, ctx->stream>>>(
        (const __nv_bfloat16*)mas->dig64[0], mas->dig64_exp[0], mas->remap0, mas->n_domains[0], mas->N, nrhs,
        f64tc_levels(mas), r, stride, zl, lstride, z, ctx->d_flags);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  }
  const auto tabs = (const __nv_bfloat16* const*)mas->d_dig_tab;
  const auto etabs = (const int32_t* const*)(mas->d_dig_tab + 8);
  const size_t smem = f64tc::smem_bytes<f64tc::kSlots>(3 * mas->N);
  // 3 N = 96 or 48 (the digit storage is made only for N = 32 and 16)
#define GS_F64TC_L0(LD, T)                                                                                     \
  GS_CUDA(cudaFuncSetAttribute(f64tc::k_level0_f64tc<false, f64tc::kSlots, LD, T>,                             \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));                       \
  f64tc::k_level0_f64tc<false, f64tc::kSlots, LD, T><<<mas->n_domains[0], T, smem, ctx->stream>>>(              \
      tabs, etabs, nullptr, nullptr, mas->remap0, mas->N, nrhs, f64tc_levels(mas), r, stride, zl, lstride, z,   \
      ctx->d_flags, skip)
  const bool wide = ctx->tune[GS_TUNE_F64_TC] == 4;  // 256 threads per domain
  if (mas->N == 32) {
    if (wide) {
      GS_F64TC_L0(96, 256);
    } else {
      GS_F64TC_L0(96, 128);
    }
  } else {
    if (wide) {
      GS_F64TC_L0(48, 256);
    } else {
      GS_F64TC_L0(48, 128);
    }
  }
#undef GS_F64TC_L0
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

int coarse_f64tc_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* rl, double* zl, int64_t lstride,
                        const int* skip) {
  GS_CHECK(level0_f64tc_usable(ctx, mas, nrhs), GS_ERR_UNSUPPORTED, "FP64 tensor-core apply: not available");
  if (ctx->tune[GS_TUNE_F64_TC] == 3) return f64sym_coarse_launch(ctx, mas, nrhs, rl, zl, lstride, skip);
  if (mas->n_coarse_jobs == 0) return GS_OK;
  // a few hundred coarse domains at most: a deeper ring per CTA shortens the
  // chain of copy latencies that bounds this small launch
  const size_t smem = f64tc::smem_bytes<f64tc::kSlotsCoarse>(3 * mas->N);
  const auto tabs = (const __nv_bfloat16* const*)mas->d_dig_tab;
  const auto etabs = (const int32_t* const*)(mas->d_dig_tab + 8);
#define GS_F64TC_CO(LD, T)                                                                                       \
  GS_CUDA(cudaFuncSetAttribute(f64tc::k_level0_f64tc<true, f64tc::kSlotsCoarse, LD, T>,                          \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));                         \
  f64tc::k_level0_f64tc<true, f64tc::kSlotsCoarse, LD, T><<<mas->n_coarse_jobs, T, smem, ctx->stream>>>(         \
      tabs, etabs, mas->d_coarse_jobs, mas->d_coarse_jobs + mas->n_coarse_jobs, nullptr, mas->N, nrhs,             \
      f64tc_levels(mas), rl, 0, nullptr, lstride, zl, ctx->d_flags, skip)
  const bool wide = ctx->tune[GS_TUNE_F64_TC] == 4;  // 256 threads per domain
  if (mas->N == 32) {
    if (wide) {
      GS_F64TC_CO(96, 256);
    } else {
      GS_F64TC_CO(96, 128);
    }
  } else {
    if (wide) {
      GS_F64TC_CO(48, 256);
    } else {
      GS_F64TC_CO(48, 128);
    }
  }
#undef GS_F64TC_CO
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs
