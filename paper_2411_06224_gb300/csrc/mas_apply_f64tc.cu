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
//     96 terms, <= 7 pairs: |G_s| < 2^24, exact in FP32): the tensor core
//     accumulates each G_s in its own 8 TMEM columns, one MMA per (digit p,
//     pair of digits q, q+1) with N = 16;
//   * z_ik = 2^(a_i + b_k - 72) sum_{s=2..9} G_s 256^(9-s), combined in
//     64-bit integers (two halves) and converted once.
// Dropped terms (p + q > 9) and the roundings of X, Y are below 2^-55 of the
// row and column maxima, the level of FP64's own rounding.
//
// One CTA per domain, 128 threads; the 7 digit matrices (18 KB each) stream
// through a 4-slot shared-memory ring filled by bulk asynchronous copies, so
// two CTAs fit on an SM and one's epilogue overlaps the other's copies.  All
// waits are bounded (kErrTimeout); TMEM is always freed.
#include <cuda_bf16.h>

#include "common.cuh"
#include "umma.cuh"

namespace gs {
namespace f64tc {

constexpr int kDigits = 7;
constexpr int kSlots = 4;
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
__host__ inline size_t smem_bytes(int ld) {
  return 128 + (size_t)kSlots * slot_bytes(ld) + 4 * (size_t)b_bytes(ld) + (2 * kSlots + 1) * 8 + 8 + 8 * 4;
}

// 2^e as a double for e in the normal range (bit construction).
__device__ __forceinline__ double pow2(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// Biased exponent field of a double (0 for zero / subnormal).
__device__ __forceinline__ int biased_exp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// rint(v * 2^(56 - b)) for |v| < 2^(b-1), in integer arithmetic (round half
// to even), so no FP64 instruction is spent on the split.
__device__ __forceinline__ long long scaled_rint(double v, int b) {
  const long long bits = __double_as_longlong(v);
  const int eb = (int)((bits >> 52) & 0x7FF);
  if (eb == 0) return 0;  // zero or subnormal: far below the column scale
  const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;  // 53 bits
  const int sh = eb - 1075 + 56 - b;  // value = mant 2^(eb - 1075); times 2^(56 - b)
  long long q;
  if (sh >= 0) {
    q = mant << sh;  // sh <= 2 by the bound on |v|
  } else {
    const int s = -sh;
    if (s > 54) return 0;
    const long long half = 1LL << (s - 1);
    q = mant >> s;
    const long long rem = mant & ((1LL << s) - 1);
    q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
  }
  return bits < 0 ? -q : q;
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

// digit p (0-based) times digit pair j -> TMEM column 8 * (p + 2 j): the
// groups s = p + 2j + 2 and s + 1 (1-based digits p+1 and 2j+1, 2j+2)
__device__ __forceinline__ int pairs_for(int p) { return (8 - (p + 1)) / 2 + 1; }

__global__ void __launch_bounds__(kThreads) k_level0_f64tc(const __nv_bfloat16* __restrict__ dig,
                                                           const int32_t* __restrict__ row_exp,
                                                           const int32_t* __restrict__ remap0, int N, int nrhs,
                                                           Levels al, const double* __restrict__ r, int64_t stride,
                                                           const double* __restrict__ zl, int64_t lstride,
                                                           double* __restrict__ z, int* __restrict__ flags) {
  using namespace umma;
  extern __shared__ unsigned char smem_raw[];
  const int ld = 3 * N;
  const uint32_t sbytes = slot_bytes(ld), bb = b_bytes(ld);
  const uint32_t dig_bytes = (uint32_t)ld * ld * 2;
  unsigned char* ring = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* sB = ring + kSlots * sbytes;  // 4 pair operands [n^(2j+1) | n^(2j+2)]
  uint64_t* full = (uint64_t*)(sB + 4 * bb);
  uint64_t* empty = full + kSlots;
  uint64_t* done = empty + kSlots;
  uint32_t* tslot = (uint32_t*)(done + 1);
  int* sfail = (int*)(tslot + 1);
  int* sexp = sfail + 1;  // [8] biased exponent maxima of the RHS columns
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t d = blockIdx.x;
  const __nv_bfloat16* dd = dig + (int64_t)d * kDigits * ld * ld;

  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) mbar_init(&full[s], 1), mbar_init(&empty[s], 1);
    mbar_init(done, 1);
    *sfail = 0;
    fence_mbar_init();
  }
  if (tid < 8) sexp[tid] = 0;
  if (warp == 0) {
    tmem_alloc(tslot, kTmemCols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  if (tid == 0)
    for (int p = 0; p < kSlots; ++p) {
      mbar_arrive_expect_tx(&full[p], dig_bytes);
      bulk_g2s(ring + p * sbytes, dd + (int64_t)p * ld * ld, dig_bytes, &full[p]);
    }
  // column exponents of r_d (RHS k < 8; columns >= nrhs stay 0)
  const int nv = ld * 8;
  for (int e = tid; e < nv; e += kThreads) {
    const int k = e / ld, j = e - k * ld;
    if (k >= nrhs) continue;
    const int32_t node = remap0[(int64_t)d * N + j / 3];
    if (node >= 0) atomicMax(&sexp[k], biased_exp(r[k * stride + 3 * (int64_t)node + j % 3]));
  }
  __syncthreads();
  // digits of r_d into the four pair operands; element (n, kk) of a pair
  // operand at (kk/8)*256 + (n/8)*128 + (n%8)*16 + (kk%8)*2
  for (int e = tid; e < nv; e += kThreads) {
    const int k = e / ld, j = e - k * ld;
    long long y = 0;
    if (k < nrhs && sexp[k]) {
      const int32_t node = remap0[(int64_t)d * N + j / 3];
      if (node >= 0) y = scaled_rint(r[k * stride + 3 * (int64_t)node + j % 3], sexp[k] - 1021);
    }
    int dg[kDigits];
    digits(y, dg);
    unsigned char* col = sB + (j >> 3) * 256 + (j & 7) * 2 + k * 16;
#pragma unroll
    for (int q = 0; q < 8; ++q)  // q = 7: the missing 8th digit, zero
      *(__nv_bfloat16*)(col + (q >> 1) * bb + (q & 1) * 128) = __int2bfloat16_rn(q < kDigits ? dg[q] : 0);
  }
  fence_proxy_async();
  __syncthreads();
  // MMA issue and ring refills (one thread).  A slot is refilled one digit
  // later than its MMAs were issued, so the tensor core is not waited on.
  if (tid == 0) {
    bool ok = true;
    int refilled = 0;  // bit s: slot s holds a second digit matrix
    const uint32_t lbo = (uint32_t)ld * 16;
    const uint32_t idesc = idesc_bf16_f32(kM, 16);
    const uint32_t b0 = smem_u32(sB);
    for (int p = 0; p < kDigits && ok; ++p) {
      const int slot = p % kSlots;
      if (!mbar_wait(&full[slot], (uint32_t)(p / kSlots) & 1u)) {
        ok = false;
        break;
      }
      fence_after_sync();
      const uint32_t a0 = smem_u32(ring + slot * sbytes);
      for (int j = 0; j < pairs_for(p); ++j)
        for (int ks = 0; ks < ld / 16; ++ks)
          mma_bf16(tmem + 8u * (p + 2 * j), smem_desc(a0 + 2u * ks * lbo, lbo, 128),
                   smem_desc(b0 + j * bb + 512u * ks, 256, 128), idesc, (p > 0 || ks > 0) ? 1u : 0u);
      mma_commit(&empty[slot]);
      const int q = p - 1;  // the previous digit's slot takes digit q + kSlots
      if (q >= 0 && q + kSlots < kDigits) {
        const int qs = q % kSlots;
        if (!mbar_wait(&empty[qs], 0)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[qs], dig_bytes);
        bulk_g2s(ring + qs * sbytes, dd + (int64_t)(q + kSlots) * ld * ld, dig_bytes, &full[qs]);
        refilled |= 1 << qs;
      }
    }
    if (ok) {
      mma_commit(done);
    } else {
      *sfail = 1;
      atomicOr(flags, kErrTimeout);
      for (int s = 0; s < kSlots; ++s) {  // let copies in flight land before the CTA leaves
        mbar_wait(&full[s], 0);
        if (refilled & (1 << s)) mbar_wait(&full[s], 1);
      }
      mbar_arrive(done);
    }
  }
  __syncwarp();
  bool ok = mbar_wait(done, 0);
  if (!ok) atomicOr(flags, kErrTimeout);
  ok = __all_sync(0xffffffffu, ok) && !*sfail;
  fence_after_sync();
  if (ok && warp * 32 < ld) {
    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
    float g[64];  // groups s = 2..9, 8 RHS each: g[8 (s - 2) + k]
    tmem_ld_32x32b_x16(ta + 0, g);
    tmem_ld_32x32b_x16(ta + 16, g + 16);
    tmem_ld_32x32b_x16(ta + 32, g + 32);
    tmem_ld_32x32b_x16(ta + 48, g + 48);
    const int i = warp * 32 + lane;
    const int32_t node = i < ld ? remap0[(int64_t)d * N + i / 3] : -1;
    if (node >= 0) {
      const int a = row_exp[(int64_t)d * ld + i];
      const int c = i % 3;
      int64_t citem[8];
#pragma unroll
      for (int l = 1; l < 8; ++l) citem[l] = l < al.L ? al.vec_off[l] + al.coarse[l][node] : 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k >= nrhs) break;
        double v = 0.0;
        if (sexp[k] && a > -100000) {
          // T = hi 2^32 + lo, hi = sum_{s=2..5} G_s 256^(5-s), lo = sum_{s=6..9} G_s 256^(9-s)
          long long hi = 0, lo = 0;
#pragma unroll
          for (int s = 0; s < 4; ++s) hi = (hi << 8) + (long long)__float2int_rn(g[8 * s + k]);
#pragma unroll
          for (int s = 4; s < 8; ++s) lo = (lo << 8) + (long long)__float2int_rn(g[8 * s + k]);
          const int e = a + (sexp[k] - 1021) - 72;  // z = T 2^e
          if (e > -1000 && e < 900)                    // outside: |z| underflows (or overflows) FP64
            v = fma((double)hi, pow2(e + 32), (double)lo * pow2(e));
        }
#pragma unroll
        for (int l = 1; l < 8; ++l)
          if (l < al.L) v += zl[k * lstride + 3 * citem[l] + c];
        z[k * stride + 3 * (int64_t)node + c] = v;
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

}  // namespace f64tc

bool level0_f64tc_usable(gs_ctx ctx, gs_mas mas, int nrhs) {
  return mas->precision == GS_PREC_FP64 && mas->dig64 != nullptr && nrhs >= 1 && nrhs <= 8 &&
         ctx->tune[GS_TUNE_F64_TC] != 0;
}

int level0_f64tc_prepare(gs_ctx ctx, gs_mas mas) {
  const int ld = 3 * mas->N;
  if (mas->precision != GS_PREC_FP64 || ld % 16 != 0 || ld > f64tc::kM || mas->dig64) return GS_OK;
  const int64_t n_dom = mas->n_domains[0];
  GS_TRY(ctx->alloc(&mas->dig64, (size_t)std::max<int64_t>(n_dom, 1) * f64tc::kDigits * ld * ld * 2));
  GS_TRY(ctx->alloc((void**)&mas->dig64_exp, (size_t)std::max<int64_t>(n_dom, 1) * ld * 4));
  if (n_dom) {
    GS_PROF(ctx, GS_K_MAS_INVERT);
    f64tc::k_split_inverse<<<n_dom, ((ld + 31) / 32) * 32, 0, ctx->stream>>>(
        mas->inv64[0], ld, (__nv_bfloat16*)mas->dig64, mas->dig64_exp);
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

int level0_f64tc_launch(gs_ctx ctx, gs_mas mas, int nrhs, const double* r, int64_t stride, const double* zl,
                        int64_t lstride, double* z) {
  GS_CHECK(level0_f64tc_usable(ctx, mas, nrhs), GS_ERR_UNSUPPORTED, "FP64 tensor-core apply: not available");
  if (mas->n_domains[0] == 0) return GS_OK;
  const int ld = 3 * mas->N;
  f64tc::Levels al{};
  al.L = mas->L;
  for (int l = 0; l < mas->L; ++l) al.coarse[l] = mas->coarse[l], al.vec_off[l] = mas->vec_off[l];
  const size_t smem = f64tc::smem_bytes(ld);
  GS_CUDA(cudaFuncSetAttribute(f64tc::k_level0_f64tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  f64tc::k_level0_f64tc<<<mas->n_domains[0], f64tc::kThreads, smem, ctx->stream>>>(
      (const __nv_bfloat16*)mas->dig64, mas->dig64_exp, mas->remap0, mas->N, nrhs, al, r, stride, zl, lstride, z,
      ctx->d_flags);
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs
