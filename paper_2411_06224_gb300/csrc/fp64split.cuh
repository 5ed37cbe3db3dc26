// Integer helpers of the FP64-accurate tensor-core products: exponent
// fields, exact scaling of a double to an integer and the rounding of a
// wide integer times a power of two back to a double.  Every step runs on
// the integer units, so no FP64 instruction is spent on the splits.
#pragma once

#include <stdint.h>

namespace gs {

// Biased exponent field of a double (0 for zero / subnormal).
__device__ __forceinline__ int biased_exp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// rint(v * 2^(56 - b)) for |v| < 2^(b-1), in integer arithmetic (round half
// to even), so |result| <= 2^55.
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

// The digits of y (|y| < 2^55) as BF16 bit patterns, written 128 bytes apart
// from col (digit 0, the most significant, first), for the tensor-core
// operand of r.  Balanced digits of y are the plain digits of y + C minus the
// offset, C holding the offset in every digit but the top one, so each digit
// is one bit-field extract; the BF16 of a digit d is the top half of the
// float 1.5 2^23 + d - 1.5 2^23 (exact: d has at most 8 significant bits).
__device__ __forceinline__ uint16_t small_int_bf16_bits(int d) {
  return (uint16_t)(__float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16);
}

// base 256, digits 0..6 (d_0 in [-128, 128], the others in [-128, 127]); an
// eighth, zero digit is written at 7 * 128
__device__ __forceinline__ void write_digits256_bf16(long long y, unsigned char* col) {
  const long long z = y + 0x808080808080LL;  // 128 in digits 1..6
  const uint32_t lo = (uint32_t)z, hi = (uint32_t)((unsigned long long)z >> 32);
  *(uint16_t*)(col + 0 * 128) = small_int_bf16_bits((int)(z >> 48));
  *(uint16_t*)(col + 1 * 128) = small_int_bf16_bits((int)((hi >> 8) & 255u) - 128);
  *(uint16_t*)(col + 2 * 128) = small_int_bf16_bits((int)(hi & 255u) - 128);
  *(uint16_t*)(col + 3 * 128) = small_int_bf16_bits((int)(lo >> 24) - 128);
  *(uint16_t*)(col + 4 * 128) = small_int_bf16_bits((int)((lo >> 16) & 255u) - 128);
  *(uint16_t*)(col + 5 * 128) = small_int_bf16_bits((int)((lo >> 8) & 255u) - 128);
  *(uint16_t*)(col + 6 * 128) = small_int_bf16_bits((int)(lo & 255u) - 128);
  *(uint16_t*)(col + 7 * 128) = 0;
}

// base 128, digits 0..7 (d_0 in [-64, 64], the others in [-64, 63]) into d[]
__device__ __forceinline__ void digits128_fast(long long y, int (&d)[8]) {
  const long long z = y + 0x1020408102040LL;  // 64 in digits 1..7: 64 (128^7 - 1) / 127
  const uint32_t lo = (uint32_t)z, hi = (uint32_t)((unsigned long long)z >> 32);
  d[0] = (int)(z >> 49);
  d[1] = (int)((hi >> 10) & 127u) - 64;
  d[2] = (int)((hi >> 3) & 127u) - 64;
  d[3] = (int)(((hi << 4) | (lo >> 28)) & 127u) - 64;
  d[4] = (int)((lo >> 21) & 127u) - 64;
  d[5] = (int)((lo >> 14) & 127u) - 64;
  d[6] = (int)((lo >> 7) & 127u) - 64;
  d[7] = (int)(lo & 127u) - 64;
}

// (hi 2^S + lo) 2^e as the nearest double (ties to even), |hi|, |lo| < 2^52,
// 24 <= S <= 40, in 64-bit integer arithmetic: the 128-bit sum as two words,
// its magnitude normalised to a leading one in bit 63 of `top`, the bits
// below it OR-ed into a sticky word.  Results below the normal range flush
// to zero.
__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ double combine_to_double(long long hi, long long lo, int S, int e) {
  unsigned long long L0 = (unsigned long long)hi << S;
  long long H = hi >> (64 - S);  // sign-extended high word of hi 2^S
  unsigned long long L = L0 + (unsigned long long)lo;
  H += (lo < 0 ? -1 : 0) + (L < L0 ? 1 : 0);
  unsigned long long sign = 0;
  if (H < 0) {  // magnitude of the 128-bit two's complement value
    sign = 0x8000000000000000ULL;
    L = ~L + 1;
    H = ~H + (L == 0 ? 1 : 0);
  }
  const unsigned long long UH = (unsigned long long)H;
  if (UH == 0 && L == 0) return 0.0;
  int lz;
  unsigned long long top, sticky;
  if (UH) {
    lz = clz64(UH);  // >= 1: |hi 2^S + lo| < 2^127
    top = (UH << lz) | (L >> (64 - lz));
    sticky = L << lz;
  } else {
    const int l = clz64(L);
    lz = 64 + l;
    top = L << l;
    sticky = 0;
  }
  unsigned long long m = top >> 11;  // 53 bits, leading one at bit 52
  const unsigned long long g = top & 0x7FFULL;
  int E = 127 - lz + e;  // value = 1.f 2^E
  if (g > 0x400ULL || (g == 0x400ULL && (sticky != 0 || (m & 1ULL)))) {
    if (++m == (1ULL << 53)) {
      m >>= 1;
      ++E;
    }
  }
  if (E < -1022) return 0.0;
  const unsigned long long bits = sign | ((unsigned long long)(E + 1023) << 52) | (m & 0xFFFFFFFFFFFFFULL);
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double v;
  __builtin_memcpy(&v, &bits, 8);
  return v;
#endif
}

}  // namespace gs
