// Float-float helpers shared by the float-float SpMV (spmv_ff.cu) and the
// PCG direction update that writes its operand (pcg.cu).
#pragma once

#include <cuda_runtime.h>

namespace gs {

// Exponent of an all-zero row or vector: below every real exponent, and the
// word that a memset with bytes 0x80 writes.
constexpr int kExpNone = (int)0x80808080;

// |v| < 2^ex_bound(v) for a double v != 0, from its exponent field
// (subnormals count as below 2^-1022); kExpNone for 0.
__device__ __forceinline__ int ex_bound(double v) {
  const int hi = __double2hiint(v);
  const int e = (hi >> 20) & 0x7ff;
  if (e == 0) return ((hi & 0x7fffffff) | __double2loint(v)) ? -1022 : kExpNone;
  return e - 1022;
}

// 2^e as a double, e clamped to the normal range.
__device__ __forceinline__ double pow2(int e) {
  e = max(-1022, min(1023, e));
  return __hiloint2double((e + 1023) << 20, 0);
}

// (hi, lo) = (rn(w), rn(w - hi)) of w = v 2^e.  The scaling adds e to the
// exponent field (no FP64 instruction); a w below the normal double range,
// and a subnormal v, become 0.  Callers choose e so that |w| <= 1.
__device__ __forceinline__ float2 ff_split_scaled(double v, int e) {
  const int hi = __double2hiint(v);
  const int ef = (hi >> 20) & 0x7ff;
  const int ne = ef + e;
  double w = 0.0;
  if (ef != 0 && ne > 0) w = __hiloint2double(hi + (min(ne, 2046) - ef) * (1 << 20), __double2loint(v));
  const float h = __double2float_rn(w);
  return make_float2(h, __double2float_rn(w - (double)h));
}

// The same split of w = v 2^e without FP64 instructions or conversions (on
// this part both run on the FP64 pipe): hi is w with its mantissa cut to 24
// significant bits, so |w - hi| < 2^-23 |w| and lo has w's sign; lo is the
// remaining 29 bits rounded to 24, made as T - 2^E from bit patterns (T has
// exponent E and those bits as its fraction; the subtraction is exact, and a
// rounding carry moves into T's exponent, which stays exact).  Error:
// |w - hi - lo| <= 2^-47 |w|.  A w below 2^-126 becomes 0, one below 2^-103
// loses lo; callers choose e so that |w| <= 1.
__device__ __forceinline__ float2 ff_split_bits(double v, int e) {
  const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
  const int ef = (int)((hw >> 20) & 0x7ffu);
  const int fe = ef + e - 896;  // float exponent field of w (double bias 1023, float bias 127)
  if (ef == 0 || fe <= 0) return make_float2(0.f, 0.f);
  const unsigned sign = hw & 0x80000000u;
  const unsigned hb = sign | ((unsigned)min(fe, 254) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
  float lo = 0.f;
  const int le = fe - 23;
  if (le > 0) {
    const unsigned base = sign | ((unsigned)le << 23);
    const unsigned r = ((lw & 0x1fffffffu) + 32u) >> 6;  // 29 bits rounded to 23, carry included
    lo = __fsub_rn(__uint_as_float(base + r), __uint_as_float(base));
  }
  return make_float2(__uint_as_float(hb), lo);
}

}  // namespace gs
