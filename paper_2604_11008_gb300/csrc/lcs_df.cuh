// Float-float ("double-float") arithmetic for the FP64 step on GB300.
//
// GB300 issues FP64 instructions (DFMA, DADD, DMUL and the f32<->f64
// conversions) at roughly 1/70 of the FP32 rate, so a plain FP64 step is
// bound by the FP64 pipe far below the memory roofline.  The DF step keeps
// positions in int64 fixed point (52 fraction bits, grid-cell units) and
// velocities as float pairs in its record buffers, and evaluates the
// interpolation and the Heun increments with unevaluated sums of two floats
// (h + l, about 48 significant bits) built from error-free transformations:
//   two_sum (Knuth 1969), fast_two_sum (Dekker 1971), and the exact product
// error fma(a, b, -a*b) (the FMA-based variant of Dekker's TwoProduct).
// Position increments are added exactly in fixed point.  Conversions between
// double and float pairs use integer bit operations, not the FP64 pipe; the
// only FP64-pipe instructions on the Stokes path are the float -> int64
// conversions of the fixed-point increments.  FP64 values appear only at the
// boundary (import of the initial state, export of the state).
#pragma once

#include <cstdint>

namespace lcs {

struct df {
  float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// Multiplication by a power of two is exact.
__device__ __forceinline__ df df_scale2(df a, float p2) { return {a.h * p2, a.l * p2}; }

// 1/a with one Newton step in float-float (relative error ~2^-46).
__device__ __forceinline__ df df_recip(df a) {
  const float r = __frcp_rn(a.h);
  const float p = __fmul_rn(a.h, r);
  const float pe = __fmaf_rn(a.h, r, -p);           // a.h * r = p + pe exactly
  // e = 1 - a*r = (1 - p) - pe - a.l*r ; 1 - p is exact (p close to 1)
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(a.l, r));
  return fast_two_sum(r, __fmul_rn(r, e));
}

// Split an FP64 value into a float pair by bit operations (no FP64 pipe):
// hi = the leading 24 significand bits (truncated), lo = the next 23 bits.
// |x - (hi + lo)| <= 2^-47 |x|.  Magnitudes below 2^-60 give (0, 0); the
// result is meaningless for non-finite x (callers check the FP64 results).
__device__ __forceinline__ df split_d(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned sign = hi & 0x80000000u;
  const bool ok = e >= 1023 - 60 && e <= 1023 + 100;
  const unsigned hbits = sign | ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned r23 = (lo & 0x1fffffffu) >> 6;
  const float r = __fsub_rn(__uint_as_float(0x4B000000u | r23), 8388608.0f);  // exact integer
  const float scale = __uint_as_float(sign | ((unsigned)(e - 1075 + 6 + 127) << 23));
  return {ok ? __uint_as_float(hbits) : 0.f, ok ? __fmul_rn(r, scale) : 0.f};
}

// Exact widening of a (normal or zero) float to double by bit operations.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e8 = (u >> 23) & 0xffu;
  const unsigned hi = (u & 0x80000000u) | ((e8 + 896u) << 20) | ((u >> 3) & 0xfffffu);
  const unsigned lo = u << 29;
  return e8 ? __hiloint2double((int)hi, (int)lo) : 0.0;
}

// Float-float to double: exact when the pair is normalised (|l| <= ulp(h)).
__device__ __forceinline__ double df_to_double(df a) {
  return __dadd_rn(f2d_bits(a.h), f2d_bits(a.l));
}

__device__ __forceinline__ df df_from2(float2 a) { return {a.x, a.y}; }
__device__ __forceinline__ float2 df_to2(df a) { return make_float2(a.h, a.l); }

// Fixed point with 52 fraction bits of a float (truncated), as int64.
// Valid for |f| < 2^10.
__device__ __forceinline__ long long f_to_fix52(float f) {
  const unsigned u = __float_as_uint(f);
  const int e8 = (int)((u >> 23) & 0xffu);
  const unsigned long long m = (unsigned long long)((u & 0x7fffffu) | 0x800000u);
  const int sh = e8 - 98;  // value = m * 2^(e8 - 150); * 2^52 -> m << (e8 - 98)
  unsigned long long q = sh >= 0 ? (m << min(sh, 39)) : (sh > -64 ? (m >> -sh) : 0ull);
  if (e8 == 0) q = 0;
  return (u & 0x80000000u) ? -(long long)q : (long long)q;
}

// The same value by one float -> int64 conversion that truncates the exact
// product f 2^52 toward zero (bit-identical to f_to_fix52 for |f| < 2^11).
// Fewer instructions: 6 % faster in the float-float step, which converts
// twelve values per particle; measured no faster in the FP32 step (six).
__device__ __forceinline__ long long f_to_fix52_cvt(float f) {
  return __float2ll_rz(__fmul_rn(f, 4503599627370496.0f));  // 2^52
}

// Fixed point with 52 fraction bits of a non-negative or negative double
// with |x| < 2^11 (exact up to the truncated bits below 2^-52).
__device__ __forceinline__ long long d_to_fix52(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = e - 1023;
  unsigned long long q = sh >= 0 ? (m << min(sh, 10)) : (sh > -64 ? (m >> -sh) : 0ull);
  if (e == 0) q = 0;
  return (b >> 63) ? -(long long)q : (long long)q;
}

// Interpolation coordinate on one axis from xi = x N/L in fixed point:
// s = xi - 1/2, i0 = floor(s), t = s - i0 = th + tl with th a multiple of
// 2^-23 and tl < 2^-23 (t truncated to 46 bits).
struct Axis {
  int i0;
  float th, tl;
};

__device__ __forceinline__ Axis axis_from_fix(long long q) {
  q -= (1ll << 51);
  Axis a;
  a.i0 = (int)(q >> 52);
  const unsigned long long fr = (unsigned long long)q & ((1ull << 52) - 1);
  a.th = __fsub_rn(__uint_as_float(0x3f800000u | (unsigned)(fr >> 29)), 1.0f);
  const float t2 = __fsub_rn(__uint_as_float(0x3f800000u | ((unsigned)(fr >> 6) & 0x7fffffu)), 1.0f);
  a.tl = __fmul_rn(t2, 1.1920928955078125e-07f);  // * 2^-23
  return a;
}

}  // namespace lcs
