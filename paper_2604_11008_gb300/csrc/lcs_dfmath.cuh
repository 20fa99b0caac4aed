// Float-float logarithm, exponential and power for the drag factor of
// Eq. (7) in the float-float step: f = 1 + 0.15 z^0.3435 with
// z = c tau |U - V|^2.  CUDA's FP64 pow runs on the FP64 pipe (about 1/80 of
// the FP32 rate on GB300) and made the nonlinear-drag step four times
// slower than the Stokes step; these routines use the FP32 pipe only.
//
// Method: table-driven reduction (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15 (1989) 144-157, and "... of the logarithm
// function", ACM TOMS 16 (1990) 378-400), carried out in float-float
// arithmetic:
//   log2 x = k + log2 c_j + log2(1 + r),  x = 2^k m,  c_j = 1 + (j + 1/2)/128
//            the table point nearest m,  r = m/c_j - 1,  |r| < 2^-8,
//            ln(1 + r) = r - r^2/2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6);
//   2^y    = 2^n 2^(j/64) e^u,  n = round(y),  j = round(64 (y - n)),
//            u = ln2 (y - n - j/64),  |u| < 2^-7.5,
//            e^u - 1 = u + u^2/2 + u^3 (1/6 + u/24 + u^2/120 + u^3/720).
// The quadratic terms are float-float, the cubic and higher tails plain
// FP32 (their rounding errors sit below 2^-47).  The tables (log2 c_j, 1/c_j,
// 2^(j/64) as float pairs) are computed at compile time in double precision
// from series: ln c = 2 atanh((c - 1)/(c + 1)), e^x by its Taylor series.
#pragma once

#include "lcs_df.cuh"

namespace lcs {

namespace dfm {

// ln c for c in [1/2, 2] from 2 atanh((c - 1)/(c + 1)) (|s| <= 1/3).
constexpr double ln_atanh(double c) {
  const double s = (c - 1.0) / (c + 1.0), s2 = s * s;
  double t = s, sum = 0.0;
  for (int k = 0; k < 40; ++k) {
    sum += t / (2 * k + 1);
    t *= s2;
  }
  return 2.0 * sum;
}

// e^x for |x| <= 1/2 by its Taylor series.
constexpr double exp_taylor(double x) {
  double t = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    t *= x / k;
    sum += t;
  }
  return sum;
}

constexpr double kLn2 = ln_atanh(2.0);

constexpr df split(double v) {
  const float h = (float)v;
  return df{h, (float)(v - (double)h)};
}

struct Tables {
  df log2c[128];   // log2(1 + (j + 1/2)/128)
  df rcpc[128];    // 1 / (1 + (j + 1/2)/128)
  df exp2j[65];    // 2^((j - 32)/64)
};

constexpr Tables make_tables() {
  Tables t{};
  for (int j = 0; j < 128; ++j) {
    const double c = 1.0 + (j + 0.5) / 128.0;
    t.log2c[j] = split(ln_atanh(c) / kLn2);
    t.rcpc[j] = split(1.0 / c);
  }
  for (int j = 0; j <= 64; ++j) t.exp2j[j] = split(exp_taylor((j - 32) / 64.0 * kLn2));
  return t;
}

}  // namespace dfm

static __device__ const dfm::Tables kDfmTables = dfm::make_tables();

__device__ __forceinline__ df dfm_load(const df *p) {
  const float2 v = __ldg((const float2 *)p);
  return {v.x, v.y};
}

// Square of a float pair.
__device__ __forceinline__ df df_sqr(df a) {
  const float p = __fmul_rn(a.h, a.h);
  float e = __fmaf_rn(a.h, a.h, -p);
  e = __fmaf_rn(__fadd_rn(a.h, a.h), a.l, e);
  return fast_two_sum(p, e);
}

// 2^k for an integer k in [-126, 127], exactly.
__device__ __forceinline__ float pow2i(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

// log2 x of a float pair x > 0 with x.h in [2^-100, 2^100]; absolute error
// a few units of 2^-48.
__device__ __forceinline__ df df_log2(df x) {
  const unsigned u = __float_as_uint(x.h);
  const int k = (int)((u >> 23) & 0xffu) - 127;
  const float mh = __uint_as_float((u & 0x007fffffu) | 0x3f800000u);  // x.h / 2^k in [1, 2)
  const float ml = __fmul_rn(x.l, pow2i(-k));                          // exact
  const int j = (int)((u >> 16) & 0x7fu);                                 // top 7 fraction bits
  const float c = __fadd_rn(1.0f, __fmul_rn((float)j + 0.5f, 0.0078125f));  // exact
  const df d = two_sum(__fsub_rn(mh, c), ml);  // m - c (mh - c is exact)
  const df r = df_mul(d, dfm_load(&kDfmTables.rcpc[j]));
  const df r2 = df_sqr(r);
  const float rh = r.h;
  const float tail = __fmul_rn(
      __fmul_rn(r2.h, rh),
      __fmaf_rn(rh, __fmaf_rn(rh, __fmaf_rn(rh, -1.0f / 6.0f, 0.2f), -0.25f), 1.0f / 3.0f));
  df ln1p = df_add(r, df_scale2(r2, -0.5f));
  ln1p = df_add(ln1p, df{tail, 0.0f});
  constexpr df kLog2e = dfm::split(1.0 / dfm::kLn2);
  const df v = df_add(dfm_load(&kDfmTables.log2c[j]), df_mul(ln1p, kLog2e));
  return df_add(df{(float)k, 0.0f}, v);
}

// 2^y of a float pair with |y| <= 120; relative error a few units of 2^-48.
__device__ __forceinline__ df df_exp2(df y) {
  const float n = rintf(y.h);
  const df f = two_sum(__fsub_rn(y.h, n), y.l);          // y - n (y.h - n is exact)
  const float jf = rintf(__fmul_rn(f.h, 64.0f));         // -32 .. 32
  const df g = two_sum(__fsub_rn(f.h, __fmul_rn(jf, 0.015625f)), f.l);  // exact difference
  constexpr df kLn2df = dfm::split(dfm::kLn2);
  const df uu = df_mul(g, kLn2df);
  const df u2 = df_sqr(uu);
  const float uh = uu.h;
  const float tail = __fmul_rn(
      __fmul_rn(u2.h, uh),
      __fmaf_rn(uh, __fmaf_rn(uh, __fmaf_rn(uh, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f),
                1.0f / 6.0f));
  df em1 = df_add(uu, df_scale2(u2, 0.5f));
  em1 = df_add(em1, df{tail, 0.0f});
  const df T = dfm_load(&kDfmTables.exp2j[(int)jf + 32]);
  const df r = df_add(T, df_mul(T, em1));
  const float s = pow2i((int)n);
  return {__fmul_rn(r.h, s), __fmul_rn(r.l, s)};
}

// Drag factor f = 1 + 0.15 (c tau |D|^2)^0.3435 of Eq. (7) in float-float
// (c = 18/(nu rho_p/rho), so that c tau |D|^2 = Re_p^2), given ct = c tau with
// ct.h in [2^-90, 2^90].  D is scaled by a power of two so that |D|^2 is
// formed without under- or overflow; when every |D_s| < 2^-100 the power
// term is below 2^-49 f and f = 1 is returned, as it is for D = 0.
// Non-finite D give a non-finite f.
__device__ __forceinline__ df drag_factor_dfp(df ct, const df D[3]) {
  const float m = fmaxf(fabsf(D[0].h), fmaxf(fabsf(D[1].h), fabsf(D[2].h)));
  if (!(D[0].h == D[0].h && D[1].h == D[1].h && D[2].h == D[2].h) || m > 3.0e38f)
    return df{m + D[0].h + D[1].h + D[2].h, 0.0f};  // NaN or inf
  if (m < 7.8886091e-31f) return df{1.0f, 0.0f};   // 2^-100
  const int E = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;  // -100 .. 127
  const float s1 = pow2i(-(E >> 1)), s2 = pow2i(-(E - (E >> 1)));
  df d2 = {0.0f, 0.0f};
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df ds = {__fmul_rn(__fmul_rn(D[s].h, s1), s2), __fmul_rn(__fmul_rn(D[s].l, s1), s2)};
    d2 = s == 0 ? df_sqr(ds) : df_add(d2, df_sqr(ds));   // in [1, 12)
  }
  const df z = df_mul(ct, d2);                       // Re_p^2 / 2^(2E)
  const df L = df_add(df_log2(z), df{(float)(2 * E), 0.0f});
  constexpr df kExp = dfm::split(0.3435);
  constexpr df k015 = dfm::split(0.15);
  const df p = df_exp2(df_mul(kExp, L));
  return df_add(df{1.0f, 0.0f}, df_mul(k015, p));
}

}  // namespace lcs
