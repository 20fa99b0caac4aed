// Per-particle arithmetic of the step, shared by the fused step kernel and
// by the adjoint's recompute (which must reproduce the forward bit for bit):
// trilinear interpolation from cell-centre values (Sec. 2.2) and one Heun
// step of Eqs. (5)-(6) with f = 1, gravity and the periodic wrap (Sec. 2.1),
// in FP64 (interp64 / heun_step64) or in float-float (interp_df, interp_lo,
// heun_step_df).
#pragma once

#include "lcs_df.cuh"
#include "lcs_dfmath.cuh"
#include "lcs_internal.cuh"

namespace lcs {

// ---------------------------------------------------------------- interpolation

// One 32-byte field record (a cell of the float-pair or the FP64 field) in a
// single 256-bit non-coherent load (sm_100 and later); the record must be
// 32-byte aligned, which the cudaMalloc'd field arrays guarantee.  Two
// 128-bit loads per cell made the float-float step 6 % slower.
__device__ __forceinline__ void ldg_cell32(const float4 *p, float4 &a, float4 &b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

__device__ __forceinline__ void ldg_cell32(const double2 *p, double2 &a, double2 &b) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
      : "=d"(a.x), "=d"(a.y), "=d"(b.x), "=d"(b.y)
      : "l"(p));
}

struct Stencil {
  uint32_t c[8];   // corner cell indices, order (a, b, d) = x outer, z inner
  double w[8];     // FP64 weights wx[a] * wy[b] * wz[d]
};

// Cell-centre stencil of the trilinear interpolation (Sec. 2.2):
// s = x N/L - 1/2, i0 = floor(s), t = s - i0, corners i0, i0+1 mod N.
__device__ __forceinline__ void axis64(double x, double inv_dx, int N, int &i0, double &t) {
  const double s = x * inv_dx - 0.5;
  const double f = floor(s);
  t = s - f;
  i0 = wrap_cell((int)f, N);
}

__device__ __forceinline__ void stencil64(const Geom &g, double x, double y, double z,
                                          Stencil &S) {
  const int N = g.N;
  int i0, j0, k0;
  double tx, ty, tz;
  axis64(x, g.inv_dx, N, i0, tx);
  axis64(y, g.inv_dx, N, j0, ty);
  axis64(z, g.inv_dx, N, k0, tz);
  const int i1 = i0 + 1 == N ? 0 : i0 + 1, j1 = j0 + 1 == N ? 0 : j0 + 1,
            k1 = k0 + 1 == N ? 0 : k0 + 1;
  const double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
  const uint32_t ii[2] = {(uint32_t)i0, (uint32_t)i1};
  const uint32_t jj[2] = {(uint32_t)j0 * N, (uint32_t)j1 * N};
  const uint32_t kk[2] = {(uint32_t)k0 * N * N, (uint32_t)k1 * N * N};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const int q = a * 4 + b * 2 + d;
        S.c[q] = ii[a] + jj[b] + kk[d];
        S.w[q] = wx[a] * wy[b] * wz[d];
      }
}

// FP64 trilinear interpolation of the FP64 field (all arithmetic on the FP64
// pipe; the reference form of the step, LCS_KERNEL_FP64).
__device__ __forceinline__ void interp64(const void *field, const Geom &g, double x, double y,
                                         double z, double &u, double &v, double &w) {
  Stencil S;
  stencil64(g, x, y, z, S);
  const double2 *f = (const double2 *)field;
  double au = 0.0, av = 0.0, aw = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double2 p, r;
    ldg_cell32(f + 2 * (size_t)S.c[q], p, r);
    au = fma(S.w[q], p.x, au);
    av = fma(S.w[q], p.y, av);
    aw = fma(S.w[q], r.x, aw);
  }
  u = au, v = av, w = aw;
}

// Shared-memory copy of a box of field cells for the sorted gather: cells
// [ox, ox+nx) x [oy, oy+ny) x [oz, oz+nz) in unwrapped cell coordinates
// (i = -2 .. N+1), records laid out as in global memory, x fastest.
// s == nullptr means no staged box.
struct FieldBox {
  const void *s;
  int ox, oy, oz, nx, ny, nz;
};

// Cell offset of corner (0,0,0) of a stencil inside the box, or -1.
__device__ __forceinline__ int box_base(const FieldBox &b, int i0, int j0, int k0) {
  if (!b.s) return -1;
  const int li = i0 - b.ox, lj = j0 - b.oy, lk = k0 - b.oz;
  if ((unsigned)li >= (unsigned)(b.nx - 1) || (unsigned)lj >= (unsigned)(b.ny - 1) ||
      (unsigned)lk >= (unsigned)(b.nz - 1))
    return -1;
  return (lk * b.ny + lj) * b.nx + li;
}

// Owned-field mode: a subdomain's own field brick in global memory, cells
// [p W - 2, p W + W + 2) per axis (its W cells plus a halo of two, wrapped
// into the periodic grid when the brick is built), x fastest, described by
// a FieldBox whose s points to the brick.  Cell offset of stencil corner
// (0,0,0), clamped into the brick so that every load stays inside it (a
// stencil that does not fit is reported by brick_holds).
__device__ __forceinline__ int brick_base(const FieldBox &b, int i0, int j0, int k0) {
  const int li = min(max(i0 - b.ox, 0), b.nx - 2), lj = min(max(j0 - b.oy, 0), b.ny - 2),
            lk = min(max(k0 - b.oz, 0), b.nz - 2);
  return (lk * b.ny + lj) * b.nx + li;
}

// Whether the brick holds the whole stencil of fixed-point position q.
__device__ __forceinline__ bool brick_holds(const FieldBox &b, const long long q[3]) {
  bool ok = true;
  const int o[3] = {b.ox, b.oy, b.oz}, n[3] = {b.nx, b.ny, b.nz};
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int i0 = (int)((q[s] - (1ll << 51)) >> 52);
    ok &= (unsigned)(i0 - o[s]) <= (unsigned)(n[s] - 2);
  }
  return ok;
}

// Fixed-point (52 fraction bits) coordinate x N/L of the first stage: one
// correctly rounded FP64 product, then bit operations.
__device__ __forceinline__ long long fix_stage1(double x, double inv_dx) {
  return d_to_fix52(__dmul_rn(x, inv_dx));
}

// Coordinate of the predictor X* = X + dt V: q1 + (dt N/L) V in fixed point.
__device__ __forceinline__ long long fix_stage2(long long q1, df V, df cx) {
  const df cv = df_mul(cx, V);
  return q1 + f_to_fix52_cvt(cv.h) + f_to_fix52_cvt(cv.l);
}

// The same for the FP32 increments of FP32 / BF16 storage: q1 + fix(cx V)
// with cx = dt N/L and V both rounded to FP32.
__device__ __forceinline__ long long fix_stage2_lo(long long q1, float V, float cx) {
  return q1 + f_to_fix52(cx * V);
}

// Predictor position of the FP64 step.
__device__ __forceinline__ double predictor64(double x, double v, double dt) { return x + dt * v; }

// ---------------------------------------------------------------- DF interpolation

// Product of two float pairs without renormalisation: (p, e) with
// p = RN(a.h b.h) and e = the exact rounding error plus the cross terms.
__device__ __forceinline__ df mul_un(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return {p, e};
}

// Trilinear interpolation (Sec. 2.2) in float-float arithmetic from the
// fixed-point coordinates q[s] = x_s N/L * 2^52.  The field record of a
// cell holds the float pairs of u, v, w: (hu, hv, hw, lu) (lv, lw, -, -).
// Corner weights are float-float products of the per-axis weights; each
// weight-times-value product is split exactly (fma error), the high parts
// are summed with two_sum and every small term goes to a compensation sum.
template <bool OWNED = false>
__device__ __forceinline__ void interp_df(const float4 *__restrict__ f, int N,
                                          const long long q[3], df U[3], const FieldBox &box) {
  const Axis ax = axis_from_fix(q[0]), ay = axis_from_fix(q[1]), az = axis_from_fix(q[2]);
  const int sb = OWNED ? brick_base(box, ax.i0, ay.i0, az.i0) : box_base(box, ax.i0, ay.i0, az.i0);
  const int i0 = wrap_cell(ax.i0, N), j0 = wrap_cell(ay.i0, N), k0 = wrap_cell(az.i0, N);
  const int i1 = i0 + 1 == N ? 0 : i0 + 1, j1 = j0 + 1 == N ? 0 : j0 + 1,
            k1 = k0 + 1 == N ? 0 : k0 + 1;
  const df wx[2] = {{__fsub_rn(1.0f, ax.th), -ax.tl}, {ax.th, ax.tl}};
  const df wy[2] = {{__fsub_rn(1.0f, ay.th), -ay.tl}, {ay.th, ay.tl}};
  const df wz[2] = {{__fsub_rn(1.0f, az.th), -az.tl}, {az.th, az.tl}};
  const uint32_t ii[2] = {(uint32_t)i0, (uint32_t)i1};
  const uint32_t jj[2] = {(uint32_t)j0 * N, (uint32_t)j1 * N};
  const uint32_t kk[2] = {(uint32_t)k0 * N * N, (uint32_t)k1 * N * N};
  float s[3], c[3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const df wab = mul_un(wx[a], wy[b]);
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const df w = mul_un(wab, wz[d]);
        float4 A, B;
        if (OWNED) {
          ldg_cell32((const float4 *)box.s + 2 * (sb + a + box.nx * (b + box.ny * d)), A, B);
        } else if (sb >= 0) {
          const float4 *sm = (const float4 *)box.s + 2 * (sb + a + box.nx * (b + box.ny * d));
          A = sm[0], B = sm[1];
        } else {
          const size_t cell = (size_t)(ii[a] + jj[b] + kk[d]);
          ldg_cell32(f + 2 * cell, A, B);
        }
        const float hv[3] = {A.x, A.y, A.z}, lv[3] = {A.w, B.x, B.y};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float P = __fmul_rn(w.h, hv[k]);
          const float E = __fmaf_rn(w.h, hv[k], -P);
          float t;
          if (a == 0 && b == 0 && d == 0) {
            s[k] = P;
            t = E;
          } else {
            const df st = two_sum(s[k], P);
            s[k] = st.h;
            t = __fadd_rn(st.l, E);
          }
          float small = __fmaf_rn(w.h, lv[k], t);
          small = __fmaf_rn(w.l, hv[k], small);
          c[k] = (a == 0 && b == 0 && d == 0) ? small : __fadd_rn(c[k], small);
        }
      }
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) U[k] = fast_two_sum(s[k], c[k]);
}

// Trilinear interpolation (Sec. 2.2) for FP32 / BF16 field storage: weights
// from the fixed-point coordinates rounded to FP32, FP32 accumulation.
template <int KIND, bool OWNED = false>
__device__ __forceinline__ void interp_lo(const void *__restrict__ field, int N,
                                          const long long q[3], df U[3], const FieldBox &box) {
  const Axis ax = axis_from_fix(q[0]), ay = axis_from_fix(q[1]), az = axis_from_fix(q[2]);
  const int sb = OWNED ? brick_base(box, ax.i0, ay.i0, az.i0) : box_base(box, ax.i0, ay.i0, az.i0);
  const int i0 = wrap_cell(ax.i0, N), j0 = wrap_cell(ay.i0, N), k0 = wrap_cell(az.i0, N);
  const int i1 = i0 + 1 == N ? 0 : i0 + 1, j1 = j0 + 1 == N ? 0 : j0 + 1,
            k1 = k0 + 1 == N ? 0 : k0 + 1;
  const float tx = __fadd_rn(ax.th, ax.tl), ty = __fadd_rn(ay.th, ay.tl),
              tz = __fadd_rn(az.th, az.tl);
  const float wx[2] = {__fsub_rn(1.0f, tx), tx}, wy[2] = {__fsub_rn(1.0f, ty), ty},
              wz[2] = {__fsub_rn(1.0f, tz), tz};
  const uint32_t ii[2] = {(uint32_t)i0, (uint32_t)i1};
  const uint32_t jj[2] = {(uint32_t)j0 * N, (uint32_t)j1 * N};
  const uint32_t kk[2] = {(uint32_t)k0 * N * N, (uint32_t)k1 * N * N};
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float wab = __fmul_rn(wx[a], wy[b]);
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const float w = __fmul_rn(wab, wz[d]);
        const uint32_t cell = ii[a] + jj[b] + kk[d];
        const int sc = sb + a + box.nx * (b + box.ny * d);
        float f[3];
        if (KIND == FK_F32) {
          const float4 p = OWNED     ? __ldg((const float4 *)box.s + sc)
                           : sb >= 0 ? ((const float4 *)box.s)[sc]
                                     : __ldg((const float4 *)field + cell);
          f[0] = p.x, f[1] = p.y, f[2] = p.z;
        } else {
          const uint2 p = OWNED     ? __ldg((const uint2 *)box.s + sc)
                          : sb >= 0 ? ((const uint2 *)box.s)[sc]
                                    : __ldg((const uint2 *)field + cell);
          f[0] = __uint_as_float((p.x & 0xffffu) << 16);
          f[1] = __uint_as_float(p.x & 0xffff0000u);
          f[2] = __uint_as_float((p.y & 0xffffu) << 16);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k] = __fmaf_rn(w, f[k], acc[k]);
      }
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) U[k] = {acc[k], 0.f};
}

template <int KIND, bool OWNED = false>
__device__ __forceinline__ void interp_any(const void *field, int N, const long long q[3],
                                           df U[3], const FieldBox &box) {
  if (KIND == FK_DF) interp_df<OWNED>((const float4 *)field, N, q, U, box);
  else interp_lo<KIND, OWNED>(field, N, q, U, box);
}

// Drag factor of Eq. (7): f = 1 + 0.15 Re_p^0.687 with Re_p^2 = c tau |D|^2,
// c = 18 / (nu rho_p/rho) (the radius from tau_p = (2/9)(rho_p/rho) r^2/nu,
// Sec. 2.2), D = U - V, so f = 1 + 0.15 (c tau |D|^2)^(0.687/2).  The float-
// float kernel evaluates it with the float-float log2 / exp2 of
// lcs_dfmath.cuh (relative error about 2^-46) whenever c tau lies in
// [2^-90, 2^90], which covers every physical case, else in FP64 with CUDA's
// pow; the FP32/BF16 kernels in FP32 with powf.
static __device__ __noinline__ df drag_factor_df(double c, double tau, const df D[3]) {
  const df ct = df_mul(split_d(c), split_d(tau));
  if (ct.h >= 8.0779356e-28f && ct.h <= 1.2379400e27f) return drag_factor_dfp(ct, D);
  double d2 = 0.0;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double d = df_to_double(D[s]);
    d2 = fma(d, d, d2);
  }
  return split_d(1.0 + 0.15 * pow(c * tau * d2, 0.3435));
}

static __device__ __noinline__ float drag_factor_f32(float c, float tau, const float D[3]) {
  const float d2 = fmaf(D[0], D[0], fmaf(D[1], D[1], D[2] * D[2]));
  return 1.0f + 0.15f * powf(c * tau * d2, 0.3435f);
}

// Time fractions of a step's two stages between the field snapshots
// (evolving field only): U = U_a + th (U_b - U_a).
struct StageTimes {
  double th1, th2;
};

__device__ __forceinline__ StageTimes stage_times(const StepArgs &a) {
  if (!a.field_b) return {0.0, 0.0};
  const double th1 = fma((double)*a.m.nstep, a.dth, a.th0);
  return {th1, th1 + a.dth};
}

// Wrap a fixed-point coordinate into [0, N 2^52) (Sec. 2.1): one image per
// step; img counts the images crossed.
__device__ __forceinline__ long long wrap_fix(long long q, long long qL, int &img) {
  if (q < 0) {
    q += qL;
    img -= 1;
  } else if (q >= qL) {
    q -= qL;
    img += 1;
  }
  return q;
}

// The second snapshot's view of an owned-field brick: same geometry, the
// same subdomain's brick in bricks_b.
__device__ __forceinline__ FieldBox brick_b_of(const StepArgs &a, const FieldBox &box) {
  FieldBox b = box;
  b.s = (const unsigned char *)a.bricks_b +
        ((const unsigned char *)box.s - (const unsigned char *)a.bricks);
  return b;
}

// U <- U + th (U_b - U) with U_b interpolated from the second snapshot
// (float-float; FP32 for FP32/BF16 storage, whose U carries no low part);
// OWNED: from the subdomain's brick of the second snapshot.
template <int KIND, bool OWNED = false>
__device__ __forceinline__ void lerp_field_df(const StepArgs &a, const long long q[3], double th,
                                           df U[3], const FieldBox &box = FieldBox{}) {
  df Ub[3];
  interp_any<KIND, OWNED>(a.field_b, a.geo.N, q, Ub, OWNED ? brick_b_of(a, box) : FieldBox{});
  const df t = split_d(th);
#pragma unroll
  for (int s = 0; s < 3; ++s) U[s] = df_add(U[s], df_mul(t, df_add(Ub[s], df_neg(U[s]))));
}

template <int KIND, bool OWNED = false>
__device__ __forceinline__ void lerp_field_lo(const StepArgs &a, const long long q[3], float th,
                                           df U[3], const FieldBox &box = FieldBox{}) {
  df Ub[3];
  interp_lo<KIND, OWNED>(a.field_b, a.geo.N, q, Ub, OWNED ? brick_b_of(a, box) : FieldBox{});
#pragma unroll
  for (int s = 0; s < 3; ++s) U[s].h = fmaf(th, Ub[s].h - U[s].h, U[s].h);
}

// Heun step of Eqs. (5)-(6) (gravity g) with float-float increments, on the
// fixed-point position q (cell units, 52 fraction bits) and the float-pair
// velocity V, with h = dt/tau and f = 1 (Stokes) or the factor of Eq. (7):
//   X* = X + dt V                          (needs only the record: taken first)
//   a1 = h1 (U(X) - V) + dt g              (dt A1, h1 = f(D1) h)
//   V* = V + a1,  Vh = V + a1/2
//   X' = X + dt Vh                         [= X + (dt/2)(V + V*)]
//   a2 = h2 (U(X*) - V*) + dt g            (dt A2)
//   V' = Vh + a2/2                         [= V + (dt/2)(A1 + A2)]
// X' is added to q in fixed point (exact addition of a float-float
// displacement converted to fixed point) and wrapped before the second
// interpolation, so only X', V* and Vh stay live across it.  No FP64
// instruction on the Stokes path.
template <int KIND, bool EVOLVE = false, bool OWNED = false>
__device__ __forceinline__ void heun_step_df(const StepArgs &a, long long q[3], df V[3],
                                             double tau, int img[3], int &bad,
                                             const FieldBox &box = FieldBox{},
                                             StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const df cx = {a.dfk[4], a.dfk[5]};  // dt N/L
  const df h = df_mul(df{a.dfk[0], a.dfk[1]}, df_recip(split_d(tau)));
  long long q2[3];
  df U[3], Vs[3], Vh[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) q2[s] = fix_stage2(q[s], V[s], cx);
  if (OWNED && !brick_holds(box, q)) bad |= 2;
  interp_any<KIND, OWNED>(a.field, g.N, q, U, box);
  if (EVOLVE && a.field_b) lerp_field_df<KIND, OWNED>(a, q, tt.th1, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) U[s] = df_add(U[s], df_neg(V[s]));  // D1
  const df h1 = a.drag ? df_mul(h, drag_factor_df(a.drag_c, tau, U)) : h;
  const float half_box = 0.5f * (float)g.N;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df gd = {a.dfk[6 + 2 * s], a.dfk[7 + 2 * s]};
    const df a1 = df_add(df_mul(h1, U[s]), gd);
    Vs[s] = df_add(V[s], a1);
    Vh[s] = df_add(V[s], df_scale2(a1, 0.5f));
    const df dXc = df_mul(cx, Vh[s]);  // displacement in cell units
    if (!(fabsf(dXc.h) < half_box)) bad |= isfinite(dXc.h) ? 2 : 1;
    q[s] = wrap_fix(q[s] + f_to_fix52_cvt(dXc.h) + f_to_fix52_cvt(dXc.l), g.qL, img[s]);
  }
  if (OWNED && !brick_holds(box, q2)) bad |= 2;
  interp_any<KIND, OWNED>(a.field, g.N, q2, U, box);
  if (EVOLVE && a.field_b) lerp_field_df<KIND, OWNED>(a, q2, tt.th2, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) U[s] = df_add(U[s], df_neg(Vs[s]));  // D2
  const df h2 = a.drag ? df_mul(h, drag_factor_df(a.drag_c, tau, U)) : h;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df gd = {a.dfk[6 + 2 * s], a.dfk[7 + 2 * s]};
    const df a2 = df_add(df_mul(h2, U[s]), gd);
    const df vn = df_add(Vh[s], df_scale2(a2, 0.5f));
    if (!isfinite(vn.h)) bad |= 1;
    V[s] = vn;
  }
}

// Heun step of Eqs. (5)-(6) for FP32 / BF16 field storage: the same
// formulas as heun_step_df with the increments in FP32 (the field itself
// carries 2^-24 or 2^-8 relative error), accumulated exactly into the
// fixed-point position and in float-float into the velocity.
template <int KIND, bool EVOLVE = false, bool OWNED = false>
__device__ __forceinline__ void heun_step_lo(const StepArgs &a, long long q[3], df V[3],
                                             double tau, int img[3], int &bad,
                                             const FieldBox &box = FieldBox{},
                                             StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const float dt = a.dfk[0], cx = a.dfk[4];
  const float taus = split_d(tau).h;
  const float h = dt * __frcp_rn(taus);
  long long q2[3];
  df U[3];
  float a1[3], Vs[3], D[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) q2[s] = fix_stage2_lo(q[s], V[s].h, cx);
  if (OWNED && !brick_holds(box, q)) bad |= 2;
  interp_lo<KIND, OWNED>(a.field, g.N, q, U, box);
  if (EVOLVE && a.field_b) lerp_field_lo<KIND, OWNED>(a, q, (float)tt.th1, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) D[s] = U[s].h - V[s].h;
  const float h1 = a.drag ? h * drag_factor_f32((float)a.drag_c, taus, D) : h;
  const float half_box = 0.5f * (float)g.N;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    a1[s] = h1 * D[s] + a.dfk[6 + 2 * s];
    Vs[s] = V[s].h + a1[s];
    const float dXc = cx * (V[s].h + 0.5f * a1[s]);  // cell units
    if (!(fabsf(dXc) < half_box)) bad |= isfinite(dXc) ? 2 : 1;
    q[s] = wrap_fix(q[s] + f_to_fix52(dXc), g.qL, img[s]);
  }
  if (OWNED && !brick_holds(box, q2)) bad |= 2;
  interp_lo<KIND, OWNED>(a.field, g.N, q2, U, box);
  if (EVOLVE && a.field_b) lerp_field_lo<KIND, OWNED>(a, q2, (float)tt.th2, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) D[s] = U[s].h - Vs[s];
  const float h2 = a.drag ? h * drag_factor_f32((float)a.drag_c, taus, D) : h;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const float a2 = h2 * D[s] + a.dfk[6 + 2 * s];
    const df vn = df_add(V[s], df{0.5f * (a1[s] + a2), 0.f});
    if (!isfinite(vn.h)) bad |= 1;
    V[s] = vn;
  }
}

// ---------------------------------------------------------------- stages taken apart

// The two Heun stages as separate passes, for migration after each stage
// (Sec. 3.2.2).  Stage 1 moves the particle to its predictor position and
// records the stage velocity:  X* = X + dt V (wrapped),  V* = V + h1 D1 + dt g,
// V unchanged.  Stage 2 completes the step from X*, V, V*:
//   X' = X* + (dt/2)(V* - V)          [= X + (dt/2)(V + V*)]
//   V' = (V + V* + h2 D2 + dt g) / 2  [= V + (dt/2)(A1 + A2), dt A1 = V* - V]
// with D2 = U(X*) - V*.  Same arithmetic pieces as the fused step.
template <int KIND, bool OWNED = false, bool EVOLVE = false>
__device__ __forceinline__ void heun_stage1_df(const StepArgs &a, long long q[3], const df V[3],
                                               df Vs[3], double tau, int img[3], int &bad,
                                               const FieldBox &box = FieldBox{},
                                               StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const df dt = {a.dfk[0], a.dfk[1]}, cx = {a.dfk[4], a.dfk[5]};
  const df h = df_mul(dt, df_recip(split_d(tau)));
  df U[3], D[3];
  if (OWNED && !brick_holds(box, q)) bad |= 2;
  interp_any<KIND, OWNED>(a.field, g.N, q, U, box);
  if (EVOLVE && a.field_b) lerp_field_df<KIND, OWNED>(a, q, tt.th1, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) D[s] = df_add(U[s], df_neg(V[s]));
  const df h1 = a.drag ? df_mul(h, drag_factor_df(a.drag_c, tau, D)) : h;
  const float half_box = 0.5f * (float)g.N;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df gd = {a.dfk[6 + 2 * s], a.dfk[7 + 2 * s]};
    Vs[s] = df_add(df_add(V[s], df_mul(h1, D[s])), gd);
    const df dXc = df_mul(cx, V[s]);
    if (!(fabsf(dXc.h) < half_box)) bad |= isfinite(dXc.h) ? 2 : 1;
    if (!isfinite(Vs[s].h)) bad |= 1;
    q[s] = wrap_fix(fix_stage2(q[s], V[s], cx), g.qL, img[s]);
  }
}

template <int KIND, bool OWNED = false, bool EVOLVE = false>
__device__ __forceinline__ void heun_stage2_df(const StepArgs &a, long long q[3], df V[3],
                                               const df Vs[3], double tau, int img[3],
                                               int &bad,
                                               const FieldBox &box = FieldBox{},
                                               StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const df dt = {a.dfk[0], a.dfk[1]}, cx = {a.dfk[4], a.dfk[5]};
  const df hcx = df_scale2(cx, 0.5f);
  const df h = df_mul(dt, df_recip(split_d(tau)));
  df U[3], D[3];
  if (OWNED && !brick_holds(box, q)) bad |= 2;
  interp_any<KIND, OWNED>(a.field, g.N, q, U, box);
  if (EVOLVE && a.field_b) lerp_field_df<KIND, OWNED>(a, q, tt.th2, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) D[s] = df_add(U[s], df_neg(Vs[s]));
  const df h2 = a.drag ? df_mul(h, drag_factor_df(a.drag_c, tau, D)) : h;
  const float half_box = 0.5f * (float)g.N;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df gd = {a.dfk[6 + 2 * s], a.dfk[7 + 2 * s]};
    const df dXc = df_mul(hcx, df_add(Vs[s], df_neg(V[s])));
    const df vn =
        df_scale2(df_add(df_add(V[s], Vs[s]), df_add(df_mul(h2, D[s]), gd)), 0.5f);
    if (!(fabsf(dXc.h) < half_box)) bad |= isfinite(dXc.h) ? 2 : 1;
    if (!isfinite(vn.h)) bad |= 1;
    q[s] = wrap_fix(q[s] + f_to_fix52_cvt(dXc.h) + f_to_fix52_cvt(dXc.l), g.qL, img[s]);
    V[s] = vn;
  }
}

template <int KIND, bool OWNED = false, bool EVOLVE = false>
__device__ __forceinline__ void heun_stage1_lo(const StepArgs &a, long long q[3], const df V[3],
                                               df Vs[3], double tau, int img[3], int &bad,
                                               const FieldBox &box = FieldBox{},
                                               StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const float dt = a.dfk[0], cx = a.dfk[4];
  const float taus = split_d(tau).h;
  const float h = dt * __frcp_rn(taus);
  df U[3];
  float D[3];
  if (OWNED && !brick_holds(box, q)) bad |= 2;
  interp_lo<KIND, OWNED>(a.field, g.N, q, U, box);
  if (EVOLVE && a.field_b) lerp_field_lo<KIND, OWNED>(a, q, (float)tt.th1, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) D[s] = U[s].h - V[s].h;
  const float h1 = a.drag ? h * drag_factor_f32((float)a.drag_c, taus, D) : h;
  const float half_box = 0.5f * (float)g.N;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    Vs[s] = df_add(V[s], df{h1 * D[s] + a.dfk[6 + 2 * s], 0.f});
    const float dXc = cx * V[s].h;
    if (!(fabsf(dXc) < half_box)) bad |= isfinite(dXc) ? 2 : 1;
    if (!isfinite(Vs[s].h)) bad |= 1;
    q[s] = wrap_fix(fix_stage2_lo(q[s], V[s].h, cx), g.qL, img[s]);
  }
}

template <int KIND, bool OWNED = false, bool EVOLVE = false>
__device__ __forceinline__ void heun_stage2_lo(const StepArgs &a, long long q[3], df V[3],
                                               const df Vs[3], double tau, int img[3],
                                               int &bad,
                                               const FieldBox &box = FieldBox{},
                                               StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const float dt = a.dfk[0], cx = a.dfk[4];
  const float taus = split_d(tau).h;
  const float h = dt * __frcp_rn(taus);
  df U[3];
  float D[3];
  if (OWNED && !brick_holds(box, q)) bad |= 2;
  interp_lo<KIND, OWNED>(a.field, g.N, q, U, box);
  if (EVOLVE && a.field_b) lerp_field_lo<KIND, OWNED>(a, q, (float)tt.th2, U, box);
#pragma unroll
  for (int s = 0; s < 3; ++s) D[s] = U[s].h - Vs[s].h;
  const float h2 = a.drag ? h * drag_factor_f32((float)a.drag_c, taus, D) : h;
  const float half_box = 0.5f * (float)g.N;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df dv = df_add(Vs[s], df_neg(V[s]));   // dt A1 = V* - V
    const float dXc = 0.5f * cx * dv.h;
    const df vn = df_add(V[s], df{0.5f * (dv.h + h2 * D[s] + a.dfk[6 + 2 * s]), 0.f});
    if (!(fabsf(dXc) < half_box)) bad |= isfinite(dXc) ? 2 : 1;
    if (!isfinite(vn.h)) bad |= 1;
    q[s] = wrap_fix(q[s] + f_to_fix52(dXc), g.qL, img[s]);
    V[s] = vn;
  }
}

// FP64 position of a fixed-point coordinate and velocity of a float pair
// (the all-FP64 kernel and its adjoint read the state through these).
__device__ __forceinline__ double pos_of_fix(long long q, const Geom &g) {
  return __dmul_rn(__ll2double_rn(q), g.fix_dx);
}
__device__ __forceinline__ double vel_of_df(df v) { return __dadd_rn((double)v.h, (double)v.l); }
__device__ __forceinline__ df df_of_double(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(__dsub_rn(v, (double)h))};
}

// u <- u + th (u_b - u) in FP64 (evolving field).
__device__ __forceinline__ void lerp_field64(const StepArgs &a, const double x[3], double th,
                                                 double u[3]) {
  double ub[3];
  interp64(a.field_b, a.geo, x[0], x[1], x[2], ub[0], ub[1], ub[2]);
#pragma unroll
  for (int s = 0; s < 3; ++s) u[s] = fma(th, ub[s] - u[s], u[s]);
}

// Drag factor of Eq. (7) in FP64 (see drag_factor_df).
static __device__ __noinline__ double drag_factor64(double c, double tau, const double u[3],
                                                const double v[3]) {
  double d2 = 0.0;
#pragma unroll
  for (int s = 0; s < 3; ++s) d2 = fma(u[s] - v[s], u[s] - v[s], d2);
  return 1.0 + 0.15 * pow(c * tau * d2, 0.3435);
}

// One Heun step of Eqs. (5)-(6) (gravity g; f = 1 or Eq. 7) in FP64
// arithmetic: the state is read as FP64 position and velocity, advanced with
// FP64 operations only, and stored back (position rounded to the fixed-point
// grid of 2^-52 cells, velocity to a float pair), then wrapped.
template <bool EVOLVE = false>
__device__ __forceinline__ void heun_step64(const StepArgs &a, long long q[3], df V[3],
                                          double tau, int img[3], int &bad,
                                          StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const double itau = 1.0 / tau;
  double x[3], v[3], u1[3], a1[3], xs[3], vs[3], u2[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    x[s] = pos_of_fix(q[s], g);
    v[s] = vel_of_df(V[s]);
  }
  interp64(a.field, g, x[0], x[1], x[2], u1[0], u1[1], u1[2]);
  if (EVOLVE && a.field_b) lerp_field64(a, x, tt.th1, u1);
  const double f1 = a.drag ? drag_factor64(a.drag_c, tau, u1, v) * itau : itau;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    a1[s] = (u1[s] - v[s]) * f1 + a.g[s];
    xs[s] = predictor64(x[s], v[s], a.dt);
    vs[s] = v[s] + a.dt * a1[s];
  }
  interp64(a.field, g, xs[0], xs[1], xs[2], u2[0], u2[1], u2[2]);
  if (EVOLVE && a.field_b) lerp_field64(a, xs, tt.th2, u2);
  const double f2 = a.drag ? drag_factor64(a.drag_c, tau, u2, vs) * itau : itau;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double a2 = (u2[s] - vs[s]) * f2 + a.g[s];
    const double xn = x[s] + a.half_dt * (v[s] + vs[s]);
    const double vn = v[s] + a.half_dt * (a1[s] + a2);
    if (!(fabs(xn - x[s]) < 0.5 * g.L)) bad |= fabs(xn) <= 1e300 ? 2 : 1;
    if (!isfinite(vn)) bad |= 1;
    q[s] = wrap_fix(d_to_fix52(__dmul_rn(xn, g.inv_dx)), g.qL, img[s]);
    V[s] = df_of_double(vn);
  }
}

// The two stages in FP64 arithmetic (see heun_stage1_df).
template <bool EVOLVE = false>
__device__ __forceinline__ void heun_stage1_64(const StepArgs &a, long long q[3], const df V[3],
                                               df Vs[3], double tau, int img[3], int &bad,
                                               StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const double itau = 1.0 / tau;
  double x[3], v[3], u1[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    x[s] = pos_of_fix(q[s], g);
    v[s] = vel_of_df(V[s]);
  }
  interp64(a.field, g, x[0], x[1], x[2], u1[0], u1[1], u1[2]);
  if (EVOLVE && a.field_b) lerp_field64(a, x, tt.th1, u1);
  const double f1 = a.drag ? drag_factor64(a.drag_c, tau, u1, v) * itau : itau;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double a1 = (u1[s] - v[s]) * f1 + a.g[s];
    const double xs = predictor64(x[s], v[s], a.dt);
    const double vs = v[s] + a.dt * a1;
    if (!(fabs(xs - x[s]) < 0.5 * g.L)) bad |= fabs(xs) <= 1e300 ? 2 : 1;
    if (!isfinite(vs)) bad |= 1;
    q[s] = wrap_fix(d_to_fix52(__dmul_rn(xs, g.inv_dx)), g.qL, img[s]);
    Vs[s] = df_of_double(vs);
  }
}

template <bool EVOLVE = false>
__device__ __forceinline__ void heun_stage2_64(const StepArgs &a, long long q[3], df V[3],
                                               const df Vs[3], double tau, int img[3],
                                               int &bad, StageTimes tt = StageTimes{0.0, 0.0}) {
  const Geom &g = a.geo;
  const double itau = 1.0 / tau;
  double xs[3], v[3], vs[3], u2[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    xs[s] = pos_of_fix(q[s], g);
    v[s] = vel_of_df(V[s]);
    vs[s] = vel_of_df(Vs[s]);
  }
  interp64(a.field, g, xs[0], xs[1], xs[2], u2[0], u2[1], u2[2]);
  if (EVOLVE && a.field_b) lerp_field64(a, xs, tt.th2, u2);
  const double f2 = a.drag ? drag_factor64(a.drag_c, tau, u2, vs) * itau : itau;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double a2 = (u2[s] - vs[s]) * f2 + a.g[s];
    const double xn = xs[s] + a.half_dt * (vs[s] - v[s]);
    const double vn = 0.5 * (v[s] + vs[s]) + a.half_dt * a2;
    if (!(fabs(xn - xs[s]) < 0.5 * g.L)) bad |= fabs(xn) <= 1e300 ? 2 : 1;
    if (!isfinite(vn)) bad |= 1;
    q[s] = wrap_fix(d_to_fix52(__dmul_rn(xn, g.inv_dx)), g.qL, img[s]);
    V[s] = df_of_double(vn);
  }
}

}  // namespace lcs
