// Fused particle step: interpolate + Heun + wrap + destination flag +
// decoupled look-back prefix scan + pack, then offsets and unpack.
//
// Method (Tominaga & Onishi, LCS.jl, arXiv 2604.11008):
//   Sec. 2.2, Eqs. (5)-(6): dX/dt = V, dV/dt = -(f/tau_p)(V - U(X)), f = 1,
//     plus a constant g; U(X) by trilinear interpolation from the eight
//     surrounding cell-centre values; two-stage second-order RK (Heun).
//   Sec. 2.1: periodic cube of side L, grid spacing L/N.
//   Sec. 2.3.3: particles leaving a subdomain are flagged (mask), a prefix
//     scan of the flags gives every leaving particle its send-buffer slot,
//     and all particles are packed in parallel.  Here the flag is a
//     destination direction (27 bins), the scan counts stayers and leavers
//     at once, and stayers are written straight to their compacted slot.
//   Sec. 3.2.2: unpack = compaction of the stayers plus appending the
//     arrivals, ordered by source subdomain.
#include <algorithm>
#include <cuda/atomic>

#include "lcs_df.cuh"
#include "lcs_internal.cuh"

namespace lcs {

// ---------------------------------------------------------------- field

__device__ __forceinline__ uint16_t bf16_rne_from_double(double x) {
  // Round to nearest even directly from the FP64 bit pattern (no detour
  // through FP32, which could round twice).
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint16_t sign = (uint16_t)((b >> 63) << 15);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & ((1ull << 52) - 1);
  if (e == 0x7ff) return (uint16_t)(sign | 0x7f80 | (m ? 0x40 : 0));
  if (e == 0) return sign;  // zero or FP64 subnormal (far below BF16 range)
  int E = e - 1023;
  const unsigned long long full = (1ull << 52) | m;
  if (E >= -126) {
    unsigned long long q = full >> 45, rem = full & ((1ull << 45) - 1), half = 1ull << 44;
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q == 256) { q = 128; ++E; }
    if (E > 127) return (uint16_t)(sign | 0x7f80);
    return (uint16_t)(sign | ((E + 127) << 7) | (q & 127));
  }
  const int shift = -81 - E;  // count of 2^-133 units: full * 2^(E-52+133)
  if (shift >= 64) return sign;
  unsigned long long q = full >> shift, rem = full & ((1ull << shift) - 1),
                     half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1))) ++q;
  return (uint16_t)(sign | q);
}

__global__ void k_field_convert(const double *__restrict__ src, int64_t ncell, int kind,
                                void *dst) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double u = src[c], v = src[ncell + c], w = src[2 * ncell + c];
    if (kind == FK_F64) {
      double2 *d = (double2 *)dst;
      d[2 * c] = make_double2(u, v);
      d[2 * c + 1] = make_double2(w, 0.0);
    } else if (kind == FK_DF) {
      const float hu = __double2float_rn(u), hv = __double2float_rn(v), hw = __double2float_rn(w);
      const float lu = __double2float_rn(u - (double)hu), lv = __double2float_rn(v - (double)hv),
                  lw = __double2float_rn(w - (double)hw);
      float4 *d = (float4 *)dst;
      d[2 * c] = make_float4(hu, hv, hw, lu);
      d[2 * c + 1] = make_float4(lv, lw, 0.f, 0.f);
    } else if (kind == FK_F32) {
      ((float4 *)dst)[c] =
          make_float4(__double2float_rn(u), __double2float_rn(v), __double2float_rn(w), 0.f);
    } else {
      const uint32_t a = bf16_rne_from_double(u), b = bf16_rne_from_double(v),
                     cc = bf16_rne_from_double(w);
      ((uint2 *)dst)[c] = make_uint2(a | (b << 16), cc);
    }
  }
}

// Expand the stored field back to FP64 [3][N^3] (inspection / tests).
__global__ void k_field_expand(const void *src, int64_t ncell, int kind, double *dst) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double u, v, w;
    if (kind == FK_F64) {
      const double2 *s = (const double2 *)src;
      u = s[2 * c].x, v = s[2 * c].y, w = s[2 * c + 1].x;
    } else if (kind == FK_DF) {
      const float4 *s = (const float4 *)src;
      const float4 a = s[2 * c], b = s[2 * c + 1];
      u = (double)a.x + (double)a.w, v = (double)a.y + (double)b.x, w = (double)a.z + (double)b.y;
    } else if (kind == FK_F32) {
      const float4 a = ((const float4 *)src)[c];
      u = a.x, v = a.y, w = a.z;
    } else {
      const uint2 a = ((const uint2 *)src)[c];
      u = __uint_as_float((a.x & 0xffffu) << 16);
      v = __uint_as_float(a.x & 0xffff0000u);
      w = __uint_as_float((a.y & 0xffffu) << 16);
    }
    dst[c] = u, dst[ncell + c] = v, dst[2 * ncell + c] = w;
  }
}

cudaError_t launch_field_convert(const double *src, int N, FieldKind kind, void *dst,
                                 cudaStream_t st) {
  const int64_t ncell = (int64_t)N * N * N;
  const int grid = (int)std::min<int64_t>((ncell + 255) / 256, 152 * 32);
  k_field_convert<<<grid, 256, 0, st>>>(src, ncell, (int)kind, dst);
  return cudaGetLastError();
}

cudaError_t launch_field_expand(const void *src, int N, FieldKind kind, double *dst,
                                cudaStream_t st) {
  const int64_t ncell = (int64_t)N * N * N;
  const int grid = (int)std::min<int64_t>((ncell + 255) / 256, 152 * 32);
  k_field_expand<<<grid, 256, 0, st>>>(src, ncell, (int)kind, dst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- interpolation

struct Stencil {
  uint32_t c[8];   // corner cell indices, order (a, b, d) = x outer, z inner
  double w[8];     // FP64 weights wx[a] * wy[b] * wz[d]
};

// Cell-centre stencil of the trilinear interpolation (Sec. 2.2):
// s = x N/L - 1/2, i0 = floor(s), t = s - i0, corners i0, i0+1 mod N.
__device__ __forceinline__ void stencil64(const Geom &g, double x, double y, double z,
                                          Stencil &S) {
  const double sx = x * g.inv_dx - 0.5, sy = y * g.inv_dx - 0.5, sz = z * g.inv_dx - 0.5;
  const double fx = floor(sx), fy = floor(sy), fz = floor(sz);
  const double tx = sx - fx, ty = sy - fy, tz = sz - fz;
  const int N = g.N;
  const int i0 = wrap_cell((int)fx, N), j0 = wrap_cell((int)fy, N), k0 = wrap_cell((int)fz, N);
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
    const double2 p = __ldg(f + 2 * (size_t)S.c[q]);
    const double2 r = __ldg(f + 2 * (size_t)S.c[q] + 1);
    au = fma(S.w[q], p.x, au);
    av = fma(S.w[q], p.y, av);
    aw = fma(S.w[q], r.x, aw);
  }
  u = au, v = av, w = aw;
}

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
__device__ __forceinline__ void interp_df(const float4 *__restrict__ f, int N,
                                          const long long q[3], df U[3]) {
  const Axis ax = axis_from_fix(q[0]), ay = axis_from_fix(q[1]), az = axis_from_fix(q[2]);
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
        const size_t cell = (size_t)(ii[a] + jj[b] + kk[d]);
        const float4 A = __ldg(f + 2 * cell), B = __ldg(f + 2 * cell + 1);
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
template <int KIND>
__device__ __forceinline__ void interp_lo(const void *__restrict__ field, int N,
                                          const long long q[3], df U[3]) {
  const Axis ax = axis_from_fix(q[0]), ay = axis_from_fix(q[1]), az = axis_from_fix(q[2]);
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
        float f[3];
        if (KIND == FK_F32) {
          const float4 p = __ldg((const float4 *)field + cell);
          f[0] = p.x, f[1] = p.y, f[2] = p.z;
        } else {
          const uint2 p = __ldg((const uint2 *)field + cell);
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

template <int KIND>
__device__ __forceinline__ void interp_any(const void *field, int N, const long long q[3],
                                           df U[3]) {
  if (KIND == FK_DF) interp_df((const float4 *)field, N, q, U);
  else interp_lo<KIND>(field, N, q, U);
}

// Heun step of Eqs. (5)-(6) (f = 1, gravity g) with float-float increments:
//   h = dt/tau, D1 = U(X) - V, V* = V + h D1 + dt g, X* = X + dt V,
//   D2 = U(X*) - V*, dV = (h D1 + h D2)/2 + dt g,
//   dX = dt V + (dt/2)(h D1 + dt g)          [= dt (V + V*)/2]
// then X' = X + dX and V' = V + dV in FP64, and the periodic wrap.
template <int KIND>
__device__ __forceinline__ void heun_step_df(const StepArgs &a, double x[3], double v[3],
                                             double tau, int img[3], int &bad) {
  const Geom &g = a.geo;
  const df dt = {a.dfk[0], a.dfk[1]}, hdt = {a.dfk[2], a.dfk[3]}, cx = {a.dfk[4], a.dfk[5]};
  const df h = df_mul(dt, df_recip(split_d(tau)));
  long long q[3];
  df V[3], U[3], hD1[3], Vs[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) q[s] = d_to_fix52(__dmul_rn(x[s], g.inv_dx));
  interp_any<KIND>(a.field, g.N, q, U);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df gd = {a.dfk[6 + 2 * s], a.dfk[7 + 2 * s]};
    V[s] = split_d(v[s]);
    hD1[s] = df_mul(h, df_add(U[s], df_neg(V[s])));
    Vs[s] = df_add(df_add(V[s], hD1[s]), gd);
    const df cv = df_mul(cx, V[s]);
    q[s] += f_to_fix52(cv.h) + f_to_fix52(cv.l);
  }
  interp_any<KIND>(a.field, g.N, q, U);
  const long long bitsL = __double_as_longlong(g.L);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df gd = {a.dfk[6 + 2 * s], a.dfk[7 + 2 * s]};
    const df hD2 = df_mul(h, df_add(U[s], df_neg(Vs[s])));
    const df dV = df_add(df_scale2(df_add(hD1[s], hD2), 0.5f), gd);
    const df dX = df_add(df_mul(dt, V[s]), df_mul(hdt, df_add(hD1[s], gd)));
    if (!(fabsf(dX.h) < (float)(0.5 * g.L))) bad |= 2;
    double xn = __dadd_rn(x[s], df_to_double(dX));
    const double vn = __dadd_rn(v[s], df_to_double(dV));
    const long long bx = __double_as_longlong(xn);
    if (((bx >> 52) & 0x7ff) == 0x7ff || ((__double_as_longlong(vn) >> 52) & 0x7ff) == 0x7ff)
      bad |= 1;
    if (bx < 0) {
      xn = __dadd_rn(xn, g.L);
      img[s] -= 1;
    } else if (bx >= bitsL) {
      xn = __dsub_rn(xn, g.L);
      img[s] += 1;
    }
    if (__double_as_longlong(xn) == bitsL) xn = 0.0;
    x[s] = xn;
    v[s] = vn;
  }
}

// ---------------------------------------------------------------- look-back

constexpr unsigned long long FLAG_AGG = 1ull << 62;
constexpr unsigned long long FLAG_PRE = 2ull << 62;
constexpr unsigned long long FLAG_MASK = 3ull << 62;
constexpr unsigned long long VAL_MASK = ~FLAG_MASK;

__device__ __forceinline__ unsigned long long pack_sm(unsigned long long stay,
                                                      unsigned long long mig) {
  return (stay << 31) | mig;
}

using atom_u64 = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;

// Exclusive (stay, mig) prefix of tile `t` within its segment (first tile of
// the segment at t0).  Publishes the tile's aggregate, then its inclusive
// prefix.  Bounded: on timeout the error is latched and the partial sum used.
__device__ unsigned long long lookback(unsigned long long *status_arr, int t, int t0,
                                       unsigned long long agg, int *err) {
  if (t == t0) {
    atom_u64(status_arr[t]).store(FLAG_PRE | agg, cuda::memory_order_release);
    return 0;
  }
  atom_u64(status_arr[t]).store(FLAG_AGG | agg, cuda::memory_order_release);
  unsigned long long excl = 0;
  int j = t - 1;
  long long spins = 0;
  unsigned ns = 8;
  while (true) {
    const unsigned long long s = atom_u64(status_arr[j]).load(cuda::memory_order_acquire);
    const unsigned long long f = s & FLAG_MASK;
    if (f == FLAG_PRE) {
      excl += s & VAL_MASK;
      break;
    }
    if (f == FLAG_AGG) {
      excl += s & VAL_MASK;
      if (j == t0) break;  // cannot happen (first tile publishes a prefix)
      --j;
      continue;
    }
    if (++spins > SPIN_LIMIT / 64) {
      latch(err, LCS_ERR_TIMEOUT);
      break;
    }
    __nanosleep(ns);
    ns = ns < 256 ? ns * 2 : 256;
  }
  atom_u64(status_arr[t]).store(FLAG_PRE | (excl + agg), cuda::memory_order_release);
  return excl;
}

// ---------------------------------------------------------------- step kernel

__device__ __forceinline__ void load_rec(const Rec &R, int64_t i, double x[3], double v[3],
                                         double &tau, uint32_t &id, int img[3], double tau_c) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    x[s] = R.x[s][i];
    v[s] = R.v[s][i];
    img[s] = R.img[s] ? R.img[s][i] : 0;
  }
  tau = R.tau ? R.tau[i] : tau_c;
  id = R.id[i];
}

__device__ __forceinline__ void store_rec(const Rec &R, int64_t i, const double x[3],
                                          const double v[3], double tau, uint32_t id,
                                          const int img[3]) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    R.x[s][i] = x[s];
    R.v[s][i] = v[s];
    if (R.img[s]) R.img[s][i] = img[s];
  }
  if (R.tau) R.tau[i] = tau;
  R.id[i] = id;
}

// One Heun step of Eqs. (5)-(6) (f = 1, gravity g) with periodic wrap, in FP64.
__device__ __forceinline__ void heun_step64(const StepArgs &a, double x[3], double v[3],
                                          double tau, int img[3], int &bad) {
  const Geom &g = a.geo;
  const double itau = 1.0 / tau;
  double u1[3], a1[3], xs[3], vs[3], u2[3];
  interp64(a.field, g, x[0], x[1], x[2], u1[0], u1[1], u1[2]);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    a1[s] = (u1[s] - v[s]) * itau + a.g[s];
    xs[s] = x[s] + a.dt * v[s];
    vs[s] = v[s] + a.dt * a1[s];
  }
  interp64(a.field, g, xs[0], xs[1], xs[2], u2[0], u2[1], u2[2]);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double a2 = (u2[s] - vs[s]) * itau + a.g[s];
    double xn = x[s] + a.half_dt * (v[s] + vs[s]);
    const double vn = v[s] + a.half_dt * (a1[s] + a2);
    if (!(fabs(xn - x[s]) < 0.5 * g.L)) bad |= fabs(xn) <= 1e300 ? 2 : 1;
    if (!isfinite(vn)) bad |= 1;
    if (xn >= g.L) {
      xn -= g.L;
      img[s] += 1;
    } else if (xn < 0.0) {
      xn += g.L;
      img[s] -= 1;
    }
    if (xn == g.L) xn = 0.0;
    x[s] = xn;
    v[s] = vn;
  }
}

// Destination direction bin (0..26, 13 = stay) of a particle at x from
// segment `seg`; -1 if the destination is not a neighbour.
__device__ __forceinline__ int dest_bin(const Geom &g, int seg, const double x[3]) {
  const int ps[3] = {seg % g.P[0], (seg / g.P[0]) % g.P[1], seg / (g.P[0] * g.P[1])};
  int bin = 0, mul = 1;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    // floor of the correctly rounded product x N/L (x >= 0 after the wrap),
    // taken from its fixed-point form without the FP64 floor
    int c = (int)(d_to_fix52(__dmul_rn(x[s], g.inv_dx)) >> 52);
    c = min(max(c, 0), g.N - 1);
    const int dc = dir_comp(ps[s], c / g.W[s], g.P[s]);
    if (dc == 2) return -1;
    bin += (dc + 1) * mul;
    mul *= 3;
  }
  return bin;
}

template <int KIND>
__global__ void __launch_bounds__(STEP_BLOCK) k_step(StepArgs a) {
  __shared__ int s_tile;
  __shared__ unsigned s_warp[STEP_BLOCK / 32];
  __shared__ unsigned long long s_excl;
  __shared__ int s_hist[NBIN];
  const int ph = *a.m.phase;
  const Rec A = a.buf[ph], B = a.buf[ph ^ 1];
  const int64_t *baseA = a.m.lay_base[ph];
  const int64_t *baseB = a.m.lay_base[ph ^ 1];
  const int64_t *capB = a.m.lay_cap[ph ^ 1];
  const int P = a.geo.Ptot;
  const int total = a.m.tile_off[P];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.m.tile_counter, 1u);
    if (threadIdx.x < NBIN) s_hist[threadIdx.x] = 0;
    __syncthreads();
    const int tile = s_tile;
    if (tile >= total) break;
    const int seg = find_segment(a.m.tile_off, P, tile);
    const int t0 = a.m.tile_off[seg];
    const int ntile = a.m.tile_off[seg + 1] - t0;
    const int jt = tile - t0;
    const int64_t cnt = a.m.cnt[seg];
    const int64_t l0 = (int64_t)jt * STEP_TILE + (int64_t)threadIdx.x * STEP_ITEMS;
    const int64_t bA = baseA[seg];

    double x[STEP_ITEMS][3], v[STEP_ITEMS][3], tau[STEP_ITEMS];
    uint32_t id[STEP_ITEMS];
    int img[STEP_ITEMS][3], bin[STEP_ITEMS];
    unsigned packed = 0;
    int bad = 0;
#pragma unroll
    for (int k = 0; k < STEP_ITEMS; ++k) {
      bin[k] = -2;  // invalid item
      if (l0 + k < cnt) {
        load_rec(A, bA + l0 + k, x[k], v[k], tau[k], id[k], img[k], a.tau_const);
        if (KIND == FK_F64) heun_step64(a, x[k], v[k], tau[k], img[k], bad);
        else heun_step_df<KIND>(a, x[k], v[k], tau[k], img[k], bad);
        int b = dest_bin(a.geo, seg, x[k]);
        if (b < 0) {
          bad |= 2;
          b = BIN_STAY;  // keep it in place; the error is latched
        }
        bin[k] = b;
        if (b == BIN_STAY) {
          packed += 1u << 16;
        } else {
          packed += 1u;
          atomicAdd(&s_hist[b], 1);
        }
      }
    }
    if (bad & 1) latch(a.m.status, LCS_ERR_NONFINITE);
    if (bad & 2) latch(a.m.status, LCS_ERR_DISPLACEMENT);

    // block exclusive scan of the packed (stay << 16 | mig) counts
    unsigned incl = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned wv = lane < STEP_BLOCK / 32 ? s_warp[lane] : 0u;
      unsigned wi = wv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < STEP_BLOCK / 32) s_warp[lane] = wi - wv;  // exclusive warp offsets
      if (lane == STEP_BLOCK / 32 - 1) {
        const unsigned long long agg = pack_sm(wi >> 16, wi & 0xffffu);
        const unsigned long long ex = lookback(a.m.tile_status, tile, t0, agg, a.m.status);
        s_excl = ex;
        if (jt == ntile - 1) {
          const unsigned long long inc = ex + agg;
          a.m.stay_tot[seg] = (int64_t)(inc >> 31);
          a.m.mig_tot[seg] = (int64_t)(inc & ((1ull << 31) - 1));
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < NBIN && threadIdx.x != BIN_STAY && s_hist[threadIdx.x])
      atomicAdd(&a.m.bincnt[seg * NBIN + threadIdx.x], s_hist[threadIdx.x]);

    const unsigned excl = incl - packed + s_warp[warp];
    int64_t stay_pos = (int64_t)(s_excl >> 31) + (excl >> 16);
    int64_t mig_pos = (int64_t)(s_excl & ((1ull << 31) - 1)) + (excl & 0xffffu);
    const int64_t bB = baseB[seg], cB = capB[seg];
#pragma unroll
    for (int k = 0; k < STEP_ITEMS; ++k) {
      if (bin[k] == -2) continue;
      if (bin[k] == BIN_STAY) {
        if (stay_pos < cB) {
          store_rec(B, bB + stay_pos, x[k], v[k], tau[k], id[k], img[k]);
        } else {
          latch(a.m.status, LCS_ERR_CAPACITY);
        }
        ++stay_pos;
      } else {
        const int64_t o = bA + mig_pos;
        store_rec(a.pack, o, x[k], v[k], tau[k], id[k], img[k]);
        a.pack_bin[o] = (uint8_t)bin[k];
        ++mig_pos;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_step(const StepArgs &a, FieldKind kind, int grid, cudaStream_t st) {
  switch (kind) {
    case FK_F64: k_step<FK_F64><<<grid, STEP_BLOCK, 0, st>>>(a); break;
    case FK_F32: k_step<FK_F32><<<grid, STEP_BLOCK, 0, st>>>(a); break;
    case FK_BF16: k_step<FK_BF16><<<grid, STEP_BLOCK, 0, st>>>(a); break;
    case FK_DF: k_step<FK_DF><<<grid, STEP_BLOCK, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int step_kernel_occupancy(FieldKind kind) {
  int n = 0;
  switch (kind) {
    case FK_F64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<FK_F64>, STEP_BLOCK, 0); break;
    case FK_F32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<FK_F32>, STEP_BLOCK, 0); break;
    case FK_BF16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<FK_BF16>, STEP_BLOCK, 0); break;
    case FK_DF: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<FK_DF>, STEP_BLOCK, 0); break;
    default: break;
  }
  return n;
}

// ---------------------------------------------------------------- finish

// Per destination d: arrival offsets of every (source, direction) pair in
// source order after the stayers, the new count, and the next layout.
__global__ void __launch_bounds__(1024) k_finish(StepArgs a) {
  const Geom &g = a.geo;
  const int P = g.Ptot;
  const int ph = *a.m.phase;
  const int64_t *capB = a.m.lay_cap[ph ^ 1];
  for (int d = threadIdx.x; d < P; d += blockDim.x) {
    const int pd[3] = {d % g.P[0], (d / g.P[0]) % g.P[1], d / (g.P[0] * g.P[1])};
    int src[NBIN - 1], bn[NBIN - 1], n = 0;
    for (int b = 0; b < NBIN; ++b) {
      if (b == BIN_STAY) continue;
      const int dir[3] = {b % 3 - 1, (b / 3) % 3 - 1, b / 9 - 1};
      int ps[3], ok = 1;
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        ps[s] = ((pd[s] - dir[s]) % g.P[s] + g.P[s]) % g.P[s];
        if (dir_comp(ps[s], pd[s], g.P[s]) != dir[s]) ok = 0;
      }
      if (!ok) continue;
      const int s_id = ps[0] + g.P[0] * (ps[1] + g.P[1] * ps[2]);
      if (s_id == d) continue;
      // insertion by source id (each source appears once)
      int j = n++;
      while (j > 0 && src[j - 1] > s_id) {
        src[j] = src[j - 1];
        bn[j] = bn[j - 1];
        --j;
      }
      src[j] = s_id;
      bn[j] = b;
    }
    int64_t off = a.m.stay_tot[d];
    for (int j = 0; j < n; ++j) {
      const int e = src[j] * NBIN + bn[j];
      a.m.off_in[e] = off;
      off += a.m.bincnt[e];
      a.m.bincnt[e] = 0;
    }
    a.m.stay_tot[d] = 0;
    if (off > capB[d]) latch(a.m.status, LCS_ERR_CAPACITY);
    a.m.cnt[d] = off;
  }
  __syncthreads();
  layout_from_counts(P, a.m.cnt, a.m.cstart, a.m.tile_off, a.m.stile_off, a.m.next_base,
                     a.m.next_cap);
}

cudaError_t launch_finish(const StepArgs &a, cudaStream_t st) {
  k_finish<<<1, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- unpack

// One block per source subdomain: place its packed leavers, in pack order,
// after the stayers of their destination (offsets from k_finish), keeping
// the order within each (source, direction) pair.
__global__ void __launch_bounds__(256) k_unpack(StepArgs a) {
  __shared__ int s_wc[8][NBIN];
  __shared__ int s_run[NBIN];
  const Geom &g = a.geo;
  const int s = blockIdx.x;
  const int ph = *a.m.phase;
  const Rec B = a.buf[ph ^ 1];
  const int64_t bA = a.m.lay_base[ph][s];
  const int64_t *baseB = a.m.lay_base[ph ^ 1];
  const int64_t *capB = a.m.lay_cap[ph ^ 1];
  const int64_t nm = a.m.mig_tot[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ps[3] = {s % g.P[0], (s / g.P[0]) % g.P[1], s / (g.P[0] * g.P[1])};
  if (threadIdx.x < NBIN) s_run[threadIdx.x] = 0;
  for (int i = threadIdx.x; i < 8 * NBIN; i += blockDim.x) (&s_wc[0][0])[i] = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nm; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const bool valid = i < nm;
    const int b = valid ? a.pack_bin[bA + i] : 255;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(peers & ((1u << lane) - 1));
    if (valid && rank == 0) s_wc[warp][b] = __popc(peers);
    __syncthreads();
    int woff = 0;
    if (valid) {
      woff = s_run[b];
      for (int w = 0; w < warp; ++w) woff += s_wc[w][b];
    }
    __syncthreads();
    if (threadIdx.x < NBIN) {
      int t = 0;
      for (int w = 0; w < 8; ++w) {
        t += s_wc[w][threadIdx.x];
        s_wc[w][threadIdx.x] = 0;
      }
      s_run[threadIdx.x] += t;
    }
    if (valid) {
      const int dir[3] = {b % 3 - 1, (b / 3) % 3 - 1, b / 9 - 1};
      int pd[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) pd[q] = (ps[q] + dir[q] + g.P[q]) % g.P[q];
      const int d = pd[0] + g.P[0] * (pd[1] + g.P[1] * pd[2]);
      const int64_t rel = a.m.off_in[s * NBIN + b] + woff + rank;
      if (rel < capB[d]) {
        copy_rec(a.pack, bA + i, B, baseB[d] + rel);
      } else {
        latch(a.m.status, LCS_ERR_CAPACITY);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) a.m.mig_tot[s] = 0;
}

cudaError_t launch_unpack(const StepArgs &a, cudaStream_t st) {
  k_unpack<<<a.geo.Ptot, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- flip

// The old input buffer becomes the next output with the layout from
// k_finish; the output becomes the input.
__global__ void k_flip(StepArgs a) {
  const int ph = *a.m.phase;
  for (int d = threadIdx.x; d < a.geo.Ptot; d += blockDim.x) {
    a.m.lay_base[ph][d] = a.m.next_base[d];
    a.m.lay_cap[ph][d] = a.m.next_cap[d];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *a.m.phase = ph ^ 1;
    *a.m.tile_counter = 0u;
  }
}

cudaError_t launch_flip(const StepArgs &a, cudaStream_t st) {
  k_flip<<<1, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lcs
