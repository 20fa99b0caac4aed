// Hand-written adjoint of the particle step, with checkpointing.
//
// Forward (Sec. 2.2, Eqs. 5-6 with f = 1, Heun):
//   A1 = (U(X) - V)/tau + g,  X* = X + dt V,  V* = V + dt A1,
//   A2 = (U(X*) - V*)/tau + g,
//   X' = X + dt/2 (V + V*),   V' = V + dt/2 (A1 + A2).
// Reverse of one step, from lamX', lamV' (mu1 = lamA1/tau, mu2 = lamA2/tau):
//   lamA2 = lamA1 = dt/2 lamV',      mu2 = lamA2/tau,
//   lamV* = dt/2 lamX' - mu2,        lamX* = J(X*)^T mu2,
//   lamA1 += dt lamV*,               mu1 = lamA1/tau,
//   lamX = lamX' + lamX* + J(X)^T mu1,
//   lamV = lamV' + dt lamX' - mu2 + dt lamX* - mu1,
//   dL/dU += interp(X*)^T mu2 + interp(X)^T mu1,
// with J = dU/dX of the trilinear map (piecewise constant per cell) and
// interp^T the transpose of the 8-corner weighted sum.  The periodic wrap is
// the identity for the adjoint (losses use unwrapped positions); migration
// and sort only permute storage.
//
// Precision: the stage coordinates (which cell, hence which piece of the
// piecewise-linear map) are recomputed with exactly the forward's code, so
// the adjoint differentiates the same pieces the forward used.  mu1, mu2,
// dt lamX' and J^T mu are computed in float-float (FP32 rounding there,
// repeated over hundreds of steps, shows up at ~1e-6 in the gradients);
// the scatter values w_q mu_c are FP32 (independent per contribution);
// lamX, lamV are kept in FP64 and dL/dU is accumulated with FP64 atomics.
#include <algorithm>

#include "lcs_physics.cuh"

namespace lcs {

// Checkpoint: the live particles of the input buffer, compacted, in storage order.
__global__ void k_tape_store(StepArgs a, TapeSlot t, int64_t np) {
  const int ph = *a.m.phase;
  const Rec A = a.buf[ph];
  const int64_t *base = a.m.lay_base[ph];
  const int P = a.geo.Ptot;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = P;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.m.cstart[mid] <= i) lo = mid; else hi = mid;
    }
    const int64_t slot = base[lo] + (i - a.m.cstart[lo]);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      t.x[s * np + i] = A.x[s][slot];
      t.v[s * np + i] = A.v[s][slot];
    }
    if (t.tau) t.tau[i] = A.tau[slot];
    t.id[i] = A.id[slot];
  }
}

// Re-run `len` steps from a checkpoint with the forward's own arithmetic,
// storing the state at the start of every step: states[(j*6 + c)*np + i]
// (c < 3: fixed-point positions, c >= 3: velocity float pairs, as 64-bit
// words).
__device__ __forceinline__ unsigned long long bits_of_df(df v) {
  return ((unsigned long long)__float_as_uint(v.l) << 32) | __float_as_uint(v.h);
}
__device__ __forceinline__ df df_of_bits(unsigned long long b) {
  return {__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32))};
}

template <int KIND>
__global__ void k_recompute(StepArgs a, TapeSlot t, unsigned long long *states, int len,
                            int64_t np) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  long long x[3];
  df v[3];
  int img[3] = {0, 0, 0};
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    x[s] = t.x[s * np + i];
    v[s] = df_from2(t.v[s * np + i]);
  }
  const double tau = t.tau ? t.tau[i] : a.tau_const;
  for (int j = 0; j < len; ++j) {
    unsigned long long *st = states + (int64_t)j * 6 * np;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      st[s * np + i] = (unsigned long long)x[s];
      st[(3 + s) * np + i] = bits_of_df(v[s]);
    }
    int bad = 0;
    if (KIND == FK_F64) heun_step64(a, x, v, tau, img, bad);
    else if (KIND == FK_DF) heun_step_df<KIND>(a, x, v, tau, img, bad);
    else heun_step_lo<KIND>(a, x, v, tau, img, bad);
  }
}

// lam in storage order <-> lam in particle-id order (6 arrays of np).
__global__ void k_lam_permute(const uint32_t *id, const double *src, double *dst, int64_t np,
                              int to_storage, int *status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t p = id[i];
    if (p >= np) {  // ids must be 0..np-1 for id-ordered gradients
      latch(status, LCS_ERR_ARG);
      continue;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      if (to_storage) dst[c * np + i] = src[c * np + p];
      else dst[c * np + p] = src[c * np + i];
    }
  }
}

// One interpolation stencil in FP32 for the adjoint.
struct AStage {
  uint32_t cell[8];
  float wx[2], wy[2], wz[2];    // FP32 weights (scatter values)
  df dwx[2], dwy[2], dwz[2];    // float-pair weights (J^T mu)
};

__device__ __forceinline__ void astage_from_fix(const long long q[3], int N, AStage &S) {
  int i0[3];
  float t[3];
  df w1[3][2];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const Axis ax = axis_from_fix(q[s]);
    i0[s] = wrap_cell(ax.i0, N);
    t[s] = __fadd_rn(ax.th, ax.tl);
    w1[s][0] = {__fsub_rn(1.0f, ax.th), -ax.tl};
    w1[s][1] = {ax.th, ax.tl};
  }
  S.dwx[0] = w1[0][0], S.dwx[1] = w1[0][1];
  S.dwy[0] = w1[1][0], S.dwy[1] = w1[1][1];
  S.dwz[0] = w1[2][0], S.dwz[1] = w1[2][1];
  S.wx[0] = 1.0f - t[0], S.wx[1] = t[0];
  S.wy[0] = 1.0f - t[1], S.wy[1] = t[1];
  S.wz[0] = 1.0f - t[2], S.wz[1] = t[2];
  const uint32_t ii[2] = {(uint32_t)i0[0], (uint32_t)(i0[0] + 1 == N ? 0 : i0[0] + 1)};
  const uint32_t jj[2] = {(uint32_t)i0[1] * N, (uint32_t)(i0[1] + 1 == N ? 0 : i0[1] + 1) * N};
  const uint32_t kk[2] = {(uint32_t)i0[2] * N * N,
                          (uint32_t)(i0[2] + 1 == N ? 0 : i0[2] + 1) * N * N};
#pragma unroll
  for (int q = 0; q < 8; ++q) S.cell[q] = ii[q >> 2] + jj[(q >> 1) & 1] + kk[q & 1];
}

__device__ __forceinline__ void astage_from_pos64(const double p[3], double inv_dx, int N,
                                                  AStage &S) {
  int i0[3];
  float t[3];
  df w1[3][2];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    double tt;
    axis64(p[s], inv_dx, N, i0[s], tt);
    const df td = split_d(tt), od = split_d(1.0 - tt);
    t[s] = td.h;
    w1[s][0] = od;
    w1[s][1] = td;
  }
  S.dwx[0] = w1[0][0], S.dwx[1] = w1[0][1];
  S.dwy[0] = w1[1][0], S.dwy[1] = w1[1][1];
  S.dwz[0] = w1[2][0], S.dwz[1] = w1[2][1];
  S.wx[0] = 1.0f - t[0], S.wx[1] = t[0];
  S.wy[0] = 1.0f - t[1], S.wy[1] = t[1];
  S.wz[0] = 1.0f - t[2], S.wz[1] = t[2];
  const uint32_t ii[2] = {(uint32_t)i0[0], (uint32_t)(i0[0] + 1 == N ? 0 : i0[0] + 1)};
  const uint32_t jj[2] = {(uint32_t)i0[1] * N, (uint32_t)(i0[1] + 1 == N ? 0 : i0[1] + 1) * N};
  const uint32_t kk[2] = {(uint32_t)i0[2] * N * N,
                          (uint32_t)(i0[2] + 1 == N ? 0 : i0[2] + 1) * N * N};
#pragma unroll
  for (int q = 0; q < 8; ++q) S.cell[q] = ii[q >> 2] + jj[(q >> 1) & 1] + kk[q & 1];
}

// Field record of one cell as float pairs (hi, lo) per component; for FP32
// and BF16 storage lo = 0.
template <int KIND>
__device__ __forceinline__ void field_pair(const void *field, uint32_t cell, float h[3],
                                           float l[3]) {
  if (KIND == FK_DF) {
    float4 A, B;
    ldg_cell32((const float4 *)field + 2 * (size_t)cell, A, B);
    h[0] = A.x, h[1] = A.y, h[2] = A.z, l[0] = A.w, l[1] = B.x, l[2] = B.y;
  } else if (KIND == FK_F64) {
    double2 A, B;
    ldg_cell32((const double2 *)field + 2 * (size_t)cell, A, B);
    const df u = split_d(A.x), v = split_d(A.y), w = split_d(B.x);
    h[0] = u.h, h[1] = v.h, h[2] = w.h, l[0] = u.l, l[1] = v.l, l[2] = w.l;
  } else if (KIND == FK_F32) {
    const float4 A = __ldg((const float4 *)field + cell);
    h[0] = A.x, h[1] = A.y, h[2] = A.z, l[0] = l[1] = l[2] = 0.f;
  } else {
    const uint2 p = __ldg((const uint2 *)field + cell);
    h[0] = __uint_as_float((p.x & 0xffffu) << 16);
    h[1] = __uint_as_float(p.x & 0xffff0000u);
    h[2] = __uint_as_float((p.y & 0xffffu) << 16);
    l[0] = l[1] = l[2] = 0.f;
  }
}

// J(X)^T mu for one stage in float-float, and the scatter values w_q mu_c
// (FP32, q-major).  With G_q = sum_c mu_c U_c[q] (the field at corner q
// projected on mu), the trilinear map gives
//   (J^T mu)_x = N/L sum_{b,d} wy_b wz_d (G_{1bd} - G_{0bd})   (and y, z alike).
// G_q is formed from exact products (fma error terms) and two_sum, so its
// differences keep ~46 bits even where neighbouring corners nearly cancel.
template <int KIND>
__device__ __forceinline__ void stage_adjoint(const void *field, const AStage &S, df inv_dx,
                                              const df mu[3], df jt[3], float val[24]) {
  df G[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float h[3], l[3];
    field_pair<KIND>(field, S.cell[q], h, l);
    const float w = S.wx[q >> 2] * S.wy[(q >> 1) & 1] * S.wz[q & 1];
    float sum = 0.f, err = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      val[q * 3 + c] = w * mu[c].h;
      const float P = __fmul_rn(mu[c].h, h[c]);
      float e = __fmaf_rn(mu[c].h, h[c], -P);
      e = __fmaf_rn(mu[c].h, l[c], e);
      e = __fmaf_rn(mu[c].l, h[c], e);
      if (c == 0) {
        sum = P;
        err = e;
      } else {
        const df t2 = two_sum(sum, P);
        sum = t2.h;
        err = __fadd_rn(err, __fadd_rn(t2.l, e));
      }
    }
    G[q] = fast_two_sum(sum, err);
  }
  df jx = {0.f, 0.f}, jy = {0.f, 0.f}, jz = {0.f, 0.f};
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int qx1 = 4 + u * 2 + r, qx0 = u * 2 + r;
      const int qy1 = u * 4 + 2 + r, qy0 = u * 4 + r;
      const int qz1 = u * 4 + r * 2 + 1, qz0 = u * 4 + r * 2;
      jx = df_add(jx, df_mul(df_mul(S.dwy[u], S.dwz[r]), df_add(G[qx1], df_neg(G[qx0]))));
      jy = df_add(jy, df_mul(df_mul(S.dwx[u], S.dwz[r]), df_add(G[qy1], df_neg(G[qy0]))));
      jz = df_add(jz, df_mul(df_mul(S.dwx[u], S.dwy[r]), df_add(G[qz1], df_neg(G[qz0]))));
    }
  jt[0] = df_mul(jx, inv_dx), jt[1] = df_mul(jy, inv_dx), jt[2] = df_mul(jz, inv_dx);
}

// Scatter-add of the 24 values of a stencil into dL/dU with warp aggregation:
// lanes whose stencils share the same 8 cells (same base cell) are summed by
// the group's lowest lane, which alone issues the 24 FP64 atomics.
__device__ __forceinline__ void scatter_agg(double *gU, int64_t ncell, const AStage &S,
                                            float val[24], bool valid) {
  const unsigned lane = threadIdx.x & 31;
  const uint32_t key = valid ? S.cell[0] : 0xffffffffu - lane;  // invalid lanes stay alone
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(peers) - 1;
  const bool is_leader = (int)lane == leader;
  unsigned others = is_leader ? (peers & ~(1u << lane)) : 0u;
  float acc[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = val[k];
  while (__any_sync(0xffffffffu, others != 0)) {
    const bool pull = others != 0;
    const int src = pull ? __ffs(others) - 1 : (int)lane;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      const float o = __shfl_sync(0xffffffffu, val[k], src);
      if (pull) acc[k] += o;
    }
    if (pull) others &= others - 1;
  }
  if (valid && is_leader) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        atomicAdd(gU + (int64_t)c * ncell + S.cell[q], (double)acc[q * 3 + c]);
  }
}

struct AdjArgs {
  StepArgs a;
  const unsigned long long *state;  // [6][np] state at the start of this step (k_recompute)
  const double *tau;    // [np] or nullptr
  double *lam;          // [6][np] lamX, lamV in the same storage order (in/out)
  double *gU;           // [3][N^3]
  int64_t np;
};

template <int KIND>
__global__ void __launch_bounds__(256) k_adjoint(AdjArgs p) {
  const StepArgs &a = p.a;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = i < p.np;
  const int64_t np = p.np, ii = valid ? i : 0;
  const int N = a.geo.N;
  long long q1[3];
  df v[3];
  double lx[3], lv[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    q1[s] = (long long)p.state[s * np + ii];
    v[s] = df_of_bits(p.state[(3 + s) * np + ii]);
    lx[s] = p.lam[s * np + ii];
    lv[s] = p.lam[(3 + s) * np + ii];
  }
  const double tau = p.tau ? p.tau[ii] : a.tau_const;
  const df inv_dx = split_d(a.geo.inv_dx);
  // the forward's stage coordinates
  AStage S1, S2;
  if (KIND == FK_F64) {
    double x[3], xs[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      x[s] = pos_of_fix(q1[s], a.geo);
      xs[s] = predictor64(x[s], vel_of_df(v[s]), a.dt);
    }
    astage_from_pos64(x, a.geo.inv_dx, N, S1);
    astage_from_pos64(xs, a.geo.inv_dx, N, S2);
  } else {
    const df cx = {a.dfk[4], a.dfk[5]};
    long long q2[3];
#pragma unroll
    for (int s = 0; s < 3; ++s)
      q2[s] = KIND == FK_DF ? fix_stage2(q1[s], v[s], cx)
                            : fix_stage2_lo(q1[s], v[s].h, a.dfk[4]);
    astage_from_fix(q1, N, S1);
    astage_from_fix(q2, N, S2);
  }
  // float-float for the terms that are O(dt/tau) of the adjoint state
  // (mu1, mu2, dt lamX'): their rounding would otherwise accumulate over the
  // steps; J^T mu is O(dt |grad U|) smaller and stays FP32.
  const df itd = df_recip(split_d(tau));
  const df dtd = {a.dfk[0], a.dfk[1]}, hdt = {a.dfk[2], a.dfk[3]};
  const df c2 = df_mul(hdt, itd);  // dt / (2 tau)
  df mu2[3], mu1[3], dlx[3], jt2[3], jt1[3];
  float val[24];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const df LX = split_d(lx[s]), LV = split_d(lv[s]);
    mu2[s] = df_mul(c2, LV);                                // lamA2 / tau
    dlx[s] = df_mul(dtd, LX);                               // dt lamX'
    // lamA1 = dt/2 lamV' + dt (dt/2 lamX' - mu2) ; mu1 = lamA1 / tau
    const df lA1 = df_add(df_mul(hdt, LV), df_mul(dtd, df_add(df_scale2(dlx[s], 0.5f),
                                                              df_neg(mu2[s]))));
    mu1[s] = df_mul(lA1, itd);
  }
  stage_adjoint<KIND>(a.field, S2, inv_dx, mu2, jt2, val);
  scatter_agg(p.gU, (int64_t)N * N * N, S2, val, valid);
  stage_adjoint<KIND>(a.field, S1, inv_dx, mu1, jt1, val);
  scatter_agg(p.gU, (int64_t)N * N * N, S1, val, valid);
  if (!valid) return;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    // lamX = lamX' + J(X*)^T mu2 + J(X)^T mu1
    p.lam[s * np + i] = __dadd_rn(lx[s], df_to_double(df_add(jt2[s], jt1[s])));
    // lamV = lamV' + dt lamX' - mu2 - mu1 + dt J(X*)^T mu2
    const df inc = df_add(df_add(dlx[s], df_neg(df_add(mu2[s], mu1[s]))), df_mul(dtd, jt2[s]));
    p.lam[(3 + s) * np + i] = __dadd_rn(lv[s], df_to_double(inc));
  }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_tape_store(const StepArgs &a, const TapeSlot &t, int64_t np, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, device_sms() * 8));
  k_tape_store<<<grid, 256, 0, st>>>(a, t, np);
  return cudaGetLastError();
}

cudaError_t launch_recompute(const StepArgs &a, FieldKind kind, const TapeSlot &t,
                             unsigned long long *states, int len, int64_t np, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, (np + 127) / 128);
  switch (kind) {
    case FK_F64: k_recompute<FK_F64><<<grid, 128, 0, st>>>(a, t, states, len, np); break;
    case FK_DF: k_recompute<FK_DF><<<grid, 128, 0, st>>>(a, t, states, len, np); break;
    case FK_F32: k_recompute<FK_F32><<<grid, 128, 0, st>>>(a, t, states, len, np); break;
    case FK_BF16: k_recompute<FK_BF16><<<grid, 128, 0, st>>>(a, t, states, len, np); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_lam_permute(const uint32_t *id, const double *src, double *dst, int64_t np,
                               int to_storage, int *status, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, device_sms() * 8));
  k_lam_permute<<<grid, 256, 0, st>>>(id, src, dst, np, to_storage, status);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const StepArgs &a, FieldKind kind, const unsigned long long *state,
                           const double *tau, double *lam, double *gU, int64_t np,
                           cudaStream_t st) {
  AdjArgs p{a, state, tau, lam, gU, np};
  const int grid = (int)std::max<int64_t>(1, (np + 255) / 256);
  switch (kind) {
    case FK_F64: k_adjoint<FK_F64><<<grid, 256, 0, st>>>(p); break;
    case FK_DF: k_adjoint<FK_DF><<<grid, 256, 0, st>>>(p); break;
    case FK_F32: k_adjoint<FK_F32><<<grid, 256, 0, st>>>(p); break;
    case FK_BF16: k_adjoint<FK_BF16><<<grid, 256, 0, st>>>(p); break;
  }
  return cudaGetLastError();
}

}  // namespace lcs
