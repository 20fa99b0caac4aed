/*
 * CPU oracle for the Lagrangian particle hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded FP64 C.  It shares no code with the CUDA
 * library and is used only by the tests, by the smoke check and by the
 * timed CPU baseline of the benchmark.  Every function follows the paper
 * (Tominaga & Onishi, "LCS.jl", arXiv 2604.11008) step by step:
 *
 *   orc_interp        trilinear interpolation from the eight surrounding
 *                     cell-centre values (Sec. 2.2, last paragraph)
 *   orc_advance       particle ODE dX/dt = V, dV/dt = -(f/tau_p)(V - U(X, t))
 *                     (Eqs. 5-6) with f = 1 (Stokes drag) or the nonlinear
 *                     drag factor of Eq. (7), plus an optional
 *                     constant gravity g, in a frozen field or one linear in
 *                     time between two snapshots, advanced with the two-stage
 *                     second-order Runge-Kutta method of Sec. 2.2 read as
 *                     Heun's method, then periodic wrap into [0, L)
 *                     (periodic cube of side L, Sec. 2.1)
 *   orc_keys          destination subdomain of each particle (the "mask
 *                     computation" of Sec. 2.3.3, generalised from 0/1 to a
 *                     destination id) and its cell sort key
 *   orc_migrate       the sequential per-direction-counter packing of the
 *                     original Fortran LCS (Sec. 2.3.3, second paragraph),
 *                     followed by unpack = stayers kept in order, incoming
 *                     particles appended by source subdomain (Sec. 3.2.2)
 *   orc_sort          stable sort of every subdomain segment by cell key
 *   orc_loss          mean squared distance of final (unwrapped) positions
 *                     to targets
 *   orc_adjoint       reverse-mode derivative of orc_advance, written out
 *                     from the forward definitions above
 *   orc_round_f32/bf16  round-to-nearest-even of FP64 values to FP32 / BF16
 *   orc_pair_hist     histogram of pair separations (minimum image in the
 *                     periodic box), the counts behind the radial
 *                     distribution function g(r) of Sec. 3 (particle-phase
 *                     validation), by brute force over all pairs
 *
 * Layouts: field [3][N][N][N] float64 with cell (i,j,k) at i + N*(j + N*k),
 * x fastest; particle data structure-of-arrays float64.
 * Compile with -ffp-contract=off so that x86 and Arm give identical bits.
 * Built a second time with -fopenmp for the timed CPU baseline on all host
 * cores: the particle loop of orc_advance then runs in parallel (particles
 * are independent, Eqs. 5-6 have no coupling term); the arithmetic of every
 * particle is the same, so both builds give identical bits.  Migration and
 * sort stay sequential.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_DISPLACEMENT 1
#define ORC_ERR_ARG 2
#define ORC_ERR_NOMEM 3

static int64_t wrap_index(int64_t i, int64_t n) {
  int64_t r = i % n;
  return r < 0 ? r + n : r;
}

/* Trilinear interpolation (Sec. 2.2): with s = x/dx - 1/2, i0 = floor(s) and
 * t = s - i0 on each axis, U(X) = sum over the eight corners (i0+a, j0+b,
 * k0+c), a,b,c in {0,1}, of wx[a] wy[b] wz[c] U[corner], wx = (1-t, t).
 * Cell-centre indices wrap modulo N (periodic domain).  inv_dx = N/L. */
void orc_interp(const double *field, int N, double inv_dx, double x, double y, double z,
                double u[3]) {
  const double pos[3] = {x, y, z};
  int64_t lo[3], hi[3];
  double w[3][2];
  for (int s = 0; s < 3; ++s) {
    double g = pos[s] * inv_dx - 0.5;
    double f = floor(g);
    double t = g - f;
    lo[s] = wrap_index((int64_t)f, N);
    hi[s] = wrap_index((int64_t)f + 1, N);
    w[s][0] = 1.0 - t;
    w[s][1] = t;
  }
  const int64_t nn = (int64_t)N * N * N;
  for (int c = 0; c < 3; ++c) {
    double acc = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 2; ++d) {
          int64_t i = a ? hi[0] : lo[0];
          int64_t j = b ? hi[1] : lo[1];
          int64_t k = d ? hi[2] : lo[2];
          double wt = w[0][a] * w[1][b] * w[2][d];
          acc += wt * field[c * nn + i + (int64_t)N * (j + (int64_t)N * k)];
        }
    u[c] = acc;
  }
}

void orc_interp_many(const double *field, int N, double inv_dx, int64_t n, const double *x,
                     const double *y, const double *z, double *u, double *v, double *w) {
  for (int64_t p = 0; p < n; ++p) {
    double r[3];
    orc_interp(field, N, inv_dx, x[p], y[p], z[p], r);
    u[p] = r[0];
    v[p] = r[1];
    w[p] = r[2];
  }
}

/* Fold the interpolation cell (floor indices) of one gather into h (FNV-1a
 * style), to detect runs that visit different cells. */
static uint64_t cell_hash(uint64_t h, double inv_dx, const double p[3]) {
  for (int s = 0; s < 3; ++s) {
    double f = floor(p[s] * inv_dx - 0.5);
    h = (h ^ (uint64_t)(int64_t)f) * 1099511628211ULL;
  }
  return h;
}

/* Periodic wrap into [0, L) (Sec. 2.1): one image per step; a value that
 * rounds to exactly L after adding L is mapped to 0.  Returns the image shift
 * (-1, 0, +1) applied to the unwrapped coordinate count. */
static int wrap_coord(double *x, double L) {
  int img = 0;
  if (*x >= L) {
    *x -= L;
    img = 1;
  } else if (*x < 0.0) {
    *x += L;
    img = -1;
  }
  if (*x == L) *x = 0.0;
  return img;
}

/* Drag factor f of Eq. (7) for a particle with relaxation time tp and
 * velocity relative to the fluid vrel = V - U(X), in a fluid of kinematic
 * viscosity nu, particle-to-fluid density ratio rr (Sec. 2.2):
 *   radius r from tau_p = (2/9) rr r^2 / nu,
 *   Re_p = 2 r |V - U| / nu,
 *   f = 1 + 0.15 Re_p^0.687. */
static double drag_factor(double tp, double nu, double rr, const double vrel[3]) {
  const double r = sqrt(9.0 * nu * tp / (2.0 * rr));
  const double speed = sqrt(vrel[0] * vrel[0] + vrel[1] * vrel[1] + vrel[2] * vrel[2]);
  const double re = 2.0 * r * speed / nu;
  return 1.0 + 0.15 * pow(re, 0.687);
}

/* Fluid velocity at position p and time fraction theta between two field
 * snapshots (the coupling to an evolving Eulerian field, U(X, t) of Eq. 6):
 * U = (1 - theta) U_a(p) + theta U_b(p), linear in time; U_a alone when
 * fb is NULL (frozen field). */
static void fluid_velocity(const double *fa, const double *fb, double theta, int N,
                           double inv_dx, const double p[3], double u[3]) {
  orc_interp(fa, N, inv_dx, p[0], p[1], p[2], u);
  if (!fb) return;
  double ub[3];
  orc_interp(fb, N, inv_dx, p[0], p[1], p[2], ub);
  for (int s = 0; s < 3; ++s) u[s] = (1.0 - theta) * u[s] + theta * ub[s];
}

/* Advance n particles by nsteps Heun steps of Eqs. (5)-(6):
 *   A1 = f1 (U(X) - V)/tau + g,   X* = X + dt V,   V* = V + dt A1,
 *   A2 = f2 (U(X*) - V*)/tau + g,
 *   X' = X + dt/2 (V + V*),    V' = V + dt/2 (A1 + A2),
 * then wrap X' into [0, L).  drag = 0: f1 = f2 = 1 (Stokes drag); drag = 1:
 * f1, f2 from Eq. (7) with the relative velocity of their stage (nu, rr as
 * in drag_factor).  With a second snapshot field_b (time t_b; field at
 * t_a), step k of the call starts at t = t_start + k dt and its two stages
 * see the field at t and t + dt:
 *   U1 = U(X, t),  U2 = U(X*, t + dt),  theta(t) = (t - t_a) / (t_b - t_a)
 * (field_b NULL: the frozen field).  tau may be NULL (then tau_const for all).
 * img (3*n int32, SoA) counts the periodic images crossed (may be NULL).
 * cellhash (n uint64, may be NULL) folds in the floor index of every gather,
 * so that two runs which visit different interpolation cells can be told
 * apart.  Returns ORC_ERR_DISPLACEMENT if any step moves a particle by half
 * a box or more along an axis (one periodic image per step). */
/* Stage 1 of Heun's method for one particle (Eqs. 5-6):
 *   A1 = f1 (U(X, t) - V)/tau + g,  X* = X + dt V,  V* = V + dt A1. */
static void heun_stage1(const double *field, const double *field_b, double th1, int N,
                        double inv_dx, double tp, double dt, const double *g, int drag,
                        double nu, double rr, const double x0[3], const double v0[3],
                        double a1[3], double xs[3], double vs[3]) {
  double u1[3];
  fluid_velocity(field, field_b, th1, N, inv_dx, x0, u1);
  double f1 = 1.0;
  if (drag) {
    const double rel[3] = {v0[0] - u1[0], v0[1] - u1[1], v0[2] - u1[2]};
    f1 = drag_factor(tp, nu, rr, rel);
  }
  for (int s = 0; s < 3; ++s) {
    a1[s] = f1 * (u1[s] - v0[s]) / tp + g[s];
    xs[s] = x0[s] + dt * v0[s];
    vs[s] = v0[s] + dt * a1[s];
  }
}

/* Stage 2: A2 = f2 (U(X*, t + dt) - V*)/tau + g,
 *   X' = X + dt/2 (V + V*),  V' = V + dt/2 (A1 + A2)   (X' not wrapped). */
static void heun_stage2(const double *field, const double *field_b, double th2, int N,
                        double inv_dx, double tp, double dt, const double *g, int drag,
                        double nu, double rr, const double x0[3], const double v0[3],
                        const double a1[3], const double xs[3], const double vs[3],
                        double xn[3], double vn[3]) {
  double u2[3];
  fluid_velocity(field, field_b, th2, N, inv_dx, xs, u2);
  double f2 = 1.0;
  if (drag) {
    const double rel[3] = {vs[0] - u2[0], vs[1] - u2[1], vs[2] - u2[2]};
    f2 = drag_factor(tp, nu, rr, rel);
  }
  for (int s = 0; s < 3; ++s) {
    const double a2 = f2 * (u2[s] - vs[s]) / tp + g[s];
    xn[s] = x0[s] + 0.5 * dt * (v0[s] + vs[s]);
    vn[s] = v0[s] + 0.5 * dt * (a1[s] + a2);
  }
}

static int check_model(int drag, double nu, double rr, const double *field_b, double t_a,
                       double t_b) {
  if (drag != 0 && (drag != 1 || !(nu > 0.0) || !(rr > 0.0))) return ORC_ERR_ARG;
  if (field_b && !(t_b > t_a)) return ORC_ERR_ARG;
  return ORC_OK;
}

int orc_advance(const double *field, int N, double L, double inv_dx, int64_t n, double *x,
                double *y, double *z, double *vx, double *vy, double *vz, const double *tau,
                double tau_const, double dt, const double *g, int nsteps, int32_t *img,
                uint64_t *cellhash, int drag, double nu, double rr, const double *field_b,
                double t_start, double t_a, double t_b) {
  int status = check_model(drag, nu, rr, field_b, t_a, t_b);
  if (status != ORC_OK) return status;
  double *X[3] = {x, y, z};
  double *V[3] = {vx, vy, vz};
  int moved_far = 0;
  for (int step = 0; step < nsteps; ++step) {
    const double t = t_start + step * dt;
    const double th1 = field_b ? (t - t_a) / (t_b - t_a) : 0.0;
    const double th2 = field_b ? (t + dt - t_a) / (t_b - t_a) : 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : moved_far)
#endif
    for (int64_t p = 0; p < n; ++p) {
      const double tp = tau ? tau[p] : tau_const;
      double x0[3], v0[3], a1[3], xs[3], vs[3], xn[3], vn[3];
      for (int s = 0; s < 3; ++s) {
        x0[s] = X[s][p];
        v0[s] = V[s][p];
      }
      if (cellhash) cellhash[p] = cell_hash(cellhash[p], inv_dx, x0);
      heun_stage1(field, field_b, th1, N, inv_dx, tp, dt, g, drag, nu, rr, x0, v0, a1, xs, vs);
      if (cellhash) cellhash[p] = cell_hash(cellhash[p], inv_dx, xs);
      heun_stage2(field, field_b, th2, N, inv_dx, tp, dt, g, drag, nu, rr, x0, v0, a1, xs, vs,
                  xn, vn);
      for (int s = 0; s < 3; ++s) {
        if (fabs(xn[s] - x0[s]) >= 0.5 * L) moved_far = 1;
        int im = wrap_coord(&xn[s], L);
        if (img) img[(int64_t)s * n + p] += im;
        X[s][p] = xn[s];
        V[s][p] = vn[s];
      }
    }
  }
  return moved_far ? ORC_ERR_DISPLACEMENT : status;
}

/* Threads of the particle loop of orc_advance: n > 0 sets them (OpenMP
 * build only); returns the number in use (1 without OpenMP). */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* The two stages of one step taken separately, for migration after each
 * stage (Sec. 3.2.2: the particles are exchanged after every Runge-Kutta
 * stage).  All arrays are (3, n) structure of arrays; the step starts at
 * time t (field_b as in orc_advance).
 * orc_stage1: from X, V compute X* (not wrapped), V* and A1.
 * orc_stage2: from X, V, X*, V*, A1 compute X', V' in place of X, V, with
 * the wrap of X' counted in img (may be NULL).  The arithmetic is exactly
 * that of orc_advance. */
int orc_stage1(const double *field, int N, double L, double inv_dx, int64_t n, const double *x,
               const double *v, const double *tau, double tau_const, double dt, const double *g,
               int drag, double nu, double rr, const double *field_b, double t, double t_a,
               double t_b, double *xs, double *vs, double *a1) {
  int status = check_model(drag, nu, rr, field_b, t_a, t_b);
  if (status != ORC_OK) return status;
  (void)L;
  const double th1 = field_b ? (t - t_a) / (t_b - t_a) : 0.0;
  for (int64_t p = 0; p < n; ++p) {
    const double tp = tau ? tau[p] : tau_const;
    double x0[3], v0[3], pa[3], px[3], pv[3];
    for (int s = 0; s < 3; ++s) {
      x0[s] = x[s * n + p];
      v0[s] = v[s * n + p];
    }
    heun_stage1(field, field_b, th1, N, inv_dx, tp, dt, g, drag, nu, rr, x0, v0, pa, px, pv);
    for (int s = 0; s < 3; ++s) {
      a1[s * n + p] = pa[s];
      xs[s * n + p] = px[s];
      vs[s * n + p] = pv[s];
    }
  }
  return ORC_OK;
}

int orc_stage2(const double *field, int N, double L, double inv_dx, int64_t n, double *x,
               double *v, const double *xs, const double *vs, const double *a1,
               const double *tau, double tau_const, double dt, const double *g, int drag,
               double nu, double rr, const double *field_b, double t, double t_a, double t_b,
               int32_t *img) {
  int status = check_model(drag, nu, rr, field_b, t_a, t_b);
  if (status != ORC_OK) return status;
  const double th2 = field_b ? (t + dt - t_a) / (t_b - t_a) : 0.0;
  for (int64_t p = 0; p < n; ++p) {
    const double tp = tau ? tau[p] : tau_const;
    double x0[3], v0[3], pa[3], px[3], pv[3], xn[3], vn[3];
    for (int s = 0; s < 3; ++s) {
      x0[s] = x[s * n + p];
      v0[s] = v[s * n + p];
      pa[s] = a1[s * n + p];
      px[s] = xs[s * n + p];
      pv[s] = vs[s * n + p];
    }
    heun_stage2(field, field_b, th2, N, inv_dx, tp, dt, g, drag, nu, rr, x0, v0, pa, px, pv,
                xn, vn);
    for (int s = 0; s < 3; ++s) {
      if (fabs(xn[s] - x0[s]) >= 0.5 * L) status = ORC_ERR_DISPLACEMENT;
      int im = wrap_coord(&xn[s], L);
      if (img) img[(int64_t)s * n + p] += im;
      x[s * n + p] = xn[s];
      v[s * n + p] = vn[s];
    }
  }
  return status;
}

/* Destination subdomain and cell sort key of every particle (Sec. 2.3.3,
 * stage 1, generalised from a 0/1 mask to a destination id).
 *   c_s  = min(floor(x_s * inv_dx), N-1)             containing cell
 *   p_s  = c_s / (N / P_s)                           subdomain coordinate
 *   dest = p_x + P_x (p_y + P_y p_z)
 * The cell key orders the cells of one subdomain brick by brick: local cell
 * l_s = c_s - p_s W_s (W_s = N/P_s), brick b_s = l_s / B, offset r_s = l_s % B,
 * nb_s = ceil(W_s / B) bricks per axis,
 *   key = ((b_z nb_y + b_y) nb_x + b_x) B^3 + (r_z B + r_y) B + r_x.
 * B = 1 gives the plain x-fastest cell order.  dest or key may be NULL. */
int orc_keys(int N, double inv_dx, const int *P, int brick, int64_t n, const double *x,
             const double *y, const double *z, int32_t *dest, int64_t *key) {
  const double *X[3] = {x, y, z};
  for (int s = 0; s < 3; ++s)
    if (P[s] <= 0 || N % P[s] != 0) return ORC_ERR_ARG;
  if (brick <= 0) return ORC_ERR_ARG;
  for (int64_t p = 0; p < n; ++p) {
    int64_t c[3], ps[3], l[3], b[3], r[3], nb[3];
    for (int s = 0; s < 3; ++s) {
      double f = floor(X[s][p] * inv_dx);
      int64_t ci = (int64_t)f;
      if (ci > N - 1) ci = N - 1;
      if (ci < 0) ci = 0;
      int64_t W = N / P[s];
      c[s] = ci;
      ps[s] = ci / W;
      l[s] = ci - ps[s] * W;
      b[s] = l[s] / brick;
      r[s] = l[s] % brick;
      nb[s] = (W + brick - 1) / brick;
    }
    if (dest) dest[p] = (int32_t)(ps[0] + (int64_t)P[0] * (ps[1] + (int64_t)P[1] * ps[2]));
    if (key)
      key[p] = ((b[2] * nb[1] + b[1]) * nb[0] + b[0]) * brick * brick * brick +
               (r[2] * brick + r[1]) * brick + r[0];
  }
  return ORC_OK;
}

/* Particle migration with the sequential algorithm of the original Fortran
 * LCS (Sec. 2.3.3): the particles of every source subdomain are scanned in
 * order; a particle that stays takes the next slot of its subdomain's stay
 * list, a particle that leaves takes the next slot of the send buffer of its
 * (source, destination) pair -- one counter per direction.  Unpack (Sec.
 * 3.2.2): destination d receives its stayers in order, then the particles
 * sent to it by source 0, 1, ..., P-1, each buffer in its packing order.
 *   seg_in[P+1]   source segments [seg_in[s], seg_in[s+1])
 *   dest[n]       destination subdomain of each particle
 *   perm[n]       out: new position -> old position
 *   seg_out[P+1]  out: destination segments
 *   slot[n]       out (may be NULL): counter value the particle received
 * Returns ORC_ERR_ARG on an out-of-range destination. */
int orc_migrate(int P, int64_t n, const int64_t *seg_in, const int32_t *dest, int64_t *perm,
                int64_t *seg_out, int64_t *slot) {
  int64_t *stay = calloc((size_t)P, sizeof(int64_t));
  int64_t *send = calloc((size_t)P * (size_t)P, sizeof(int64_t));
  int64_t *myslot = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t *base = calloc((size_t)P + 1, sizeof(int64_t));
  if (!stay || !send || !myslot || !base) {
    free(stay), free(send), free(myslot), free(base);
    return ORC_ERR_NOMEM;
  }
  int status = ORC_OK;
  /* sequential scan with per-direction counters */
  for (int src = 0; src < P && status == ORC_OK; ++src)
    for (int64_t i = seg_in[src]; i < seg_in[src + 1]; ++i) {
      int d = dest[i];
      if (d < 0 || d >= P) {
        status = ORC_ERR_ARG;
        break;
      }
      if (d == src)
        myslot[i] = stay[src]++;
      else
        myslot[i] = send[(int64_t)src * P + d]++;
    }
  if (status == ORC_OK) {
    /* destination segment sizes and bases */
    for (int d = 0; d < P; ++d) {
      int64_t in = 0;
      for (int s = 0; s < P; ++s)
        if (s != d) in += send[(int64_t)s * P + d];
      base[d + 1] = base[d] + stay[d] + in;
    }
    for (int d = 0; d <= P; ++d) seg_out[d] = base[d];
    /* unpack: stayers first, then incoming by source ascending */
    for (int src = 0; src < P; ++src)
      for (int64_t i = seg_in[src]; i < seg_in[src + 1]; ++i) {
        int d = dest[i];
        int64_t pos;
        if (d == src) {
          pos = base[d] + myslot[i];
        } else {
          pos = base[d] + stay[d];
          for (int s = 0; s < src; ++s)
            if (s != d) pos += send[(int64_t)s * P + d];
          pos += myslot[i];
        }
        perm[pos] = i;
        if (slot) slot[i] = myslot[i];
      }
  }
  free(stay), free(send), free(myslot), free(base);
  return status;
}

typedef struct {
  int64_t key, idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b) {
  const keyidx *p = a, *q = b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

/* Stable sort of every segment [seg[s], seg[s+1]) by key (ties keep their
 * order: the original index breaks ties).  perm: new position -> old. */
int orc_sort(int P, const int64_t *seg, const int64_t *key, int64_t *perm) {
  for (int s = 0; s < P; ++s) {
    int64_t a = seg[s], m = seg[s + 1] - seg[s];
    if (m <= 0) continue;
    keyidx *t = malloc((size_t)m * sizeof(keyidx));
    if (!t) return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < m; ++i) {
      t[i].key = key[a + i];
      t[i].idx = a + i;
    }
    qsort(t, (size_t)m, sizeof(keyidx), cmp_keyidx);
    for (int64_t i = 0; i < m; ++i) perm[a + i] = t[i].idx;
    free(t);
  }
  return ORC_OK;
}

/* L = (1/n) sum_p mask_p |X_p - X_target,p|^2 on unwrapped positions
 * X + L*img.  mask may be NULL (all ones). */
double orc_loss(double L, int64_t n, const double *x, const double *y, const double *z,
                const int32_t *img, const double *tx, const double *ty, const double *tz,
                const double *mask) {
  const double *X[3] = {x, y, z}, *T[3] = {tx, ty, tz};
  double acc = 0.0;
  for (int64_t p = 0; p < n; ++p) {
    double m = mask ? mask[p] : 1.0;
    double d2 = 0.0;
    for (int s = 0; s < 3; ++s) {
      double xu = X[s][p] + L * (img ? img[(int64_t)s * n + p] : 0);
      double d = xu - T[s][p];
      d2 += d * d;
    }
    acc += m * d2;
  }
  return acc / (double)n;
}

/* Corner weights and their x/y/z derivatives of the trilinear map at one
 * position: for each of the 8 corners its flat field index, its weight
 * w = wx wy wz and dw/dx_s = inv_dx * (+-1) * (product of the other two). */
static void interp_stencil(int N, double inv_dx, const double p[3], int64_t idx[8],
                           double w[8], double dw[8][3]) {
  int64_t lo[3], hi[3];
  double wt[3][2], dt[3][2];
  for (int s = 0; s < 3; ++s) {
    double g = p[s] * inv_dx - 0.5;
    double f = floor(g);
    double t = g - f;
    lo[s] = wrap_index((int64_t)f, N);
    hi[s] = wrap_index((int64_t)f + 1, N);
    wt[s][0] = 1.0 - t;
    wt[s][1] = t;
    dt[s][0] = -inv_dx;
    dt[s][1] = inv_dx;
  }
  int q = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < 2; ++d, ++q) {
        int64_t i = a ? hi[0] : lo[0], j = b ? hi[1] : lo[1], k = d ? hi[2] : lo[2];
        idx[q] = i + (int64_t)N * (j + (int64_t)N * k);
        w[q] = wt[0][a] * wt[1][b] * wt[2][d];
        dw[q][0] = dt[0][a] * wt[1][b] * wt[2][d];
        dw[q][1] = wt[0][a] * dt[1][b] * wt[2][d];
        dw[q][2] = wt[0][a] * wt[1][b] * dt[2][d];
      }
}

/* Apply the transposed interpolation at p to mu (3 comps): accumulate
 * w_corner * mu_c into gfield, and return J(p)^T mu in jt (J = dU/dX). */
static void interp_transpose(const double *field, int N, double inv_dx, const double p[3],
                             const double mu[3], double *gfield, double jt[3]) {
  int64_t idx[8];
  double w[8], dw[8][3];
  interp_stencil(N, inv_dx, p, idx, w, dw);
  const int64_t nn = (int64_t)N * N * N;
  jt[0] = jt[1] = jt[2] = 0.0;
  for (int q = 0; q < 8; ++q)
    for (int c = 0; c < 3; ++c) {
      double f = field[c * nn + idx[q]];
      if (gfield) gfield[c * nn + idx[q]] += w[q] * mu[c];
      for (int s = 0; s < 3; ++s) jt[s] += mu[c] * f * dw[q][s];
    }
}

/* interp_transpose at n points: gfield [3][N^3] accumulates w * mu, and
 * jt (3*n SoA) receives J(X)^T mu for each point (mu is 3*n SoA). */
void orc_interp_transpose_many(const double *field, int N, double inv_dx, int64_t n,
                               const double *x, const double *y, const double *z,
                               const double *mu, double *gfield, double *jt) {
  for (int64_t p = 0; p < n; ++p) {
    double pos[3] = {x[p], y[p], z[p]}, m[3], r[3];
    for (int s = 0; s < 3; ++s) m[s] = mu[(int64_t)s * n + p];
    interp_transpose(field, N, inv_dx, pos, m, gfield, r);
    for (int s = 0; s < 3; ++s) jt[(int64_t)s * n + p] = r[s];
  }
}

/* Reverse-mode derivative of orc_advance (no migration: it only permutes
 * storage).  The forward is re-run from (x, v) storing every step's state;
 * then, from the final adjoints lx, lv (3*n SoA, in/out), each Heun step is
 * reversed.  For one step, with mu1 = lamA1/tau and mu2 = lamA2/tau:
 *   lamA1 = lamA2 = dt/2 lamV'           lamV* = dt/2 lamX' - mu2
 *   lamX* = J(X*)^T mu2                  lamA1 += dt lamV*
 *   lamX  = lamX' + lamX* + J(X)^T mu1
 *   lamV  = lamV' + dt/2 lamX' + lamV* + dt lamX* - mu1
 *   dL/dU += interp^T(X*) mu2 + interp^T(X) mu1
 * The wrap is the identity for the adjoint (the loss uses unwrapped X).
 * On return lx, lv hold dL/dX0, dL/dV0 and gfield ([3][N^3], accumulated,
 * may be NULL) holds dL/dU. */
int orc_adjoint(const double *field, int N, double L, double inv_dx, int64_t n,
                const double *x0, const double *y0, const double *z0, const double *vx0,
                const double *vy0, const double *vz0, const double *tau, double tau_const,
                double dt, const double *g, int nsteps, double *lx, double *lv,
                double *gfield) {
  const size_t per = (size_t)6 * (size_t)n;
  double *traj = malloc(per * (size_t)(nsteps + 1) * sizeof(double));
  if (!traj) return ORC_ERR_NOMEM;
  /* state k stored as [x y z vx vy vz][n] at traj + k*per */
  memcpy(traj + 0 * n, x0, n * sizeof(double));
  memcpy(traj + 1 * n, y0, n * sizeof(double));
  memcpy(traj + 2 * n, z0, n * sizeof(double));
  memcpy(traj + 3 * n, vx0, n * sizeof(double));
  memcpy(traj + 4 * n, vy0, n * sizeof(double));
  memcpy(traj + 5 * n, vz0, n * sizeof(double));
  int status = ORC_OK;
  for (int k = 0; k < nsteps; ++k) {
    double *src = traj + (size_t)k * per, *dst = traj + (size_t)(k + 1) * per;
    memcpy(dst, src, per * sizeof(double));
    int st = orc_advance(field, N, L, inv_dx, n, dst, dst + n, dst + 2 * n, dst + 3 * n,
                         dst + 4 * n, dst + 5 * n, tau, tau_const, dt, g, 1, NULL, NULL, 0,
                         0.0, 0.0, NULL, 0.0, 0.0, 0.0);
    if (st != ORC_OK) status = st;
  }
  for (int k = nsteps - 1; k >= 0; --k) {
    const double *st = traj + (size_t)k * per;
    for (int64_t p = 0; p < n; ++p) {
      const double tp = tau ? tau[p] : tau_const;
      double X[3], V[3], u1[3], a1[3], xs[3], vs[3];
      for (int s = 0; s < 3; ++s) {
        X[s] = st[(size_t)s * n + p];
        V[s] = st[(size_t)(3 + s) * n + p];
      }
      orc_interp(field, N, inv_dx, X[0], X[1], X[2], u1);
      for (int s = 0; s < 3; ++s) {
        a1[s] = (u1[s] - V[s]) / tp + g[s];
        xs[s] = X[s] + dt * V[s];
        vs[s] = V[s] + dt * a1[s];
      }
      double lX1[3], lV1[3], mu1[3], mu2[3], lXs[3], lVs[3], lA1[3], jt2[3], jt1[3];
      for (int s = 0; s < 3; ++s) {
        lX1[s] = lx[(size_t)s * n + p];
        lV1[s] = lv[(size_t)s * n + p];
        double lA2 = 0.5 * dt * lV1[s];
        lA1[s] = 0.5 * dt * lV1[s];
        mu2[s] = lA2 / tp;
        lVs[s] = 0.5 * dt * lX1[s] - mu2[s];
      }
      interp_transpose(field, N, inv_dx, xs, mu2, gfield, jt2);
      for (int s = 0; s < 3; ++s) {
        lXs[s] = jt2[s];
        lA1[s] += dt * lVs[s];
        mu1[s] = lA1[s] / tp;
      }
      interp_transpose(field, N, inv_dx, X, mu1, gfield, jt1);
      for (int s = 0; s < 3; ++s) {
        lx[(size_t)s * n + p] = lX1[s] + lXs[s] + jt1[s];
        lv[(size_t)s * n + p] = lV1[s] + 0.5 * dt * lX1[s] + lVs[s] + dt * lXs[s] - mu1[s];
      }
    }
  }
  free(traj);
  return status;
}

/* Round to nearest, ties to even, to FP32 precision (returned as double). */
void orc_round_f32(int64_t n, const double *in, double *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (double)(float)in[i];
}

/* Round to nearest, ties to even, directly from FP64 to BF16 (8 exponent
 * bits, 8 significant bits; subnormal spacing 2^-133), returned as double.
 * The spacing of BF16 numbers in the binade [2^e, 2^(e+1)) is 2^(e-7). */
void orc_round_bf16(int64_t n, const double *in, double *out) {
  for (int64_t i = 0; i < n; ++i) {
    double x = in[i];
    if (x == 0.0 || !isfinite(x)) {
      out[i] = x;
      continue;
    }
    int E;
    frexp(x, &E); /* |x| = m 2^E, m in [0.5, 1) -> binade exponent E-1 */
    int e = E - 1;
    if (e < -126) e = -126; /* subnormal range: fixed spacing 2^-133 */
    double r = ldexp(nearbyint(ldexp(x, 7 - e)), e - 7);
    if (fabs(r) > 3.3895313892515355e38) r = copysign(INFINITY, x);
    out[i] = r;
  }
}

/* Histogram of the separations of all unordered particle pairs i < j in the
 * periodic cube of side L (minimum image per axis: a difference d > L/2 is
 * replaced by d - L, d < -L/2 by d + L), for separations r < r_max, in nbins
 * equal bins: bin = floor(r * (nbins / r_max)) (clamped to nbins - 1).
 * r^2 = (dx dx + dy dy) + dz dz, r = sqrt(r^2); counts (nbins) are added to. */
void orc_pair_hist(int64_t n, const double *x, const double *y, const double *z, double L,
                   double r_max, int nbins, int64_t *counts) {
  const double inv_w = (double)nbins / r_max;
  const double half = 0.5 * L;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      double d[3] = {x[i] - x[j], y[i] - y[j], z[i] - z[j]};
      for (int s = 0; s < 3; ++s) {
        if (d[s] > half) d[s] -= L;
        else if (d[s] < -half) d[s] += L;
      }
      const double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
      if (r < r_max) {
        int b = (int)(r * inv_w);
        if (b > nbins - 1) b = nbins - 1;
        counts[b] += 1;
      }
    }
}
