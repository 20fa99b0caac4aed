// Internal declarations shared by the CUDA translation units of liblcs.
//
// Memory layout (one ensemble):
//   * two particle buffers (ping-pong) plus one pack buffer, each of
//     capacity C = np + np/16 + SLACK_MIN * P + 1024 slots, structure of
//     arrays: x[3][C], v[3][C] (FP64), tau[C] (FP64, optional), id[C]
//     (uint32), img[3][C] (int32, optional);
//   * the P subdomain segments of a buffer are fixed-capacity windows
//     [base[s], base[s] + cap[s]) of which the first cnt[s] slots are live;
//     every step writes into the other buffer with a fresh layout whose
//     capacities are the current counts plus slack (cnt/16 + SLACK_MIN), so
//     stayers can be written straight to their final slot by the fused
//     integrate + scan kernel before the number of incoming particles of
//     their subdomain is known;
//   * the field is a library-owned copy, one 32-byte (FP64 variants),
//     16-byte (FP32) or 8-byte (BF16) record per cell holding u, v, w.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "../../include/lcs.h"

namespace lcs {

constexpr int NBIN = 27;          // neighbour directions including (0,0,0)
constexpr int BIN_STAY = 13;      // (0,0,0)
constexpr int SLACK_MIN = 128;
constexpr int MAX_ENS = 4096;    // ensembles per context
constexpr int STAGE_BYTES = 65536;  // shared-memory box of the staged step kernel
constexpr int SORT_BLOCK = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_BLOCK * SORT_ITEMS;  // 4096
constexpr int SORT_MAX_BITS = 9;                    // digit width limit
constexpr int SORT_MAX_D = 1 << SORT_MAX_BITS;
constexpr long long SPIN_LIMIT = 1LL << 26;         // bounded look-back wait

// First error wins; later errors are dropped.
__device__ __forceinline__ void latch(int *status, int code) { atomicCAS(status, 0, code); }

// Particle record buffer (structure of arrays, capacity C).  Positions are
// kept in fixed point in grid-cell units with 52 fraction bits,
// q = RN(x N/L) 2^52 with 0 <= q < N 2^52 (the cell of a particle is q >> 52,
// the floor of the FP64 product x N/L); velocities as unevaluated float
// pairs (hi, lo), 48 significant bits.  The C ABI converts at its edges.
struct Rec {
  int64_t *x[3];    // fixed-point positions
  float2 *v[3];     // velocity float pairs
  double *tau;      // nullptr when tau is a constant
  uint32_t *id;
  int32_t *img[3];  // nullptr entries when images are not tracked
  float2 *vs[3];    // stage velocity V* float pairs (migration per stage), else nullptr
};

// Field storage kinds.
enum FieldKind { FK_F64 = 0, FK_DF = 1, FK_F32 = 2, FK_BF16 = 3 };

// Bytes of one cell (three velocity components plus padding) of the field copy.
__host__ __device__ constexpr int cell_bytes(int kind) {
  return kind == FK_BF16 ? 8 : kind == FK_F32 ? 16 : 32;
}

struct Geom {
  int N;
  int P[3];
  int W[3];        // N / P_s (cells per subdomain along s)
  unsigned Wrcp[3];  // ceil(2^32 / W): c / W = umulhi(c, Wrcp) for 0 <= c < 2^11, W >= 2
  int Ptot;
  double L;
  double inv_dx;   // N / L, one correctly rounded division on the host
  double fix_dx;   // L / N / 2^52: FP64 position of a fixed-point coordinate
  int64_t qL;      // N 2^52: the box side in fixed point
};

// Per-ensemble device metadata arrays.
struct Meta {
  int64_t *lay_base[2];  // segment window starts of buffer 0 / 1   [Ptot]
  int64_t *lay_cap[2];   // segment window capacities                [Ptot]
  int64_t *next_base;    // layout computed for the next output      [Ptot]
  int64_t *next_cap;     //                                           [Ptot]
  int64_t *cnt;          // live particles per segment of the input  [Ptot]
  int64_t *cstart;       // exclusive prefix of cnt (compacted start) [Ptot+1]
  int *tile_off;         // step tiles per segment, prefix            [Ptot+1]
  int *stile_off;        // sort tiles per segment, prefix            [Ptot+1]
  int *phase;            // which buffer is the input (0/1)           [1]
  int *status;           // latched error code                        [1]
  unsigned long long *tile_status;  // look-back words                [max tiles]
  unsigned int *tile_counter;       // dynamic tile ids               [1]
  int *bincnt;           // migrants per (source, direction)          [Ptot*27]
  int64_t *stay_tot;     // stayers per segment                       [Ptot]
  int64_t *mig_tot;      // migrants per segment                      [Ptot]
  unsigned long long *staged;  // step tiles served from a shared-memory field box [1]
  int64_t *nstep;        // steps taken since lcs_init                  [1]
  int *fin_tab;          // arrivals of each destination: source*27 + direction,
                         // by ascending source, -1 padded             [Ptot*26]
  unsigned *tail_done;   // blocks of the step tail done (last-block count) [1]
};

struct StepArgs {
  Geom geo;
  double dt, half_dt, tau_const;
  double g[3];
  Rec buf[2];
  Rec pack;
  uint8_t *pack_bin;
  Meta m;
  const void *field;
  int max_tiles;
  int64_t cap;       // slots per record buffer
  // float-pair splits (hi, lo) of dt, dt/2, dt*N/L and dt*g for the DF step
  float dfk[12];
  int step_tile;     // particles per step tile (block or warp lanes x items per lane)
  int drag;          // 0: Stokes (f = 1); 1: drag factor of Eq. (7)
  double drag_c;     // 18 / (nu rho_p/rho): Re_p^2 = drag_c tau_p |V - U|^2
  // evolving field: second snapshot (nullptr: frozen) and the time fraction
  // of step n's first stage, th = th0 + n dth (second stage th + dth)
  const void *field_b;
  double th0, dth;
  // owned-field mode: the subdomains' own field bricks (W_s + 4 cells per
  // axis: the subdomain's cells and a halo of two), subdomain s at cell
  // s (W_x + 4)(W_y + 4)(W_z + 4); nullptr otherwise.  bricks_b: the same
  // for the second snapshot of an evolving field (else nullptr)
  const void *bricks;
  const void *bricks_b;
  // the cell sort's permutation, not yet applied: compacted rank r of the
  // input (segments in order, cstart) is record perm[r] of the input buffer;
  // set for the first step after a sort, which reads its records through it
  // (nullptr: records in storage order)
  const uint32_t *perm;
};

// The ensembles of one context, as the batched kernels see them.
struct BatchArgs {
  const StepArgs *args;     // device array [n_ens]
  int n_ens;
  const int *ens_P_off;     // device [n_ens+1] prefix of subdomain counts
  unsigned int *counter;    // device tile counters, one per step group
  int ngroups;
};

// A group of at most CAP ensembles advanced by one step-kernel launch; the
// whole struct is the kernel's parameter block (<= 32 KB for CAP = GROUP_ENS).
constexpr int GROUP_ENS = 42;
template <int CAP>
struct StepGroup {
  StepArgs a[CAP];
  int n;
  int pf_tau, pf_img;  // record rows present in some ensemble (prefetch layout)
  int pf_vs;           // stage-velocity rows (migration per stage)
  unsigned int *counter;
};
static_assert(sizeof(StepGroup<GROUP_ENS>) <= 32764, "kernel parameter block too large");

// Segment containing global tile t: largest s with off[s] <= t.
__device__ __forceinline__ int find_segment(const int *off, int P, int t) {
  int lo = 0, hi = P;  // off[lo] <= t < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Segment containing compacted index t: largest s with off[s] <= t.
__device__ __forceinline__ int find_segment64(const int64_t *off, int P, int64_t t) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int wrap_cell(int i, int N) {
  i = i < 0 ? i + N : i;
  i = i >= N ? i - N : i;
  return min(max(i, 0), N - 1);  // memory safety for non-finite input
}

// Normalised direction component from subdomain coordinate a to b.
// Returns -1, 0, +1, or 2 when b is not a neighbour of a.
__host__ __device__ __forceinline__ int dir_comp(int a, int b, int P) {
  if (P == 1) return 0;
  int d = b - a;
  if (d < 0) d += P;
  if (d == 0) return 0;
  if (d == 1) return 1;
  if (P >= 3 && d == P - 1) return -1;
  return 2;
}

// FP64 position returned by the C ABI for a fixed-point coordinate:
// RN(RN(q) L/N 2^-52), kept below L.
__device__ __forceinline__ double export_pos(long long q, const Geom &g) {
  const double x = __dmul_rn(__ll2double_rn(q), g.fix_dx);
  return x >= g.L ? __longlong_as_double(__double_as_longlong(g.L) - 1) : x;
}

__device__ __forceinline__ void copy_rec(const Rec &S, int64_t i, const Rec &D, int64_t o) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    D.x[s][o] = S.x[s][i];
    D.v[s][o] = S.v[s][i];
    if (S.img[s]) D.img[s][o] = S.img[s][i];
  }
  if (S.tau) D.tau[o] = S.tau[i];
  D.id[o] = S.id[i];
  if (S.vs[0]) {
#pragma unroll
    for (int s = 0; s < 3; ++s) D.vs[s][o] = S.vs[s][i];
  }
}

// ---------------------------------------------------------------- block scan helper

// Exclusive scan of v over the block (blockDim.x == 1024); returns the
// exclusive prefix of this thread and writes the block total to *total.
__device__ __forceinline__ int64_t block_excl_scan_1024(int64_t v, int64_t *total) {
  __shared__ int64_t s_w[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int64_t wv = s_w[lane];
    int64_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    s_w[lane] = wi - wv;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const int64_t r = inc - v + s_w[warp];
  __syncthreads();
  return r;
}

// Layout of counts: compacted starts, step/sort tile prefixes, and a fresh
// window layout (capacity = count + count/16 + SLACK_MIN).  One block of 1024.
__device__ __forceinline__ void layout_from_counts(int P, int step_tile, const int64_t *cnt,
                                                   int64_t *cstart, int *tile_off,
                                                   int *stile_off, int64_t *base, int64_t *cap) {
  __shared__ int64_t s_tot;
  int64_t carry_c = 0, carry_b = 0, carry_t = 0, carry_s = 0;
  for (int d0 = 0; d0 < P; d0 += 1024) {
    const int d = d0 + threadIdx.x;
    const int64_t c = d < P ? cnt[d] : 0;
    const int64_t cp = d < P ? c + c / 16 + SLACK_MIN : 0;
    const int64_t nt = d < P ? (c + step_tile - 1) / step_tile : 0;
    const int64_t ns = d < P ? (c + SORT_TILE - 1) / SORT_TILE : 0;
    const int64_t ec = block_excl_scan_1024(c, &s_tot);
    const int64_t tc = s_tot;
    const int64_t eb = block_excl_scan_1024(cp, &s_tot);
    const int64_t tb = s_tot;
    const int64_t et = block_excl_scan_1024(nt, &s_tot);
    const int64_t tt = s_tot;
    const int64_t es = block_excl_scan_1024(ns, &s_tot);
    const int64_t ts = s_tot;
    if (d < P) {
      if (cstart) cstart[d] = carry_c + ec;
      if (tile_off) tile_off[d] = (int)(carry_t + et);
      if (stile_off) stile_off[d] = (int)(carry_s + es);
      if (base) base[d] = carry_b + eb;
      if (cap) cap[d] = cp;
    }
    carry_c += tc, carry_b += tb, carry_t += tt, carry_s += ts;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (cstart) cstart[P] = carry_c;
    if (tile_off) tile_off[P] = (int)carry_t;
    if (stile_off) stile_off[P] = (int)carry_s;
  }
}

// Streaming multiprocessors of the current device (queried once per device
// and cached; grids of the grid-stride kernels are sized from it).
int device_sms();

// Host-side launchers (defined in the .cu files).
cudaError_t launch_field_convert(const double *src, int N, FieldKind kind, void *dst,
                                 cudaStream_t st);
cudaError_t launch_build_bricks(const void *field, const Geom &g, FieldKind kind, void *bricks,
                                cudaStream_t st);
// evolve: the evolving-field instantiation; stage: 0 whole step, 1/2 the
// Runge-Kutta stages for migration per stage (modes 3 and 4; the evolving
// field in mode 3 only)
template <int CAP>
cudaError_t launch_step_group(const StepGroup<CAP> &pb, FieldKind kind, int mode, int block,
                              int items, bool evolve, int stage, int grid, cudaStream_t st);
cudaError_t launch_tail(const BatchArgs &bt, int total_P, cudaStream_t st, int count_step);
cudaError_t launch_field_expand(const void *src, int N, FieldKind kind, double *dst,
                                cudaStream_t st);
// Pair-separation histogram (lcs_stats.cu).
cudaError_t launch_pair_keys(const StepArgs &a, uint32_t *key, uint32_t *pay, int64_t n,
                             int grid, cudaStream_t st);
cudaError_t launch_pair_hist(const StepArgs &a, const uint32_t *key, const uint32_t *pay,
                             int *start, int64_t n, double r_max, int nbins,
                             unsigned long long *counts, int sms, cudaStream_t st);
int step_kernel_occupancy(FieldKind kind, int mode, int block, int items, bool evolve,
                          int stage, bool pf_tau, bool pf_img, bool pf_vs);

// Adjoint: checkpoint of the live particles (compacted, storage order).
struct TapeSlot {
  int64_t *x;   // [3][np] fixed-point positions
  float2 *v;    // [3][np] velocity float pairs
  double *tau;  // [np] or nullptr
  uint32_t *id; // [np]
};
cudaError_t launch_tape_store(const StepArgs &a, const TapeSlot &t, int64_t np, cudaStream_t st);
cudaError_t launch_recompute(const StepArgs &a, FieldKind kind, const TapeSlot &t,
                             unsigned long long *states, int len, int64_t np, cudaStream_t st);
cudaError_t launch_lam_permute(const uint32_t *id, const double *src, double *dst, int64_t np,
                               int to_storage, int *status, cudaStream_t st);
cudaError_t launch_adjoint(const StepArgs &a, FieldKind kind, const unsigned long long *state,
                           const double *tau, double *lam, double *gU, int64_t np,
                           cudaStream_t st);

// Radix engine: stable sort of (key, payload) pairs over segmented tiles.
struct SortArgs {
  int nseg;             // segments (the sort is stable within each)
  const int64_t *cstart;// compacted segment starts [nseg+1]
  const int *tile_off;  // sort tiles per segment prefix [nseg+1]
  uint32_t *key[2];
  uint32_t *pay[2];
  int *hist;            // [tiles * D]
  int *hist_scan;       // [tiles * D]
  int *scan_blocks;     // block partials for the device scan
  int max_tiles;
  int *status;
};
cudaError_t radix_sort(const SortArgs &s, int bits, int *out_buf, cudaStream_t st,
                       int64_t *launches);
int64_t radix_scratch_ints(int max_tiles, int bits);

}  // namespace lcs
