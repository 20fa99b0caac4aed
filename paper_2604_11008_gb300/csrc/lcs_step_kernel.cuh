// The persistent step kernel (interpolate + Heun + wrap + destination flag +
// block scan + decoupled look-back + pack), as templates over the field
// storage, the tile shape and the kernel mode.  Each lcs_step_<kind>.cu
// instantiates the configurations of one field storage, so the (slow)
// device compilation runs in parallel.
//
// Method (Tominaga & Onishi, LCS.jl, arXiv 2604.11008): Sec. 2.2, Eqs. (5)-(7)
// (particle equations, trilinear interpolation, two-stage RK); Sec. 2.1
// (periodic cube); Sec. 2.3.3 (mask, prefix scan, pack); Sec. 3.2.2 (unpack).
#pragma once

#include <algorithm>

#include <cuda/atomic>

#include "lcs_physics.cuh"
#include "lcs_tma.cuh"

namespace lcs {

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

// Tile status words carry flag and value in one 64-bit word, so a reader
// that sees the flag sees its value: relaxed atomics suffice (no fences).
//
// Publish tile t's aggregate (first tile of its segment, at t0: its
// inclusive prefix directly, the exclusive prefix being 0).
__device__ __forceinline__ void publish_aggregate(unsigned long long *status_arr, int t, int t0,
                                                  unsigned long long agg) {
  atom_u64(status_arr[t]).store((t == t0 ? FLAG_PRE : FLAG_AGG) | agg,
                                cuda::memory_order_relaxed);
}

// Exclusive (stay, mig) prefix of tile `t` within its segment (first tile of
// the segment at t0), computed by one whole warp after the tile's aggregate
// has been published: the warp reads 32 predecessors per round, stops at the
// nearest inclusive prefix, and sums the aggregates in between (decoupled
// look-back, Merrill & Garland 2016); then the tile's own inclusive prefix is
// published.  Every lane returns the prefix.  Bounded: on timeout the error
// is latched and the partial sum used; a timeout latched elsewhere ends the
// wait early.
static __device__ unsigned long long resolve_prefix_warp(unsigned long long *status_arr, int t, int t0,
                                                  unsigned long long agg, int *err) {
  const int lane = threadIdx.x & 31;
  if (t == t0) return 0;
  unsigned long long excl = 0;
  int j = t - 1;  // newest predecessor not yet summed
  long long spins = 0;
  unsigned ns = 8;
  while (true) {
    const int idx = j - lane;
    unsigned long long v = FLAG_PRE;  // before the segment start: prefix 0
    if (idx >= t0) v = atom_u64(status_arr[idx]).load(cuda::memory_order_relaxed);
    const unsigned long long f = v & FLAG_MASK;
    const unsigned pre = __ballot_sync(0xffffffffu, f == FLAG_PRE);
    const unsigned inv = __ballot_sync(0xffffffffu, f == 0);
    const int upto = pre ? __ffs(pre) - 1 : 31;          // lanes 0..upto are needed
    const unsigned need = upto == 31 ? 0xffffffffu : ((2u << upto) - 1u);
    if (inv & need) {
      if (++spins > SPIN_LIMIT / 64) {
        if (lane == 0) latch(err, LCS_ERR_TIMEOUT);
        break;
      }
      // an error latched elsewhere (e.g. a block that gave up) ends the wait
      if ((spins & 63) == 0 && *(volatile int *)err == LCS_ERR_TIMEOUT) break;
      __nanosleep(ns);
      ns = ns < 256 ? ns * 2 : 256;
      continue;
    }
    unsigned long long part = lane <= upto ? (v & VAL_MASK) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    excl += part;
    if (pre) break;
    j -= 32;
  }
  if (lane == 0)
    atom_u64(status_arr[t]).store(FLAG_PRE | (excl + agg), cuda::memory_order_relaxed);
  return excl;
}

// Publish, then resolve (the tile waits for its own prefix at once).
__device__ __forceinline__ unsigned long long lookback_warp(unsigned long long *status_arr, int t,
                                                            int t0, unsigned long long agg,
                                                            int *err) {
  if ((threadIdx.x & 31) == 0) publish_aggregate(status_arr, t, t0, agg);
  return resolve_prefix_warp(status_arr, t, t0, agg, err);
}

// ---------------------------------------------------------------- step kernel

__device__ __forceinline__ void load_rec(const Rec &R, int64_t i, long long x[3], df v[3],
                                         double &tau, uint32_t &id, int img[3], double tau_c) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    x[s] = R.x[s][i];
    v[s] = df_from2(R.v[s][i]);
    img[s] = R.img[s] ? R.img[s][i] : 0;
  }
  tau = R.tau ? R.tau[i] : tau_c;
  id = R.id[i];
}

// The part of a record the integration needs: position, velocity, tau_p.
__device__ __forceinline__ void load_motion(const Rec &R, int64_t i, long long x[3], df v[3],
                                            double &tau, double tau_c) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    x[s] = R.x[s][i];
    v[s] = df_from2(R.v[s][i]);
  }
  tau = R.tau ? R.tau[i] : tau_c;
}

__device__ __forceinline__ void store_rec(const Rec &R, int64_t i, const long long x[3],
                                          const df v[3], double tau, uint32_t id,
                                          const int img[3]) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    R.x[s][i] = x[s];
    R.v[s][i] = df_to2(v[s]);
    if (R.img[s]) R.img[s][i] = img[s];
  }
  if (R.tau) R.tau[i] = tau;
  R.id[i] = id;
}

// Destination direction bin (0..26, 13 = stay) of a particle at x from the
// segment of subdomain ps; -1 if the destination is not a neighbour.  Per
// axis the containing cell c (integer part of the fixed-point coordinate) is
// taken relative to the subdomain's first cell, modulo N: d < W stays,
// d < 2W is the next subdomain, d >= N - W the previous one (for P_s = 2 the
// two coincide and the first test wins; for P_s = 1, d < W = N always).
__device__ __forceinline__ int dest_bin(const Geom &g, const int ps[3], const long long x[3]) {
  int bin = 0, mul = 1;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    int c = (int)(x[s] >> 52);
    c = min(max(c, 0), g.N - 1);
    const int W = g.W[s];
    int d = c - ps[s] * W;
    d += d < 0 ? g.N : 0;
    const int dc = d < W ? 0 : d < 2 * W ? 1 : d >= g.N - W ? -1 : 2;
    if (dc == 2) return -1;
    bin += (dc + 1) * mul;
    mul *= 3;
  }
  return bin;
}

struct BlockShared {
  int tile;
  unsigned warp[32];
  unsigned tot;
  unsigned long long excl;
  int hist[NBIN];
  int blo[32][3], bhi[32][3];  // per-warp bounding boxes (staged variant)
};

// Placement of one tile of one ensemble.  Tile j of segment s covers
// particles [j*T, (j+1)*T) of the segment (T = BLOCK*ITEMS), ITEMS
// consecutive ones per thread.
struct TileMeta {
  int gtile;      // tile id across the launch's ensembles
  int e;          // ensemble index within the launch
  int tile;       // tile id within the ensemble
  int seg, t0, ntile, ph;
  int ps[3];      // subdomain coordinates of the segment
  int n;          // particles in the tile (0..T)
  int o8, o4;     // position of the tile's first particle in its prefetched 8- / 4-byte rows
  int64_t cnt;    // live particles of the segment
  int64_t first;  // first particle of the tile within the segment
  int64_t bA;     // window start of the segment in the input buffer
  int64_t cs;     // compacted start of the segment (index of its first rank)
};

template <int T>
__device__ __forceinline__ TileMeta tile_meta(const StepArgs &a, int gtile, int e, int tile) {
  TileMeta m;
  m.gtile = gtile;
  m.e = e;
  m.tile = tile;
  m.ph = *a.m.phase;
  m.seg = find_segment(a.m.tile_off, a.geo.Ptot, tile);
  m.ps[0] = m.seg % a.geo.P[0];
  m.ps[1] = (m.seg / a.geo.P[0]) % a.geo.P[1];
  m.ps[2] = m.seg / (a.geo.P[0] * a.geo.P[1]);
  m.t0 = a.m.tile_off[m.seg];
  m.ntile = a.m.tile_off[m.seg + 1] - m.t0;
  m.cnt = a.m.cnt[m.seg];
  m.bA = a.m.lay_base[m.ph][m.seg];
  m.cs = a.m.cstart[m.seg];
  m.first = (int64_t)(tile - m.t0) * T;
  const int64_t rem = m.cnt - m.first;
  m.n = (int)(rem < 0 ? 0 : (rem > T ? T : rem));
  const int64_t g0 = m.bA + m.first;
  m.o8 = (int)(g0 & 1);
  m.o4 = (int)(g0 & 3);
  return m;
}

// The same placement computed by one whole warp and written to shared
// memory, so the other warps of the block hold none of it in registers.
// The segment of the tile is the number of segments s < P whose first tile
// tile_off[s] is at most `tile`, minus one (tile_off is non-decreasing, so
// those segments form a prefix): every lane counts a slice of tile_off
// with independent loads, one warp sum adds the slices.
// Input slot of particle l of a tile's segment: in storage order, or through
// the pending permutation of a cell sort (its rank cs + l).
__device__ __forceinline__ int64_t rec_slot(const StepArgs &a, const TileMeta &m, int64_t l) {
  return a.perm ? (int64_t)__ldg(a.perm + m.cs + l) : m.bA + l;
}

template <int T>
__device__ __forceinline__ void tile_meta_warp(const StepArgs &a, int gtile, int e, int tile,
                                               TileMeta &out) {
  const int lane = threadIdx.x & 31;
  const int P = a.geo.Ptot;
  const int *off = a.m.tile_off;
  int c = 0;
  for (int s0 = 0; s0 < P; s0 += 128) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int s = s0 + 32 * k + lane;
      c += (s < P && __ldg(off + s) <= tile) ? 1 : 0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) {
    TileMeta m;
    m.gtile = gtile;
    m.e = e;
    m.tile = tile;
    m.ph = *a.m.phase;
    m.seg = max(c - 1, 0);
    const int P0 = a.geo.P[0], P1 = a.geo.P[1];
    m.ps[0] = m.seg % P0;
    m.ps[1] = (m.seg / P0) % P1;
    m.ps[2] = m.seg / (P0 * P1);
    m.t0 = off[m.seg];
    m.ntile = off[m.seg + 1] - m.t0;
    m.cnt = a.m.cnt[m.seg];
    m.bA = a.m.lay_base[m.ph][m.seg];
    m.cs = a.m.cstart[m.seg];
    m.first = (int64_t)(tile - m.t0) * T;
    const int64_t rem = m.cnt - m.first;
    m.n = (int)(rem < 0 ? 0 : (rem > T ? T : rem));
    const int64_t g0 = m.bA + m.first;
    m.o8 = (int)(g0 & 1);
    m.o4 = (int)(g0 & 3);
    out = m;
  }
}

// Prefetched records of one tile in shared memory: rows x0 x1 x2 v0 v1 v2
// [tau] of T+2 doubles, then id [img0 img1 img2] of T+4 words.  Each row is
// copied by one bulk copy starting at the 16-byte boundary at or before the
// tile's first particle (offset o8 / o4 elements), so every copy is aligned
// and a multiple of 16 bytes; the record arrays carry 16 bytes of slack so
// the rounded-up copies stay inside their allocations.
template <int T>
struct PfLayout {
  static constexpr int S8 = (T + 2) * 8, S4 = (T + 4) * 4;
  __host__ __device__ static constexpr int bytes(bool tau, bool img) {
    return (6 + (tau ? 1 : 0)) * S8 + (1 + (img ? 3 : 0)) * S4;
  }
};

template <int T>
__device__ __forceinline__ void pf_issue(const StepArgs &a, const TileMeta &m, bool lay_tau,
                                         unsigned char *buf, uint64_t *bar) {
  using LY = PfLayout<T>;
  const Rec &A = a.buf[m.ph];
  const unsigned n8 = m.n ? (unsigned)((m.o8 + m.n + 1) & ~1) : 0u;
  const unsigned n4 = m.n ? (unsigned)((m.o4 + m.n + 3) & ~3) : 0u;
  const unsigned na8 = 6u + (A.tau ? 1u : 0u), na4 = 1u + (A.img[0] ? 3u : 0u);
  mbar_arrive_expect_tx(bar, na8 * n8 * 8u + na4 * n4 * 4u);
  if (!m.n) return;
  const int64_t g0 = m.bA + m.first, s8 = g0 - m.o8, s4 = g0 - m.o4;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    bulk_load(buf + s * LY::S8, A.x[s] + s8, n8 * 8u, bar);
    bulk_load(buf + (3 + s) * LY::S8, A.v[s] + s8, n8 * 8u, bar);
  }
  if (A.tau) bulk_load(buf + 6 * LY::S8, A.tau + s8, n8 * 8u, bar);
  unsigned char *b4 = buf + (lay_tau ? 7 : 6) * LY::S8;
  bulk_load(b4, A.id + s4, n4 * 4u, bar);
  if (A.img[0]) {
#pragma unroll
    for (int s = 0; s < 3; ++s) bulk_load(b4 + (1 + s) * LY::S4, A.img[s] + s4, n4 * 4u, bar);
  }
}

template <int T>
__device__ __forceinline__ void pf_read(const Rec &A, const TileMeta &m, bool lay_tau,
                                        const unsigned char *buf, int li, long long x[3],
                                        df v[3], double &tau, uint32_t &id, int img[3],
                                        double tau_c) {
  using LY = PfLayout<T>;
  const long long *r8 = (const long long *)buf + m.o8 + li;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    x[s] = r8[s * (T + 2)];
    v[s] = df_from2(((const float2 *)r8)[(3 + s) * (T + 2)]);
  }
  tau = A.tau ? __longlong_as_double(r8[6 * (T + 2)]) : tau_c;
  const uint32_t *r4 = (const uint32_t *)(buf + (lay_tau ? 7 : 6) * LY::S8) + m.o4 + li;
  id = r4[0];
#pragma unroll
  for (int s = 0; s < 3; ++s) img[s] = A.img[0] ? (int)r4[(1 + s) * (T + 4)] : 0;
}

// One tile of one ensemble, processed by one block: integrate + wrap + flag
// its particles, block scan of the (stay, leave) flags, look-back across the
// segment's earlier tiles (by warp 0), then stayers to their compacted slot
// in the output buffer and leavers to the pack buffer.  Records come from
// global memory, or (pf != nullptr) from the tile's prefetched rows.
template <int KIND, int BLOCK, int ITEMS, bool STAGED>
__device__ __forceinline__ void step_block_tile(const StepArgs &a, const TileMeta &mt,
                                                BlockShared &sh, void *stage,
                                                const unsigned char *pf, bool lay_tau) {
  constexpr int T = BLOCK * ITEMS;
  const int ph = mt.ph;
  const Rec A = a.buf[ph], B = a.buf[ph ^ 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = mt.seg, t0 = mt.t0, ntile = mt.ntile, tile = mt.tile;
  const int jt = tile - t0;
  const int64_t cnt = mt.cnt;
  const int64_t l0 = mt.first + (int64_t)threadIdx.x * ITEMS;
  const int64_t bA = mt.bA;
  long long x[ITEMS][3];
  df v[ITEMS][3];
  double tau[ITEMS];
  uint32_t id[ITEMS];
  int img[ITEMS][3], bin[ITEMS];
  unsigned packed = 0;
  int bad = 0;
  const StageTimes tt{0.0, 0.0};  // modes 0-2 serve frozen fields
  auto load_item = [&](int k) {
    if (pf)
      pf_read<T>(A, mt, lay_tau, pf, threadIdx.x * ITEMS + k, x[k], v[k], tau[k], id[k], img[k],
                 a.tau_const);
    else
      load_rec(A, bA + l0 + k, x[k], v[k], tau[k], id[k], img[k], a.tau_const);
  };
  FieldBox box{nullptr, 0, 0, 0, 0, 0, 0};
  if (STAGED && KIND != FK_F64) {
    // Shared-memory box of the tile's field cells: bounding box of the
    // stencil base cells of all its particles, padded by 2 cells below and 3
    // above for the stencil's +1 corner and the predictor's move, copied
    // cooperatively when it fits in STAGE_BYTES.
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if (l0 + k < cnt) {
        load_item(k);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          int c = (int)((x[k][d] - (1ll << 51)) >> 52);  // stencil base cell
          c = min(max(c, -8), a.geo.N + 8);
          lo[d] = min(lo[d], c);
          hi[d] = max(hi[d], c);
        }
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
        hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
      }
      if (lane == 0) sh.blo[warp][d] = lo[d], sh.bhi[warp][d] = hi[d];
    }
    __syncthreads();
    int b_lo[3], b_n[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int l = 1 << 30, h = -(1 << 30);
      for (int w = 0; w < BLOCK / 32; ++w) l = min(l, sh.blo[w][d]), h = max(h, sh.bhi[w][d]);
      b_lo[d] = l - 2;
      b_n[d] = h - l + 5;
    }
    const long long ncell = (long long)b_n[0] * b_n[1] * b_n[2];
    if (b_n[0] > 0 && ncell <= STAGE_BYTES / cell_bytes(KIND)) {
      const int N = a.geo.N;
      // c / n for c < 2^13 as floor((c + 1/2) * (1/n)): the float error is far
      // below the 1/(2n) margin to the next integer, so the quotient is exact
      const float rnx = 1.0f / (float)b_n[0], rny = 1.0f / (float)b_n[1];
      for (int c = threadIdx.x; c < ncell; c += BLOCK) {
        const int r = (int)(((float)c + 0.5f) * rnx), lx = c - r * b_n[0];
        const int lz = (int)(((float)r + 0.5f) * rny), ly = r - lz * b_n[1];
        int gx = b_lo[0] + lx, gy = b_lo[1] + ly, gz = b_lo[2] + lz;
        while (gx < 0) gx += N;
        while (gx >= N) gx -= N;
        while (gy < 0) gy += N;
        while (gy >= N) gy -= N;
        while (gz < 0) gz += N;
        while (gz >= N) gz -= N;
        const size_t g = (size_t)gx + (size_t)N * ((size_t)gy + (size_t)N * gz);
        if (KIND == FK_DF) {
          ldg_cell32((const float4 *)a.field + 2 * g, ((float4 *)stage)[2 * c],
                     ((float4 *)stage)[2 * c + 1]);
        } else if (KIND == FK_F32) {
          ((float4 *)stage)[c] = __ldg((const float4 *)a.field + g);
        } else {
          ((uint2 *)stage)[c] = __ldg((const uint2 *)a.field + g);
        }
      }
      box = FieldBox{stage, b_lo[0], b_lo[1], b_lo[2], b_n[0], b_n[1], b_n[2]};
      if (threadIdx.x == 0) atomicAdd(a.m.staged, 1ull);
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    bin[k] = -2;
    if (l0 + k < cnt) {
      if (!STAGED || KIND == FK_F64) load_item(k);
      if (KIND == FK_F64) heun_step64(a, x[k], v[k], tau[k], img[k], bad, tt);
      else if (KIND == FK_DF) heun_step_df<KIND>(a, x[k], v[k], tau[k], img[k], bad, box, tt);
      else heun_step_lo<KIND>(a, x[k], v[k], tau[k], img[k], bad, box, tt);
      const int ps[3] = {seg % a.geo.P[0], (seg / a.geo.P[0]) % a.geo.P[1],
                         seg / (a.geo.P[0] * a.geo.P[1])};
      int b = dest_bin(a.geo, ps, x[k]);
      if (b < 0) {
        bad |= 2;
        b = BIN_STAY;
      }
      bin[k] = b;
      if (b == BIN_STAY) {
        packed += 1u << 16;
      } else {
        packed += 1u;
        atomicAdd(&sh.hist[b], 1);
      }
    }
  }
  if (bad & 1) latch(a.m.status, LCS_ERR_NONFINITE);
  if (bad & 2) latch(a.m.status, LCS_ERR_DISPLACEMENT);
  unsigned incl = packed;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sh.warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned wv = lane < BLOCK / 32 ? sh.warp[lane] : 0u;
    unsigned wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < BLOCK / 32) sh.warp[lane] = wi - wv;
    if (lane == BLOCK / 32 - 1) sh.tot = wi;
  }
  __syncthreads();
  if (warp == 0) {
    const unsigned tot = sh.tot;
    const unsigned long long agg = pack_sm(tot >> 16, tot & 0xffffu);
    const unsigned long long ex = lookback_warp(a.m.tile_status, tile, t0, agg, a.m.status);
    if (lane == 0) {
      sh.excl = ex;
      if (jt == ntile - 1) {
        const unsigned long long inc = ex + agg;
        a.m.stay_tot[seg] = (int64_t)(inc >> 31);
        a.m.mig_tot[seg] = (int64_t)(inc & ((1ull << 31) - 1));
      }
    }
  }
  __syncthreads();
  const unsigned long long ex = sh.excl;
  if (threadIdx.x < NBIN && threadIdx.x != BIN_STAY && sh.hist[threadIdx.x])
    atomicAdd(&a.m.bincnt[seg * NBIN + threadIdx.x], sh.hist[threadIdx.x]);
  const unsigned excl = incl - packed + sh.warp[warp];
  int64_t stay_pos = (int64_t)(ex >> 31) + (excl >> 16);
  int64_t mig_pos = (int64_t)(ex & ((1ull << 31) - 1)) + (excl & 0xffffu);
  const int64_t bB = a.m.lay_base[ph ^ 1][seg], cB = a.m.lay_cap[ph ^ 1][seg];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
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
}

// Ensemble of global tile g: largest e with off[e] <= g.
__device__ __forceinline__ int find_ensemble(const int *off, int n, int g) {
  int e = 0, hi = n;
  while (hi - e > 1) {
    const int mid = (e + hi) >> 1;
    if (off[mid] <= g) e = mid; else hi = mid;
  }
  return e;
}

// Shared-memory rows of a parked tile (modes 3 and 4): x0 x1 x2 v0 v1 v2
// [tau] of T doubles, id [img0 img1 img2] of T words, then T 16-bit words
// holding the destination bin (bits 0-4) and the images crossed in this step
// per axis (2 bits each, + 1).  Stayers sit at their tile-local rank from
// the front, leavers at their rank from the back.  The id, tau_p and stored
// image counts are not held by the integrating thread: they are copied from
// the input record straight into the rows by asynchronous copies when the
// tile is parked, and the parking thread waits for its copies before the
// block barrier that precedes the write-out, one iteration later.
template <int T>
struct ParkLayout {
  __host__ __device__ static constexpr int bytes(bool tau, bool img) {
    return (6 + (tau ? 1 : 0)) * T * 8 + (1 + (img ? 3 : 0)) * T * 4 + 2 * T;
  }
  __host__ __device__ static constexpr int flags(bool tau, bool img) { return bytes(tau, img) - 2 * T; }
};

// Stage-velocity rows (migration per stage) follow the flag words: 3 rows of
// T float pairs at offset ParkLayout<T>::bytes(tau, img).  Row j receives the
// particle in input slot i of A; dimg are the images crossed in this step.
template <int T>
__device__ __forceinline__ void park_put(unsigned char *pk, bool lay_tau, bool lay_img,
                                         const Rec &A, int64_t i, int j, const long long x[3],
                                         const df v[3], const int dimg[3], int bin,
                                         const df *vs = nullptr) {
  long long *r8 = (long long *)pk;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    r8[s * T + j] = x[s];
    ((float2 *)r8)[(3 + s) * T + j] = df_to2(v[s]);
  }
  if (A.tau) cp_async8(r8 + 6 * T + j, A.tau + i);
  uint32_t *r4 = (uint32_t *)(pk + (lay_tau ? 7 : 6) * T * 8);
  cp_async4(r4 + j, A.id + i);
  unsigned fl = (unsigned)bin;
  if (A.img[0]) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      cp_async4(r4 + (1 + s) * T + j, A.img[s] + i);
      fl |= (unsigned)(dimg[s] + 1) << (5 + 2 * s);
    }
  }
  ((uint16_t *)(pk + ParkLayout<T>::flags(lay_tau, lay_img)))[j] = (uint16_t)fl;
  if (vs) {
    float2 *rv = (float2 *)(pk + ParkLayout<T>::bytes(lay_tau, lay_img));
#pragma unroll
    for (int s = 0; s < 3; ++s) rv[s * T + j] = df_to2(vs[s]);
  }
}

// Copy parked row j to record i of R (and its bin to bins[i] when given).
template <int T>
__device__ __forceinline__ void park_get(const unsigned char *pk, bool lay_tau, bool lay_img,
                                         int j, const Rec &R, int64_t i, uint8_t *bins) {
  const long long *r8 = (const long long *)pk;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    R.x[s][i] = r8[s * T + j];
    R.v[s][i] = ((const float2 *)r8)[(3 + s) * T + j];
  }
  if (R.tau) R.tau[i] = __longlong_as_double(r8[6 * T + j]);
  const uint32_t *r4 = (const uint32_t *)(pk + (lay_tau ? 7 : 6) * T * 8);
  R.id[i] = r4[j];
  const unsigned fl = ((const uint16_t *)(pk + ParkLayout<T>::flags(lay_tau, lay_img)))[j];
  if (R.img[0]) {
#pragma unroll
    for (int s = 0; s < 3; ++s)
      R.img[s][i] = (int32_t)r4[(1 + s) * T + j] + (int)((fl >> (5 + 2 * s)) & 3u) - 1;
  }
  if (bins) bins[i] = (uint8_t)(fl & 31u);
  if (R.vs[0]) {
    const float2 *rv = (const float2 *)(pk + ParkLayout<T>::bytes(lay_tau, lay_img));
#pragma unroll
    for (int s = 0; s < 3; ++s) R.vs[s][i] = rv[s * T + j];
  }
}

// Load and integrate the tile's particles (ITEMS per thread, consecutive):
// Heun step, wrap, destination bin (-2 for no particle), the per-thread
// packed (stay << 16 | leave) count and the block's direction histogram.
// STAGE 0: the whole Heun step; 1: the predictor stage (x becomes X*, vs
// receives V*); 2: the corrector stage (reads vs).
// The owned-field view of a tile's subdomain (owned-field mode): its brick,
// whose cell (0, 0, 0) is global cell p W - 2 per axis.
template <int KIND>
__device__ __forceinline__ FieldBox owned_view(const StepArgs &a, const TileMeta &mt) {
  const int bx = a.geo.W[0] + 4, by = a.geo.W[1] + 4, bz = a.geo.W[2] + 4;
  return FieldBox{(const unsigned char *)a.bricks +
                      (size_t)mt.seg * bx * by * bz * cell_bytes(KIND),
                  mt.ps[0] * a.geo.W[0] - 2, mt.ps[1] * a.geo.W[1] - 2,
                  mt.ps[2] * a.geo.W[2] - 2, bx, by, bz};
}

template <int KIND, int ITEMS, bool EVOLVE, int STAGE, bool OWNED = false>
__device__ __forceinline__ unsigned integrate_items(const StepArgs &a, const TileMeta &mt,
                                                    int *hist, long long x[][3],
                                                    df v[][3], double tau[], uint32_t id[],
                                                    int img[][3], int bin[], df vs[][3]) {
  const Rec &A = a.buf[mt.ph];
  const int64_t l0 = mt.first + (int64_t)threadIdx.x * ITEMS;
  unsigned packed = 0;
  int bad = 0;
  const StageTimes tt = EVOLVE ? stage_times(a) : StageTimes{0.0, 0.0};
  const FieldBox fv = OWNED ? owned_view<KIND>(a, mt) : FieldBox{};
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    bin[k] = -2;
    if (l0 + k < mt.cnt) {
      // id, tau_p and the stored image counts go from the input record to
      // the park rows by asynchronous copies (park_put), so that they hold
      // no registers here; img counts the images crossed in this step
      load_motion(A, rec_slot(a, mt, l0 + k), x[k], v[k], tau[k], a.tau_const);
      img[k][0] = img[k][1] = img[k][2] = 0;
      if (STAGE == 0) {
        if (KIND == FK_F64) heun_step64<EVOLVE>(a, x[k], v[k], tau[k], img[k], bad, tt);
        else if (KIND == FK_DF)
          heun_step_df<KIND, EVOLVE, OWNED>(a, x[k], v[k], tau[k], img[k], bad, fv, tt);
        else heun_step_lo<KIND, EVOLVE, OWNED>(a, x[k], v[k], tau[k], img[k], bad, fv, tt);
      } else if (STAGE == 1) {
        if (KIND == FK_F64) heun_stage1_64<EVOLVE>(a, x[k], v[k], vs[k], tau[k], img[k], bad, tt);
        else if (KIND == FK_DF)
          heun_stage1_df<KIND, OWNED, EVOLVE>(a, x[k], v[k], vs[k], tau[k], img[k], bad, fv, tt);
        else
          heun_stage1_lo<KIND, OWNED, EVOLVE>(a, x[k], v[k], vs[k], tau[k], img[k], bad, fv, tt);
      } else {
        const int64_t i = rec_slot(a, mt, l0 + k);
#pragma unroll
        for (int s = 0; s < 3; ++s) vs[k][s] = df_from2(A.vs[s][i]);
        if (KIND == FK_F64) heun_stage2_64<EVOLVE>(a, x[k], v[k], vs[k], tau[k], img[k], bad, tt);
        else if (KIND == FK_DF)
          heun_stage2_df<KIND, OWNED, EVOLVE>(a, x[k], v[k], vs[k], tau[k], img[k], bad, fv, tt);
        else
          heun_stage2_lo<KIND, OWNED, EVOLVE>(a, x[k], v[k], vs[k], tau[k], img[k], bad, fv, tt);
      }
      int b = dest_bin(a.geo, mt.ps, x[k]);
      if (b < 0) {
        bad |= 2;
        b = BIN_STAY;
      }
      bin[k] = b;
      if (b == BIN_STAY) {
        packed += 1u << 16;
      } else {
        packed += 1u;
        atomicAdd(&hist[b], 1);
      }
    }
  }
  if (bad & 1) latch(a.m.status, LCS_ERR_NONFINITE);
  if (bad & 2) latch(a.m.status, LCS_ERR_DISPLACEMENT);
  return packed;
}

// Mode 3, deferred scatter: a block integrates its next tile while its
// previous tile waits, parked in shared memory, for the look-back; by then
// every predecessor has long published its aggregate, so the look-back does
// not stall the block.  The parked tile is then written out with coalesced
// stores: its stayers form one contiguous run of the output window and its
// leavers one contiguous run of the pack buffer.
constexpr long long PF_WAIT_LIMIT = 1LL << 20;  // bounded wait for a tile's bulk copies

template <int KIND, int BLOCK, int ITEMS, int CAP, bool EVOLVE, int STAGE, bool OWNED>
__device__ __forceinline__ void step_deferred(const StepGroup<CAP> &pb, BlockShared &sh,
                                              const int *s_off, unsigned char *pk) {
  constexpr int T = BLOCK * ITEMS;
  static_assert(BLOCK >= 64, "the acquiring warp must differ from warp 0");
  // Placement of the block's tiles, in three slots: the tile integrated in
  // iteration i sits in slot i % 3, is parked through iteration i + 1, and
  // the last warp takes tile i + 1 into slot (i + 1) % 3 after integrating,
  // while warp 0 resolves the parked tile's prefix (so the tile counter and
  // placement latency overlap the look-back instead of stalling the block).
  // Every iteration passes block barriers, so no warp reads a slot that is
  // being rewritten.
  constexpr int ACQ = BLOCK / 32 - 1;
  __shared__ TileMeta s_meta[3];
  const int n = pb.n, total = s_off[n];
  const bool lay_tau = pb.pf_tau != 0, lay_img = pb.pf_img != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the acquiring warp takes the next tile id and writes its placement
  auto acquire = [&](int slot) {
    int g = 0;
    if (lane == 0) g = (int)atomicAdd(pb.counter, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    TileMeta &m = s_meta[slot];
    if (g < total) {
      const int e = CAP == 1 ? 0 : find_ensemble(s_off, n, g);
      tile_meta_warp<T>(pb.a[e], g, e, g - s_off[e], m);
    } else if (lane == 0) {
      m.gtile = g;
    }
  };
  // the parked tile: resolve its exclusive prefix (warp 0), then write its
  // stayers to the output window and its leavers to the pack buffer
  auto write_out = [&](const TileMeta &pm, unsigned tot) {
    const StepArgs &pa = pb.a[CAP == 1 ? 0 : pm.e];
    if (warp == 0) {
      const unsigned long long agg = pack_sm(tot >> 16, tot & 0xffffu);
      const unsigned long long ex =
          resolve_prefix_warp(pa.m.tile_status, pm.tile, pm.t0, agg, pa.m.status);
      if (lane == 0) {
        sh.excl = ex;
        if (pm.tile - pm.t0 == pm.ntile - 1) {
          const unsigned long long inc = ex + agg;
          pa.m.stay_tot[pm.seg] = (int64_t)(inc >> 31);
          pa.m.mig_tot[pm.seg] = (int64_t)(inc & ((1ull << 31) - 1));
        }
      }
    }
    cp_async_wait_all();  // this thread's copies into the parked rows
    __syncthreads();
    const unsigned long long ex = sh.excl;
    const int nstay = (int)(tot >> 16), nmig = (int)(tot & 0xffffu);
    const int64_t stay0 = (int64_t)(ex >> 31), mig0 = (int64_t)(ex & ((1ull << 31) - 1));
    const int ph = pm.ph;
    const Rec &B = pa.buf[ph ^ 1];
    const int64_t bB = pa.m.lay_base[ph ^ 1][pm.seg], cB = pa.m.lay_cap[ph ^ 1][pm.seg];
    for (int j = threadIdx.x; j < nstay; j += BLOCK) {
      if (stay0 + j < cB) park_get<T>(pk, lay_tau, lay_img, j, B, bB + stay0 + j, nullptr);
      else latch(pa.m.status, LCS_ERR_CAPACITY);
    }
    const int64_t bA = pm.bA;
    for (int j = threadIdx.x; j < nmig; j += BLOCK)
      park_get<T>(pk, lay_tau, lay_img, T - 1 - j, pa.pack, bA + mig0 + j, pa.pack_bin);
    __syncthreads();
  };
  bool parked = false;
  unsigned park_tot = 0;  // (stay, leave) counts of the parked tile
  // per-direction leaver counts of a tile, in two buffers by iteration
  // parity: a buffer is flushed and cleared after the scan barrier of its
  // iteration and next written two iterations later, past further barriers
  __shared__ int s_hist[2][NBIN];
  if (threadIdx.x < 2 * NBIN) (&s_hist[0][0])[threadIdx.x] = 0;
  if (warp == ACQ) acquire(0);
  __syncthreads();
  for (int it = 0;; ++it) {
    TileMeta &cur = s_meta[it % 3];
    const bool fresh = cur.gtile < total;
    long long x[ITEMS][3];
    df v[ITEMS][3];
    double tau[ITEMS];
    uint32_t id[ITEMS];
    int img[ITEMS][3], bin[ITEMS];
    df vs[ITEMS][3];
    unsigned packed = 0;
    if (fresh) {
      const int e = CAP == 1 ? 0 : cur.e;
      packed = integrate_items<KIND, ITEMS, EVOLVE, STAGE, OWNED>(pb.a[e], cur, s_hist[it & 1], x, v, tau,
                                                                  id, img, bin, vs);
      if (warp == ACQ) acquire((it + 1) % 3);
    }
    if (parked) write_out(s_meta[(it + 2) % 3], park_tot);
    if (!fresh) break;
    // block scan of the fresh tile's (stay, leave) counts
    unsigned incl = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) sh.warp[warp] = incl;
    __syncthreads();
    // every warp scans the warp sums itself (no second barrier); the parked
    // tile's total stays in a register of every thread
    unsigned woff;
    {
      constexpr int NW = BLOCK / 32;
      const unsigned wv = lane < NW ? sh.warp[lane] : 0u;
      unsigned wi = wv;
#pragma unroll
      for (int o = 1; o < NW; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      woff = __shfl_sync(0xffffffffu, wi - wv, warp);
      park_tot = __shfl_sync(0xffffffffu, wi, NW - 1);
      if (warp == 0 && lane == NW - 1) {
        const StepArgs &a = pb.a[CAP == 1 ? 0 : cur.e];
        publish_aggregate(a.m.tile_status, cur.tile, cur.t0, pack_sm(wi >> 16, wi & 0xffffu));
      }
    }
    const StepArgs &a = pb.a[CAP == 1 ? 0 : cur.e];
    if (threadIdx.x < NBIN) {
      int *hist = s_hist[it & 1];
      if (threadIdx.x != BIN_STAY && hist[threadIdx.x])
        atomicAdd(&a.m.bincnt[cur.seg * NBIN + threadIdx.x], hist[threadIdx.x]);
      hist[threadIdx.x] = 0;
    }
    const unsigned excl = incl - packed + woff;
    int rs = (int)(excl >> 16), rm = (int)(excl & 0xffffu);
    const Rec &A = a.buf[cur.ph];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if (bin[k] == -2) continue;
      const int j = bin[k] == BIN_STAY ? rs++ : T - 1 - rm++;
      park_put<T>(pk, lay_tau, lay_img, A, rec_slot(a, cur, cur.first + threadIdx.x * ITEMS + k),
                  j, x[k], v[k], img[k], bin[k],
                  STAGE == 1 ? vs[k] : nullptr);
    }
    parked = true;
  }
}

// Persistent step kernel with block tiles: blocks take tile ids from one
// counter in order (predecessors always belong to running blocks).
// Resident threads per SM asked of the compiler (so registers per thread,
// measured): 512 for the all-FP64 kernel (128 registers), 768 with two
// particles per thread (80: no spills; at 64 the FP32 kernel spilled and ran
// 7 % slower), 1024 with one (64).
#ifndef LCS_DF1_THREADS
#define LCS_DF1_THREADS 1024
#endif
template <int KIND, int BLOCK, int ITEMS>
constexpr int step_min_blocks() {
  return KIND == FK_F64 ? 512 / BLOCK
         : ITEMS == 2   ? 768 / BLOCK
         : KIND == FK_DF ? LCS_DF1_THREADS / BLOCK
                         : 1024 / BLOCK;
}


// MODE 0: records read from global memory; 1: the same with the field box
// staged in shared memory; 2: records of the next tile prefetched by bulk
// copies (TMA) into the second of two shared-memory buffers while the
// current tile is integrated, scanned and scattered.
template <int KIND, int BLOCK, int ITEMS, int CAP, int MODE, bool EVOLVE, int STAGE>
__global__ void __launch_bounds__(BLOCK, (step_min_blocks<KIND, BLOCK, ITEMS>()))
    k_step_block(const __grid_constant__ StepGroup<CAP> pb) {
  constexpr int T = BLOCK * ITEMS;
  constexpr bool STAGED = MODE == 1;
  __shared__ BlockShared sh;
  extern __shared__ __align__(128) unsigned char s_dyn[];
  __shared__ int s_off[CAP + 1];
  __shared__ uint64_t s_bar[2];
  __shared__ TileMeta s_meta[2];
  const int n = pb.n;
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int e = 0; e < n; ++e) {
      s_off[e] = acc;
      acc += pb.a[e].m.tile_off[pb.a[e].geo.Ptot];
    }
    s_off[n] = acc;
  }
  if (MODE == 3 || MODE == 4) {
    __syncthreads();
    step_deferred<KIND, BLOCK, ITEMS, CAP, EVOLVE, STAGE, MODE == 4 && KIND != FK_F64>(pb, sh,
                                                                                    s_off, s_dyn);
    return;
  }
  if (MODE != 2) {
    __syncthreads();
    const int total = s_off[n];
    for (;;) {
      if (threadIdx.x == 0) sh.tile = (int)atomicAdd(pb.counter, 1u);
      if (threadIdx.x < NBIN) sh.hist[threadIdx.x] = 0;
      __syncthreads();
      const int g = sh.tile;
      if (g >= total) break;
      const int e = CAP == 1 ? 0 : find_ensemble(s_off, n, g);
      const TileMeta m = tile_meta<T>(pb.a[e], g, e, g - s_off[e]);
      step_block_tile<KIND, BLOCK, ITEMS, STAGED>(pb.a[e], m, sh, s_dyn, nullptr, false);
      __syncthreads();
    }
    return;
  }
  const bool lay_tau = pb.pf_tau != 0;
  const int buf_bytes = PfLayout<T>::bytes(pb.pf_tau != 0, pb.pf_img != 0);
  const int *status0 = pb.a[0].m.status;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int total = s_off[n];
  auto acquire = [&](int slot) {  // thread 0: take the next tile and start its copies
    const int g = (int)atomicAdd(pb.counter, 1u);
    TileMeta m;
    m.gtile = g;
    if (g < total) {
      const int e = CAP == 1 ? 0 : find_ensemble(s_off, n, g);
      m = tile_meta<T>(pb.a[e], g, e, g - s_off[e]);
      fence_proxy_async_smem();
      pf_issue<T>(pb.a[e], m, lay_tau, s_dyn + slot * buf_bytes, &s_bar[slot]);
    }
    s_meta[slot] = m;
  };
  if (threadIdx.x == 0) acquire(0);
  if (threadIdx.x < NBIN) sh.hist[threadIdx.x] = 0;
  __syncthreads();
  for (int i = 0;; ++i) {
    const int cur = i & 1;
    const TileMeta m = s_meta[cur];
    if (m.gtile >= total) break;
    if (threadIdx.x == 0) acquire(cur ^ 1);
    const long long lim = *(volatile const int *)status0 == LCS_ERR_TIMEOUT ? 1 : PF_WAIT_LIMIT;
    if (!mbar_wait(&s_bar[cur], (unsigned)(i >> 1) & 1u, lim))
      latch(pb.a[m.e].m.status, LCS_ERR_TIMEOUT);  // then the tile's rows may be stale
    step_block_tile<KIND, BLOCK, ITEMS, false>(pb.a[m.e], m, sh, nullptr,
                                               s_dyn + cur * buf_bytes, lay_tau);
    if (threadIdx.x < NBIN) sh.hist[threadIdx.x] = 0;
    __syncthreads();
  }
}

// (kernel mode, threads per block, particles per thread) configurations the
// tuner tries; mode 1 (staged field box) has no all-FP64 form
// The last two arguments: evolving-field instantiation, Runge-Kutta stage
// (0: whole step; 1, 2: migration per stage); both exist in modes 3 and 4
// only, and together with 256 threads only.
// Mode 4 is mode 3 reading the owned-field bricks (no all-FP64 form).
#define LCS_STEP_CONFIGS(X, K, C)                                                   \
  X(K, 0, 256, 2, C, 0, 0) X(K, 0, 256, 1, C, 0, 0) X(K, 0, 128, 2, C, 0, 0)       \
  X(K, 1, 256, 2, C, 0, 0) X(K, 1, 128, 2, C, 0, 0) X(K, 2, 256, 2, C, 0, 0)       \
  X(K, 2, 128, 2, C, 0, 0) X(K, 2, 256, 1, C, 0, 0) X(K, 3, 256, 2, C, 0, 0)       \
  X(K, 3, 128, 2, C, 0, 0) X(K, 3, 256, 1, C, 0, 0) X(K, 3, 256, 2, C, 1, 0)       \
  X(K, 3, 128, 2, C, 1, 0) X(K, 3, 256, 1, C, 1, 0) X(K, 3, 256, 2, C, 0, 1)       \
  X(K, 3, 256, 2, C, 0, 2) X(K, 3, 256, 1, C, 0, 1) X(K, 3, 256, 1, C, 0, 2)       \
  X(K, 4, 256, 1, C, 0, 0) X(K, 4, 256, 2, C, 0, 0) X(K, 4, 256, 1, C, 0, 1)       \
  X(K, 4, 256, 1, C, 0, 2) X(K, 4, 256, 2, C, 0, 1) X(K, 4, 256, 2, C, 0, 2)       \
  X(K, 3, 256, 1, C, 1, 1) X(K, 3, 256, 1, C, 1, 2) X(K, 3, 256, 2, C, 1, 1)       \
  X(K, 3, 256, 2, C, 1, 2) X(K, 4, 256, 1, C, 1, 0) X(K, 4, 256, 2, C, 1, 0)       \
  X(K, 4, 256, 1, C, 1, 1) X(K, 4, 256, 1, C, 1, 2) X(K, 4, 256, 2, C, 1, 1)       \
  X(K, 4, 256, 2, C, 1, 2) X(K, 3, 128, 1, C, 0, 0) X(K, 3, 128, 1, C, 1, 0)

// Dynamic shared memory of a configuration: the staged field box (mode 1),
// the two record buffers (mode 2) or the parked tile (modes 3 and 4).
constexpr int step_dyn_smem(int kind, int mode, int tile, bool tau, bool img, bool vs = false) {
  return mode == 4 ? step_dyn_smem(kind, 3, tile, tau, img, vs)
         : mode == 3 ? (6 + (tau ? 1 : 0)) * tile * 8 + (1 + (img ? 3 : 0)) * tile * 4 +
                           2 * tile + (vs ? 3 * tile * 8 : 0)
         : mode == 1 ? (kind != FK_F64 ? STAGE_BYTES : 0)
         : mode == 2 ? 2 * ((6 + (tau ? 1 : 0)) * (tile + 2) * 8 +
                            (1 + (img ? 3 : 0)) * (tile + 4) * 4)
                     : 0;
}


// Shared-memory carveout (percent of the SM's 228 KB) that just holds the
// resident blocks the kernel is built for, so the rest of the unified
// L1 / shared array serves as L1 for the field gathers (measured: step
// kernel 1.3 % faster than the driver's choice; a carveout too small for
// the resident blocks cuts occupancy and made it 2.5x slower).
template <class K>
int step_carveout(K ker, int dyn_smem, int block) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, ker) != cudaSuccess) return -1;
  // blocks the register file holds (registers are allocated per warp in
  // units of 256), at most 2048 threads per SM
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int blocks = std::max(1, std::min(65536 / std::max(1, regs_warp * (block / 32)),
                                          2048 / block));
  const int per_block = dyn_smem + (int)fa.sharedSizeBytes + 1024;  // + the 1 KB reserved per block
  const int total = 228 * 1024;
  return std::min(100, (blocks * per_block * 100 + total - 1) / total);
}

// One field storage's configurations: launch / occupancy (lcs_step_<kind>.cu).
template <int KIND, int CAP>
cudaError_t launch_step_kind(const StepGroup<CAP> &pb, int mode, int block, int items,
                             bool evolve, int stage, int grid, cudaStream_t st) {
#define LCS_LAUNCH(K, M, B, I, C, E, S)                                                    \
  if (mode == M && block == B && items == I && evolve == (E != 0) && stage == S &&        \
      !((M == 1 || M == 4) && K == FK_F64)) {                                              \
    static_assert(PfLayout<B * I>::bytes(true, true) ==                                    \
                      step_dyn_smem(K, 2, B * I, true, true) / 2, "layout");               \
    static_assert(ParkLayout<B * I>::bytes(true, false) ==                                 \
                      step_dyn_smem(K, 3, B * I, true, false), "layout");                  \
    auto ker = k_step_block<K, B, I, CAP, M, (E != 0), S>;                                 \
    const int smem = step_dyn_smem(K, M, B * I, pb.pf_tau != 0, pb.pf_img != 0,            \
                                   pb.pf_vs != 0);                                         \
    if (smem) cudaFuncSetAttribute(ker, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    cudaFuncSetAttribute(ker, cudaFuncAttributePreferredSharedMemoryCarveout,              \
                         step_carveout(ker, smem, B));                                      \
    ker<<<grid, B, smem, st>>>(pb);                                                        \
    return cudaGetLastError();                                                             \
  }
  LCS_STEP_CONFIGS(LCS_LAUNCH, KIND, CAP)
#undef LCS_LAUNCH
  return cudaErrorInvalidValue;
}

template <int KIND>
int step_occupancy_kind(int mode, int block, int items, bool evolve, int stage, bool pf_tau,
                        bool pf_img, bool pf_vs) {
  int n = 0;
#define LCS_OCC(K, M, B, I, C, E, S)                                                       \
  if (mode == M && block == B && items == I && evolve == (E != 0) && stage == S &&        \
      !((M == 1 || M == 4) && K == FK_F64)) {                                              \
    auto ker = k_step_block<K, B, I, C, M, (E != 0), S>;                                   \
    const int smem = step_dyn_smem(K, M, B * I, pf_tau, pf_img, pf_vs);                    \
    if (smem) cudaFuncSetAttribute(ker, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    cudaFuncSetAttribute(ker, cudaFuncAttributePreferredSharedMemoryCarveout,              \
                         step_carveout(ker, smem, B));                                      \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ker, B, smem);                       \
  }
  LCS_STEP_CONFIGS(LCS_OCC, KIND, GROUP_ENS)
#undef LCS_OCC
  return n;
}

#define LCS_STEP_KIND_INSTANTIATE(K)                                                       \
  template cudaError_t launch_step_kind<K, 1>(const StepGroup<1> &, int, int, int, bool, int, \
                                              int, cudaStream_t);                         \
  template cudaError_t launch_step_kind<K, GROUP_ENS>(const StepGroup<GROUP_ENS> &, int, int, \
                                                      int, bool, int, int, cudaStream_t); \
  template int step_occupancy_kind<K>(int, int, int, bool, int, bool, bool, bool);

}  // namespace lcs
