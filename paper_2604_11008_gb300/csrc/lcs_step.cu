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
#include <atomic>

#include "lcs_physics.cuh"

namespace lcs {

// ---------------------------------------------------------------- device

int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
    return 1;
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

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
  const int grid = (int)std::min<int64_t>((ncell + 255) / 256, device_sms() * 32);
  k_field_convert<<<grid, 256, 0, st>>>(src, ncell, (int)kind, dst);
  return cudaGetLastError();
}

// Owned-field bricks (the memory pattern of the multi-GPU decomposition):
// brick p holds, x fastest, the converted field cells p_s W_s - 2 ..
// p_s W_s + W_s + 1 along each axis s, wrapped into the periodic grid, so
// that its subdomain's stencils -- with the predictor up to one cell
// outside -- never leave it.  Subdomain p = p_x + P_x (p_y + P_y p_z).
__global__ void k_build_bricks(const unsigned char *field, Geom g, int cb, unsigned char *bricks) {
  const int bx = g.W[0] + 4, by = g.W[1] + 4, bz = g.W[2] + 4;
  const int64_t per = (int64_t)bx * by * bz, total = per * g.Ptot;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / per);
    const int64_t r = i - (int64_t)p * per;
    const int lx = (int)(r % bx), ly = (int)((r / bx) % by), lz = (int)(r / ((int64_t)bx * by));
    const int pc[3] = {p % g.P[0], (p / g.P[0]) % g.P[1], p / (g.P[0] * g.P[1])};
    const int l[3] = {lx, ly, lz};
    int gc[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int c = pc[s] * g.W[s] - 2 + l[s];  // -2 .. N + 1
      c += c < 0 ? g.N : 0;
      c -= c >= g.N ? g.N : 0;
      gc[s] = c;
    }
    const int64_t src = ((int64_t)gc[2] * g.N + gc[1]) * g.N + gc[0];
    if (cb == 8) {
      ((uint2 *)bricks)[i] = ((const uint2 *)field)[src];
    } else {
      for (int k = 0; k < cb / 16; ++k)
        ((uint4 *)bricks)[i * (cb / 16) + k] = ((const uint4 *)field)[src * (cb / 16) + k];
    }
  }
}

cudaError_t launch_build_bricks(const void *field, const Geom &g, FieldKind kind, void *bricks,
                                cudaStream_t st) {
  const int64_t total = (int64_t)(g.W[0] + 4) * (g.W[1] + 4) * (g.W[2] + 4) * g.Ptot;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, device_sms() * 32);
  k_build_bricks<<<std::max(grid, 1), 256, 0, st>>>((const unsigned char *)field, g,
                                                    cell_bytes(kind), (unsigned char *)bricks);
  return cudaGetLastError();
}

cudaError_t launch_field_expand(const void *src, int N, FieldKind kind, double *dst,
                                cudaStream_t st) {
  const int64_t ncell = (int64_t)N * N * N;
  const int grid = (int)std::min<int64_t>((ncell + 255) / 256, device_sms() * 32);
  k_field_expand<<<grid, 256, 0, st>>>(src, ncell, (int)kind, dst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- step dispatch

template <int KIND, int CAP>
cudaError_t launch_step_kind(const StepGroup<CAP> &pb, int mode, int block, int items,
                             bool evolve, int stage, int grid, cudaStream_t st);
template <int KIND>
int step_occupancy_kind(int mode, int block, int items, bool evolve, int stage, bool pf_tau,
                        bool pf_img, bool pf_vs);

template <int CAP>
cudaError_t launch_step_group(const StepGroup<CAP> &pb, FieldKind kind, int mode, int block,
                              int items, bool evolve, int stage, int grid, cudaStream_t st) {
  switch (kind) {
    case FK_F64:
      return launch_step_kind<FK_F64, CAP>(pb, mode, block, items, evolve, stage, grid, st);
    case FK_DF:
      return launch_step_kind<FK_DF, CAP>(pb, mode, block, items, evolve, stage, grid, st);
    case FK_F32:
      return launch_step_kind<FK_F32, CAP>(pb, mode, block, items, evolve, stage, grid, st);
    case FK_BF16:
      return launch_step_kind<FK_BF16, CAP>(pb, mode, block, items, evolve, stage, grid, st);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t launch_step_group<1>(const StepGroup<1> &, FieldKind, int, int, int, bool,
                                          int, int, cudaStream_t);
template cudaError_t launch_step_group<GROUP_ENS>(const StepGroup<GROUP_ENS> &, FieldKind, int,
                                                  int, int, bool, int, int, cudaStream_t);

int step_kernel_occupancy(FieldKind kind, int mode, int block, int items, bool evolve,
                          int stage, bool pf_tau, bool pf_img, bool pf_vs) {
  switch (kind) {
    case FK_F64:
      return step_occupancy_kind<FK_F64>(mode, block, items, evolve, stage, pf_tau, pf_img, pf_vs);
    case FK_DF:
      return step_occupancy_kind<FK_DF>(mode, block, items, evolve, stage, pf_tau, pf_img, pf_vs);
    case FK_F32:
      return step_occupancy_kind<FK_F32>(mode, block, items, evolve, stage, pf_tau, pf_img, pf_vs);
    case FK_BF16:
      return step_occupancy_kind<FK_BF16>(mode, block, items, evolve, stage, pf_tau, pf_img,
                                          pf_vs);
  }
  return 0;
}

// ---------------------------------------------------------------- step tail

// The tail of a step, one kernel: one block of 1024 threads per (ensemble,
// source subdomain) places that source's leavers after the stayers of their
// destinations (unpack, Sec. 3.2.2) and clears its share of the look-back
// words for the next step; the last block of an ensemble to finish computes
// the new counts and the next layout and swaps the buffers.
constexpr int TAIL_BLOCK = 1024;
constexpr int TAIL_WARPS = TAIL_BLOCK / 32;
static_assert(TAIL_WARPS == 32 && TAIL_WARPS >= NBIN, "one warp per direction, one lane per warp");

// Offset, inside destination d, of the leavers of source s in direction b:
// the stayers of d, then the arrivals of d in source order (the destination's
// table fin_tab), up to (s, b).  Warp b computes direction b: lane j reads
// entry j of the table and its count, and the counts before (s, b) are
// summed by a warp reduction -- two dependent loads per warp instead of a
// walk along the table.
__device__ __forceinline__ void tail_offsets(const StepArgs &a, int s, int64_t *s_off) {
  const int lane = threadIdx.x & 31, b = threadIdx.x >> 5;
  if (b >= NBIN || b == BIN_STAY) return;  // whole warps
  const Geom &g = a.geo;
  const int ps[3] = {s % g.P[0], (s / g.P[0]) % g.P[1], s / (g.P[0] * g.P[1])};
  const int dir[3] = {b % 3 - 1, (b / 3) % 3 - 1, b / 9 - 1};
  int pd[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) pd[q] = (ps[q] + dir[q] + g.P[q]) % g.P[q];
  const int d = pd[0] + g.P[0] * (pd[1] + g.P[1] * pd[2]);
  const int me = s * NBIN + b;
  const int e = lane < NBIN - 1 ? __ldg(a.m.fin_tab + d * (NBIN - 1) + lane) : -1;
  // the table ends at its first negative entry; (s, b) itself stops the sum
  const unsigned stop = __ballot_sync(0xffffffffu, lane >= NBIN - 1 || e < 0 || e == me);
  const int j = __ffs(stop) - 1;
  long long c = lane < j ? (long long)a.m.bincnt[e] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) s_off[b] = a.m.stay_tot[d] + c;
}

// Place the packed leavers of source s (one block), in pack order, at their
// offsets, keeping the order within each (source, direction) pair.
__device__ __forceinline__ void tail_unpack(const StepArgs &a, int s, const int64_t *s_off) {
  __shared__ int s_wc[TAIL_WARPS][NBIN];
  __shared__ int s_run[NBIN];
  const Geom &g = a.geo;
  const int ph = *a.m.phase;
  const Rec B = a.buf[ph ^ 1];
  const int64_t bA = a.m.lay_base[ph][s];
  const int64_t *baseB = a.m.lay_base[ph ^ 1];
  const int64_t *capB = a.m.lay_cap[ph ^ 1];
  const int64_t nm = a.m.mig_tot[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ps[3] = {s % g.P[0], (s / g.P[0]) % g.P[1], s / (g.P[0] * g.P[1])};
  if (threadIdx.x < NBIN) s_run[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nm; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const bool valid = i < nm;
    int b = valid ? a.pack_bin[bA + i] : 255;
    if (valid && (b >= NBIN || b == BIN_STAY)) {  // not a leaver's bin: report, skip
      latch(a.m.status, LCS_ERR_STATE);
      b = 255;
    }
    const bool leaver = b != 255;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(peers & ((1u << lane) - 1));
    // row `warp` of s_wc: this warp's count per direction (only this warp
    // touches its row outside the column scan below)
    if (lane < NBIN) s_wc[warp][lane] = 0;
    __syncwarp();
    if (leaver && rank == 0) s_wc[warp][b] = __popc(peers);
    __syncthreads();
    // warp w < NBIN scans column w (direction w) over the warps of the chunk:
    // each entry becomes the rank of that warp's first leaver of direction w
    if (warp < NBIN) {
      const int v = s_wc[lane][warp];
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int run = s_run[warp];
      __syncwarp();
      s_wc[lane][warp] = run + incl - v;
      if (lane == 31) s_run[warp] = run + incl;
    }
    __syncthreads();
    if (leaver) {
      const int dir[3] = {b % 3 - 1, (b / 3) % 3 - 1, b / 9 - 1};
      int pd[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) pd[q] = (ps[q] + dir[q] + g.P[q]) % g.P[q];
      const int d = pd[0] + g.P[0] * (pd[1] + g.P[1] * pd[2]);
      const int64_t rel = s_off[b] + s_wc[warp][b] + rank;
      if (rel < capB[d]) {
        copy_rec(a.pack, bA + i, B, baseB[d] + rel);
      } else {
        latch(a.m.status, LCS_ERR_CAPACITY);
      }
    }
  }
}

// New count of destination d (stayers + arrivals) and the capacity check,
// by one warp: lane j reads entry j of d's arrival table and its count.
// Every block computes its own subdomain's count while the others unpack,
// so the last block only lays out.
__device__ __forceinline__ void tail_count(const StepArgs &a, int d) {
  const int lane = threadIdx.x & 31;
  const int ph = *a.m.phase;
  const int e = lane < NBIN - 1 ? a.m.fin_tab[d * (NBIN - 1) + lane] : -1;
  long long c = e >= 0 ? (long long)a.m.bincnt[e] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) {
    const int64_t tot = a.m.stay_tot[d] + c;
    if (tot > a.m.lay_cap[ph ^ 1][d]) latch(a.m.status, LCS_ERR_CAPACITY);
    a.m.cnt[d] = tot;
  }
}

// The layout of the new counts (the same as layout_from_counts): compacted
// starts, step / sort tile prefixes and the next window layout, with the
// four exclusive scans taken together -- one warp-sum barrier and one
// broadcast barrier per 1024 segments instead of three per scan.
__device__ __forceinline__ void tail_layout(int P, int step_tile, const int64_t *cnt,
                                            int64_t *cstart, int *tile_off, int *stile_off,
                                            int64_t *base, int64_t *cap) {
  __shared__ int64_t s_w[4][TAIL_WARPS];
  __shared__ int64_t s_tot[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t carry[4] = {0, 0, 0, 0};
  for (int d0 = 0; d0 < P; d0 += TAIL_BLOCK) {
    const int d = d0 + threadIdx.x;
    const int64_t c = d < P ? cnt[d] : 0;
    int64_t v[4];
    v[0] = c;                                             // particles
    v[1] = d < P ? c + c / 16 + SLACK_MIN : 0;            // window capacity
    v[2] = d < P ? (c + step_tile - 1) / step_tile : 0;   // step tiles
    v[3] = d < P ? (c + SORT_TILE - 1) / SORT_TILE : 0;   // sort tiles
    int64_t inc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      inc[q] = v[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc[q], o);
        if (lane >= o) inc[q] += y;
      }
      if (lane == 31) s_w[q][warp] = inc[q];
    }
    __syncthreads();
    if (warp < 4) {  // warp q scans the warp sums of value q
      const int64_t wv = s_w[warp][lane];
      int64_t wi = wv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      s_w[warp][lane] = wi - wv;
      if (lane == 31) s_tot[warp] = wi;
    }
    __syncthreads();
    int64_t ex[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ex[q] = carry[q] + inc[q] - v[q] + s_w[q][warp];
    if (d < P) {
      if (cstart) cstart[d] = ex[0];
      if (base) base[d] = ex[1];
      if (cap) cap[d] = v[1];
      if (tile_off) tile_off[d] = (int)ex[2];
      if (stile_off) stile_off[d] = (int)ex[3];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) carry[q] += s_tot[q];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (cstart) cstart[P] = carry[0];
    if (tile_off) tile_off[P] = (int)carry[2];
    if (stile_off) stile_off[P] = (int)carry[3];
  }
}

// Last block of an ensemble (every count is in place): the reset of the
// per-step counters, the next layout, and the swap: the old input buffer
// becomes the next output with the new layout, the output becomes the input.
__device__ __forceinline__ void tail_finish(const StepArgs &a, int count_step) {
  const int P = a.geo.Ptot;
  const int ph = *a.m.phase;
  // every (source, direction) count and stayer total has been read
  for (int i = threadIdx.x; i < P * NBIN; i += blockDim.x) a.m.bincnt[i] = 0;
  for (int d = threadIdx.x; d < P; d += blockDim.x) a.m.stay_tot[d] = 0;
  tail_layout(P, a.step_tile, a.m.cnt, a.m.cstart, a.m.tile_off, a.m.stile_off,
              a.m.next_base, a.m.next_cap);
  __syncthreads();
  for (int d = threadIdx.x; d < P; d += blockDim.x) {
    a.m.lay_base[ph][d] = a.m.next_base[d];
    a.m.lay_cap[ph][d] = a.m.next_cap[d];
  }
  if (threadIdx.x == 0) {
    *a.m.phase = ph ^ 1;
    *a.m.tile_counter = 0u;
    if (count_step) *a.m.nstep += 1;
    *a.m.tail_done = 0u;
  }
}

__global__ void __launch_bounds__(TAIL_BLOCK) k_tail(BatchArgs bt, int count_step) {
  __shared__ int64_t s_off[NBIN];
  __shared__ int s_last;
  const int e = find_segment(bt.ens_P_off, bt.n_ens, (int)blockIdx.x);
  const StepArgs &a = bt.args[e];
  const int s = blockIdx.x - bt.ens_P_off[e];
  const int P = a.geo.Ptot;
  // the step kernels have finished: their tile counters start over
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < bt.ngroups; k += blockDim.x) bt.counter[k] = 0u;
  // look-back words of this step's tiles, cleared in P slices for the next
  const int ntile = a.m.tile_off[P];
  {
    const int per = (ntile + P - 1) / P, t0 = s * per, t1 = min(ntile, t0 + per);
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) a.m.tile_status[t] = 0ull;
  }
  tail_offsets(a, s, s_off);  // warps 0-26
  if ((threadIdx.x >> 5) == TAIL_WARPS - 1) tail_count(a, s);
  __syncthreads();
  tail_unpack(a, s, s_off);
  if (threadIdx.x == 0) a.m.mig_tot[s] = 0;
  // the last block of the ensemble to get here finishes the step
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(a.m.tail_done, 1u) == (unsigned)(P - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  tail_finish(a, count_step);
}

cudaError_t launch_tail(const BatchArgs &bt, int total_P, cudaStream_t st, int count_step) {
  k_tail<<<total_P, TAIL_BLOCK, 0, st>>>(bt, count_step);
  return cudaGetLastError();
}

}  // namespace lcs
