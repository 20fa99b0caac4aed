// Scan-driven stable counting sort (LSD radix over digits of at most
// SORT_MAX_BITS bits) of (key, payload) pairs, stable within segments, and
// the particle passes built on it: cell sort, general migration, initial
// placement, and the stateless partition.
//
// Each digit pass is a counting sort: per-tile digit histograms, one
// exclusive prefix scan over the (segment, digit, tile) histogram table --
// which gives every (segment, digit, tile) its output offset, the same
// prefix-scan-gives-the-slot idea as the particle pack of Sec. 2.3.3 -- and
// a stable scatter that ranks equal digits inside a tile with warp match
// masks, in input order.
#include "lcs_df.cuh"
#include "lcs_internal.cuh"

namespace lcs {

// ---------------------------------------------------------------- histograms

template <int MAXD>
__global__ void __launch_bounds__(SORT_BLOCK) k_upsweep(SortArgs s, const uint32_t *key, int shift,
                                                        int D) {
  __shared__ int h[MAXD];
  const int total = s.tile_off[s.nseg];
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    for (int d = threadIdx.x; d < D; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int seg = find_segment(s.tile_off, s.nseg, tile);
    const int t0 = s.tile_off[seg], nt = s.tile_off[seg + 1] - t0, jt = tile - t0;
    const int64_t a = s.cstart[seg] + (int64_t)jt * SORT_TILE;
    const int64_t e = min(s.cstart[seg + 1], a + SORT_TILE);
    // all of a thread's keys in flight at once, then the counts
    uint32_t kk[SORT_ITEMS];
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      const int64_t i = a + r * SORT_BLOCK + threadIdx.x;
      kk[r] = i < e ? key[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r)
      if (a + r * SORT_BLOCK + threadIdx.x < e) atomicAdd(&h[(kk[r] >> shift) & (D - 1)], 1);
    __syncthreads();
    int *out = s.hist + (int64_t)t0 * D;
    for (int d = threadIdx.x; d < D; d += blockDim.x) out[(int64_t)d * nt + jt] = h[d];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- device scan

constexpr int SCAN_BLOCK = 256, SCAN_ITEMS = 16, SCAN_CHUNK = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ int block_excl_scan_int(int v, int *total) {
  __shared__ int s_w[SCAN_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int wv = lane < SCAN_BLOCK / 32 ? s_w[lane] : 0;
    int wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < SCAN_BLOCK / 32) s_w[lane] = wi - wv;
    if (lane == SCAN_BLOCK / 32 - 1) *total = wi;
  }
  __syncthreads();
  const int r = inc - v + s_w[warp];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_reduce(SortArgs s, int D) {
  __shared__ int s_tot;
  const int64_t n = (int64_t)s.tile_off[s.nseg] * D;
  const int64_t a = (int64_t)blockIdx.x * SCAN_CHUNK;
  if (a >= n) return;
  int sum = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = a + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    if (i < n) sum += s.hist[i];
  }
  block_excl_scan_int(sum, &s_tot);
  if (threadIdx.x == 0) s.scan_blocks[blockIdx.x] = s_tot;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_partials(SortArgs s, int D) {
  __shared__ int s_tot;
  const int64_t n = (int64_t)s.tile_off[s.nseg] * D;
  const int nb = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += SCAN_BLOCK) {
    const int b = b0 + threadIdx.x;
    const int v = b < nb ? s.scan_blocks[b] : 0;
    const int e = block_excl_scan_int(v, &s_tot);
    if (b < nb) s.scan_blocks[b] = carry + e;
    carry += s_tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_down(SortArgs s, int D) {
  __shared__ int s_tot;
  const int64_t n = (int64_t)s.tile_off[s.nseg] * D;
  const int64_t a = (int64_t)blockIdx.x * SCAN_CHUNK;
  if (a >= n) return;
  int v[SCAN_ITEMS], sum = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = a + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    v[k] = i < n ? s.hist[i] : 0;
    sum += v[k];
  }
  int run = block_excl_scan_int(sum, &s_tot) + s.scan_blocks[blockIdx.x];
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = a + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    if (i < n) s.hist_scan[i] = run;
    run += v[k];
  }
}

// ---------------------------------------------------------------- stable scatter

// Stable scatter of one digit pass.  Each tile ranks its keys by digit with
// warp match masks in input order (rank among the equal digits of the warp's
// earlier rounds), turns the per-(warp, digit) counts into tile-local digit
// offsets, places every key at its tile-local sorted position in shared
// memory, and then writes the tile out in that order: consecutive threads
// write consecutive slots of one digit's output run, so the stores are
// coalesced instead of landing in one digit bucket per lane.  Output slot =
// the tile's global offset for the digit (hist_scan) + the key's rank among
// the tile's keys of that digit, the same slot as a direct scatter.
template <int MAXD>
__global__ void __launch_bounds__(SORT_BLOCK, 3) k_downsweep(SortArgs s, const uint32_t *kin,
                                                          const uint32_t *pin, uint32_t *kout,
                                                          uint32_t *pout, int shift, int D) {
  constexpr int NW = SORT_BLOCK / 32;
  // per-(warp, digit) counts, then the staged tile (keys, payloads)
  __shared__ uint32_t pool[2 * SORT_TILE > NW * MAXD ? 2 * SORT_TILE : NW * MAXD];
  __shared__ int64_t base[MAXD];  // output slot of the tile's first key of each digit
  __shared__ int toff[MAXD];      // tile-local offset of each digit
  __shared__ int s_part[SORT_BLOCK / 32];
  int(*wc)[MAXD] = reinterpret_cast<int(*)[MAXD]>(pool);
  uint32_t *sk = pool, *sp = pool + SORT_TILE;
  const int total = s.tile_off[s.nseg];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1;
  constexpr int PER_WARP = SORT_TILE / NW;  // 512
  const int64_t n_all = s.cstart[s.nseg];
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int seg = find_segment(s.tile_off, s.nseg, tile);
    const int t0 = s.tile_off[seg], nt = s.tile_off[seg + 1] - t0, jt = tile - t0;
    const int64_t a = s.cstart[seg] + (int64_t)jt * SORT_TILE;
    const int64_t e = min(s.cstart[seg + 1], a + SORT_TILE);
    const int ntile = (int)(e - a);
    for (int i = threadIdx.x; i < NW * MAXD; i += blockDim.x) (&wc[0][0])[i] = 0;
    for (int d = threadIdx.x; d < D; d += blockDim.x)
      base[d] = s.hist_scan[(int64_t)t0 * D + (int64_t)d * nt + jt];
    __syncthreads();
    uint32_t k[SORT_ITEMS], p[SORT_ITEMS];
    int rk[SORT_ITEMS];
    // every key and payload of the thread in flight at once (the ranking
    // below passes warp barriers, which loads inside it would wait behind)
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      const int64_t i = a + warp * PER_WARP + r * 32 + lane;
      const bool valid = i < e;
      k[r] = valid ? kin[i] : 0u;
      p[r] = valid ? pin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      const int64_t i = a + warp * PER_WARP + r * 32 + lane;
      const bool valid = i < e;
      const int dg = valid ? (int)((k[r] >> shift) & (D - 1)) : MAXD;
      const unsigned peers = __match_any_sync(0xffffffffu, dg);
      const int rank = __popc(peers & lt);
      const int b = valid ? wc[warp][dg] : 0;
      __syncwarp();
      if (valid && rank == 0) wc[warp][dg] = b + __popc(peers);
      __syncwarp();
      rk[r] = valid ? b + rank : -1;
    }
    __syncthreads();
    // per digit: exclusive offsets over the warps, and the digit's tile count
    int cnt[(MAXD + SORT_BLOCK - 1) / SORT_BLOCK];
#pragma unroll
    for (int q = 0; q < (MAXD + SORT_BLOCK - 1) / SORT_BLOCK; ++q) {
      const int d = threadIdx.x + q * SORT_BLOCK;
      int run = 0;
      if (d < D) {
        for (int w = 0; w < NW; ++w) {
          const int t = wc[w][d];
          wc[w][d] = run;
          run += t;
        }
      }
      cnt[q] = run;
    }
    // tile-local digit offsets: exclusive scan of the counts over the digits
    // (digit d = threadIdx.x + q * SORT_BLOCK, scanned q-major)
    int carry = 0;
#pragma unroll
    for (int q = 0; q < (MAXD + SORT_BLOCK - 1) / SORT_BLOCK; ++q) {
      int inc = cnt[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) s_part[warp] = inc;
      __syncthreads();
      int wbase = 0, tot = 0;
      for (int w = 0; w < NW; ++w) {
        const int t = s_part[w];
        wbase += w < warp ? t : 0;
        tot += t;
      }
      const int d = threadIdx.x + q * SORT_BLOCK;
      if (d < MAXD) toff[d] = carry + wbase + inc - cnt[q];
      carry += tot;
      __syncthreads();
    }
    // tile-local sorted position of every key (in place of its rank), then stage
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      const int dg = (int)((k[r] >> shift) & (D - 1));
      if (rk[r] >= 0) rk[r] += toff[dg] + wc[warp][dg];
    }
    __syncthreads();  // every read of the counts is done before they are overwritten
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      if (rk[r] < 0) continue;
      sk[rk[r]] = k[r];
      sp[rk[r]] = p[r];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ntile; j += blockDim.x) {
      const uint32_t key = sk[j];
      const int dg = (int)((key >> shift) & (D - 1));
      const int64_t pos = base[dg] + (j - toff[dg]);
      if (pos < 0 || pos >= n_all) {  // inconsistent histogram: report, never write
        if (s.status) latch(s.status, LCS_ERR_STATE);
        continue;
      }
      kout[pos] = key;
      pout[pos] = sp[j];
    }
    __syncthreads();
  }
}

int64_t radix_scratch_ints(int max_tiles, int bits) {
  (void)bits;
  return (int64_t)max_tiles * SORT_MAX_D;
}

cudaError_t radix_sort(const SortArgs &s, int bits, int *out_buf, cudaStream_t st,
                       int64_t *launches) {
  int ib = 0;
  if (bits > 0) {
    const int passes = (bits + SORT_MAX_BITS - 1) / SORT_MAX_BITS;
    const int b = (bits + passes - 1) / passes;
    const int grid = max(1, min(s.max_tiles, device_sms() * 8));
    const int64_t maxn = (int64_t)s.max_tiles * SORT_MAX_D;
    const int sgrid = (int)((maxn + SCAN_CHUNK - 1) / SCAN_CHUNK);
    for (int p = 0, shift = 0; p < passes; ++p, shift += b) {
      const int bp = min(b, bits - shift);
      const int D = 1 << bp;
      if (D <= 64) k_upsweep<64><<<grid, SORT_BLOCK, 0, st>>>(s, s.key[ib], shift, D);
      else k_upsweep<SORT_MAX_D><<<grid, SORT_BLOCK, 0, st>>>(s, s.key[ib], shift, D);
      k_scan_reduce<<<sgrid, SCAN_BLOCK, 0, st>>>(s, D);
      k_scan_partials<<<1, SCAN_BLOCK, 0, st>>>(s, D);
      k_scan_down<<<sgrid, SCAN_BLOCK, 0, st>>>(s, D);
      if (D <= 64) k_downsweep<64><<<grid, SORT_BLOCK, 0, st>>>(s, s.key[ib], s.pay[ib], s.key[ib ^ 1],
                                                       s.pay[ib ^ 1], shift, D);
      else k_downsweep<SORT_MAX_D><<<grid, SORT_BLOCK, 0, st>>>(s, s.key[ib], s.pay[ib],
                                                               s.key[ib ^ 1], s.pay[ib ^ 1],
                                                               shift, D);
      if (launches) *launches += 5;
      ib ^= 1;
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return err;
    }
  }
  *out_buf = ib;
  return cudaSuccess;
}

}  // namespace lcs

// ---------------------------------------------------------------- particle passes

namespace lcs {


// Containing cell of a fixed-point coordinate (its integer part).
__device__ __forceinline__ int cell_of(const Geom &g, long long q) {
  const int c = (int)(q >> 52);
  return min(max(c, 0), g.N - 1);
}

// Brick-major cell key within the particle's subdomain (B^3 bricks,
// x fastest at both levels) -- the order of the cell sort.
__global__ void k_keys_cell(StepArgs a, uint32_t *key, uint32_t *pay, int B, int nbx, int nby) {
  const int ph = *a.m.phase;
  const Rec A = a.buf[ph];
  const int64_t *base = a.m.lay_base[ph];
  const int P = a.geo.Ptot;
  const int64_t n = a.m.cstart[P];
  // brick edge a power of two (the default 8): shifts and masks instead of
  // divisions (the same key)
  const int lb = (B & (B - 1)) == 0 ? __ffs(B) - 1 : -1;
  const uint32_t B3 = (uint32_t)(B * B * B);
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int seg = i < n ? find_segment64(a.m.cstart, P, i) : 0;  // then tracked: i only grows
  int seg_c = -1;  // segment whose origin is in o[]
  int64_t seg_s = 0, seg_b = 0, seg_e = 0;
  int o[3] = {0, 0, 0};
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (seg_c >= 0 && i >= seg_e)  // past the segment in registers: find the next
      while (seg + 1 < P && a.m.cstart[seg + 1] <= i) ++seg;
    if (seg != seg_c) {
      seg_c = seg;
      seg_s = a.m.cstart[seg];
      seg_e = a.m.cstart[seg + 1];
      seg_b = base[seg];
      const int ps[3] = {seg % a.geo.P[0], (seg / a.geo.P[0]) % a.geo.P[1],
                         seg / (a.geo.P[0] * a.geo.P[1])};
#pragma unroll
      for (int s = 0; s < 3; ++s) o[s] = ps[s] * a.geo.W[s];
    }
    const int64_t slot = seg_b + (i - seg_s);
    int l[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int c = cell_of(a.geo, A.x[s][slot]);
      l[s] = min(max(c - o[s], 0), a.geo.W[s] - 1);
    }
    uint32_t brick, in;
    if (lb >= 0) {
      const int m = B - 1;
      brick = (uint32_t)((((l[2] >> lb) * nby + (l[1] >> lb)) * nbx) + (l[0] >> lb));
      in = (uint32_t)((((l[2] & m) << lb) + (l[1] & m)) << lb) + (uint32_t)(l[0] & m);
    } else {
      brick = (uint32_t)((l[2] / B * nby + l[1] / B) * nbx + l[0] / B);
      in = (uint32_t)(((l[2] % B) * B + l[1] % B) * B + l[0] % B);
    }
    key[i] = brick * B3 + in;
    pay[i] = (uint32_t)slot;
  }
}

// Destination key 2*dest + (dest != source segment): a stable sort by it is
// the migration order (stayers first, then arrivals by source, Sec. 3.2.2).
__global__ void k_keys_dest(StepArgs a, uint32_t *key, uint32_t *pay) {
  const int ph = *a.m.phase;
  const Rec A = a.buf[ph];
  const int64_t *base = a.m.lay_base[ph];
  const int P = a.geo.Ptot;
  const int64_t n = a.m.cstart[P];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int seg = find_segment64(a.m.cstart, P, i);
    const int64_t slot = base[seg] + (i - a.m.cstart[seg]);
    int p[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const long long q = A.x[s][slot];
      if (!(q >= 0 && q < a.geo.qL)) latch(a.m.status, LCS_ERR_ARG);
      p[s] = cell_of(a.geo, q) / a.geo.W[s];
    }
    const uint32_t d = (uint32_t)(p[0] + a.geo.P[0] * (p[1] + a.geo.P[1] * p[2]));
    key[i] = 2u * d + (d != (uint32_t)seg ? 1u : 0u);
    pay[i] = (uint32_t)slot;
  }
}

// Single-segment tables {0, n} and {0, tiles(n)} for whole-array sorts.
__global__ void k_one_segment(const int64_t *cstart, int P, int64_t *cs1, int *to1) {
  const int64_t n = cstart[P];
  cs1[0] = 0, cs1[1] = n;
  to1[0] = 0, to1[1] = (int)((n + SORT_TILE - 1) / SORT_TILE);
}

// Bin starts of sorted keys: start[b] = first rank whose (key >> shift) >= b.
__global__ void k_bin_bounds(const uint32_t *key, const int64_t *cs1, int shift, int nbins,
                             int64_t *start) {
  const int64_t n = cs1[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int cur = i < n ? (int)umin(key[i] >> shift, (unsigned)nbins - 1u) : nbins;
    const int prev = i > 0 ? (int)umin(key[i - 1] >> shift, (unsigned)nbins - 1u) : -1;
    for (int b = prev + 1; b <= cur; ++b) start[b] = i;
  }
}

// New counts from compacted starts, then a fresh layout for the output buffer.
__global__ void __launch_bounds__(1024) k_relayout(StepArgs a, int from_starts) {
  const int P = a.geo.Ptot;
  const int ph = *a.m.phase;
  if (from_starts)
    for (int d = threadIdx.x; d < P; d += blockDim.x) a.m.cnt[d] = a.m.cstart[d + 1] - a.m.cstart[d];
  __syncthreads();
  layout_from_counts(P, a.step_tile, a.m.cnt, a.m.cstart, a.m.tile_off, a.m.stile_off,
                     a.m.lay_base[ph ^ 1], a.m.lay_cap[ph ^ 1]);
}

// Output rank r (compacted, segment found from cstart) <- input slot pay[r].
// A thread copies GATHER_ITEMS records per round (ranks r0 + k * stride),
// issuing all their loads before any store so that many of the scattered
// reads are in flight at once; the segment of a rank is tracked
// incrementally (a thread's ranks only grow) instead of a binary search
// per record.
constexpr int GATHER_ITEMS = 4;
__global__ void __launch_bounds__(256) k_gather(StepArgs a, const uint32_t *pay) {
  const int ph = *a.m.phase;
  const Rec A = a.buf[ph], B = a.buf[ph ^ 1];
  const int64_t *baseB = a.m.lay_base[ph ^ 1];
  const int64_t *cs = a.m.cstart;
  const int P = a.geo.Ptot;
  const int64_t n = cs[P];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int d = r0 < n ? find_segment64(cs, P, r0) : 0;
  for (; r0 < n; r0 += stride * GATHER_ITEMS) {
    int64_t src[GATHER_ITEMS], dst[GATHER_ITEMS];
#pragma unroll
    for (int k = 0; k < GATHER_ITEMS; ++k) {
      const int64_t r = r0 + k * stride;
      src[k] = -1;
      dst[k] = 0;
      if (r < n) {
        while (d + 1 < P && cs[d + 1] <= r) ++d;
        const uint32_t s = pay[r];
        if (s >= a.cap) {  // corrupt permutation: report, never read out of bounds
          latch(a.m.status, LCS_ERR_STATE);
        } else {
          src[k] = s;
          dst[k] = baseB[d] + (r - cs[d]);
        }
      }
    }
    long long x[GATHER_ITEMS][3];
    float2 v[GATHER_ITEMS][3];
    double tau[GATHER_ITEMS];
    uint32_t id[GATHER_ITEMS];
#pragma unroll
    for (int k = 0; k < GATHER_ITEMS; ++k) {
      if (src[k] < 0) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x[k][c] = A.x[c][src[k]];
        v[k][c] = A.v[c][src[k]];
      }
      tau[k] = A.tau ? A.tau[src[k]] : 0.0;
      id[k] = A.id[src[k]];
    }
#pragma unroll
    for (int k = 0; k < GATHER_ITEMS; ++k) {
      if (src[k] < 0) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        B.x[c][dst[k]] = x[k][c];
        B.v[c][dst[k]] = v[k][c];
      }
      if (A.tau) B.tau[dst[k]] = tau[k];
      B.id[dst[k]] = id[k];
      // optional rows (image counts, stage velocities), record by record
      if (A.img[0]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) B.img[c][dst[k]] = A.img[c][src[k]];
      }
      if (A.vs[0]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) B.vs[c][dst[k]] = A.vs[c][src[k]];
      }
    }
  }
}

// Both buffers take the output layout; the output becomes the input.
__global__ void k_set_phase(StepArgs a) {
  const int ph = *a.m.phase;
  for (int d = threadIdx.x; d < a.geo.Ptot; d += blockDim.x) {
    a.m.lay_base[ph][d] = a.m.lay_base[ph ^ 1][d];
    a.m.lay_cap[ph][d] = a.m.lay_cap[ph ^ 1][d];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *a.m.phase = ph ^ 1;
    *a.m.tile_counter = 0u;
  }
}

// Input = buffer 1, one compacted segment per given count (seg bounds).
__global__ void k_input_meta(StepArgs a, const int64_t *seg_dev) {
  const int P = a.geo.Ptot;
  for (int d = threadIdx.x; d < P; d += blockDim.x) {
    a.m.lay_base[1][d] = seg_dev[d];
    a.m.lay_cap[1][d] = seg_dev[d + 1] - seg_dev[d];
    a.m.cnt[d] = seg_dev[d + 1] - seg_dev[d];
  }
  for (int d = threadIdx.x; d <= P; d += blockDim.x) a.m.cstart[d] = seg_dev[d];
  if (threadIdx.x == 0) *a.m.phase = 1;
}

__global__ void k_iota(uint32_t *p, const int64_t *cstart, int P) {
  const int64_t n = cstart[P];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (uint32_t)i;
}

// Copy the input buffer's live particles to a compacted record set.
__global__ void k_compact(StepArgs a, Rec out) {
  const int ph = *a.m.phase;
  const Rec A = a.buf[ph];
  const int64_t *base = a.m.lay_base[ph];
  const int P = a.geo.Ptot;
  const int64_t n = a.m.cstart[P];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t slot;
    if (a.perm) {  // a pending cell-sort permutation: rank i is input slot perm[i]
      slot = a.perm[i];
      if (slot >= a.cap) {  // corrupt permutation: report, never read out of bounds
        latch(a.m.status, LCS_ERR_STATE);
        continue;
      }
    } else {
      const int seg = find_segment64(a.m.cstart, P, i);
      slot = base[seg] + (i - a.m.cstart[seg]);
    }
    copy_rec(A, slot, out, i);
  }
}

// The C ABI's FP64 state <-> the records' fixed-point positions and
// float-pair velocities, in place on the first n records of R (the FP64
// values occupy the same 8-byte slots).
//   import: a position outside [0, L) is first folded into the periodic box
//           (Sec. 2.1): x' = x - k L with k = floor(x / L), one FMA rounding,
//           a result below 0 or at L moved by one more image; k is added to
//           the particle's image count when images are tracked.  A
//           non-finite position, or one more than 2^30 boxes away, latches
//           LCS_ERR_ARG.  Then q = RN(x' N/L) 2^52 exactly (the product has at
//           most 53 bits, of which at least 42 are fraction bits for
//           N <= 1024); a product that rounds up to N maps to the last
//           fixed-point value below N, so that the cell is
//           min(floor(x' N/L), N-1);
//           v -> (RN32(v), RN32(v - hi)) (a non-finite velocity is reported
//           as LCS_ERR_NONFINITE by the next step).
//   export: x = RN(RN(q) L/N 2^-52), kept below L; v = hi + lo exactly.
__device__ __forceinline__ double fold_pos(double x, double L, int &img, int *status) {
  if (x >= 0.0 && x < L) return x;
  double k = floor(x / L);
  if (!(fabs(k) < 1073741824.0)) {  // also catches NaN and infinities
    latch(status, LCS_ERR_ARG);
    return 0.0;
  }
  double y = fma(-k, L, x);
  if (y < 0.0) {
    y += L;
    k -= 1.0;
  }
  if (y >= L) {
    y -= L;
    k += 1.0;
  }
  if (!(y >= 0.0 && y < L)) y = 0.0;  // not reached for finite x; keeps q in range
  img += (int)k;
  return y;
}

__device__ __forceinline__ unsigned long long import_pos(double x, const Geom &g) {
  long long q = d_to_fix52(__dmul_rn(x, g.inv_dx));
  if (q >= g.qL) q = g.qL - 1;
  return (unsigned long long)q;
}

__global__ void k_import(Rec R, int64_t n, Geom g, int *status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int img = R.img[s] ? R.img[s][i] : 0;
      const double x =
          fold_pos(__longlong_as_double((long long)R.x[s][i]), g.L, img, status);
      if (R.img[s]) R.img[s][i] = img;
      R.x[s][i] = (int64_t)import_pos(x, g);
      const double v = __longlong_as_double(*(const long long *)&R.v[s][i]);
      const float h = __double2float_rn(v);  // non-finite values surface in the next step
      R.v[s][i] = make_float2(h, __double2float_rn(v - (double)h));
    }
  }
}

__global__ void k_export(Rec R, int64_t n, Geom g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      R.x[s][i] = __double_as_longlong(export_pos((long long)R.x[s][i], g));
      const float2 p = R.v[s][i];
      *(double *)&R.v[s][i] = (double)p.x + (double)p.y;
    }
  }
}

// Sort keys of the id-ordered export: the ids of the compacted records,
// with their positions as payload.
__global__ void k_id_keys(Rec R, int64_t n, uint32_t *key, uint32_t *pay) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    key[i] = R.id[i];
    pay[i] = (uint32_t)i;
  }
}

// Id-ordered export: record r of D is record pay[r] of the exported
// (FP64) records S; with images, the position is unwrapped, x + L img (in
// FP64: RN(x + RN(L img))).  D's position and velocity rows receive FP64
// values, its id row the ids.
__global__ void k_by_id(Rec S, const uint32_t *pay, int64_t n, Rec D, double L) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = pay[r];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      double x = __longlong_as_double((long long)S.x[s][i]);
      if (S.img[s]) x = __dadd_rn(x, __dmul_rn(L, (double)S.img[s][i]));
      D.x[s][r] = __double_as_longlong(x);
      D.v[s][r] = S.v[s][i];
    }
    D.id[r] = S.id[i];
  }
}

// Stateless partition helpers.
__global__ void k_partition_in(const uint32_t *keys, int64_t n, uint32_t nbins, uint32_t *k,
                               uint32_t *p, int32_t *status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = keys[i];
    if (v >= nbins) {
      v = nbins - 1;
      if (status) atomicCAS(status, 0, LCS_ERR_ARG);
    }
    k[i] = v;
    p[i] = (uint32_t)i;
  }
}

__global__ void k_partition_tables(int64_t n, int64_t *cs1, int *to1, int32_t *status) {
  cs1[0] = 0, cs1[1] = n;
  to1[0] = 0, to1[1] = (int)((n + SORT_TILE - 1) / SORT_TILE);
  if (status) *status = LCS_OK;
}

}  // namespace lcs
