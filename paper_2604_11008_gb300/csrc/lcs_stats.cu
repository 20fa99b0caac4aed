// Particle statistics: histogram of pair separations, the counts behind the
// radial distribution function g(r) used to validate the particle phase
// (Sec. 3, particle-phase validation: g at contact quantifies clustering).
//
// Pairs closer than r_max <= L/N lie in the same or adjacent grid cells, so
// the particles are sorted by cell (the library's radix sort, one segment),
// every particle scans the 27 cells around its own, and each unordered pair
// is counted once (by the partner later in cell order).  Separations use
// the positions exactly as lcs_get_state returns them, with the minimum
// image of the periodic box and the operation order of the definition
// (r^2 = (dx dx + dy dy) + dz dz, r = sqrt(r^2), bin = floor(r nbins/r_max)),
// so the integer counts equal a brute-force count over those positions.
#include "lcs_internal.cuh"

namespace lcs {

// Global cell id (x fastest) of each live particle, by the FP64 product of
// its returned position (the cell a brute-force count would see), and its
// slot in the input buffer.
__global__ void k_pair_keys(StepArgs a, uint32_t *key, uint32_t *pay) {
  const int ph = *a.m.phase;
  const Rec A = a.buf[ph];
  const int64_t *base = a.m.lay_base[ph];
  const int P = a.geo.Ptot, N = a.geo.N;
  const int64_t n = a.m.cstart[P];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int seg = find_segment64(a.m.cstart, P, i);
    const int64_t slot = base[seg] + (i - a.m.cstart[seg]);
    int c[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const double x = export_pos((long long)A.x[s][slot], a.geo);
      c[s] = min(max((int)floor(__dmul_rn(x, a.geo.inv_dx)), 0), N - 1);
    }
    key[i] = (uint32_t)(c[0] + N * (c[1] + N * c[2]));
    pay[i] = (uint32_t)slot;
  }
}

// start[c] = first sorted position with key >= c, for c in [0, ncell].
__global__ void k_cell_starts(const uint32_t *key, int64_t n, int64_t ncell, int *start) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (key[mid] < (uint64_t)c) lo = mid + 1; else hi = mid;
    }
    start[c] = (int)lo;
  }
}

constexpr int PAIR_BLOCK = 256, PAIR_MAX_BINS = 4096;

__global__ void __launch_bounds__(PAIR_BLOCK)
    k_pair_hist(StepArgs a, const uint32_t *key, const uint32_t *pay, const int *start,
                int64_t n, double r_max, double inv_w, int nbins, unsigned long long *counts) {
  __shared__ unsigned int h[PAIR_MAX_BINS];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0u;
  __syncthreads();
  const Rec A = a.buf[*a.m.phase];
  const Geom &g = a.geo;
  const int N = g.N;
  const double half = 0.5 * g.L;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t si = pay[p], c = key[p];
    const int cx = (int)(c % (uint32_t)N), cy = (int)((c / (uint32_t)N) % (uint32_t)N),
              cz = (int)(c / ((uint32_t)N * (uint32_t)N));
    double xi[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) xi[s] = export_pos((long long)A.x[s][si], g);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int nx = (cx + dx + N) % N, ny = (cy + dy + N) % N, nz = (cz + dz + N) % N;
          const int64_t nc = (int64_t)nx + (int64_t)N * (ny + (int64_t)N * nz);
          const int64_t q0 = max((int64_t)start[nc], p + 1), q1 = start[nc + 1];
          for (int64_t q = q0; q < q1; ++q) {
            const uint32_t sj = pay[q];
            double d[3];
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              double e = __dsub_rn(xi[s], export_pos((long long)A.x[s][sj], g));
              if (e > half) e = __dsub_rn(e, g.L);
              else if (e < -half) e = __dadd_rn(e, g.L);
              d[s] = e;
            }
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                        __dmul_rn(d[2], d[2]));
            const double r = __dsqrt_rn(r2);
            if (r < r_max) atomicAdd(&h[min((int)__dmul_rn(r, inv_w), nbins - 1)], 1u);
          }
        }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (h[b]) atomicAdd(counts + b, (unsigned long long)h[b]);
}

cudaError_t launch_pair_keys(const StepArgs &a, uint32_t *key, uint32_t *pay, int64_t n,
                             int grid, cudaStream_t st) {
  k_pair_keys<<<grid, 256, 0, st>>>(a, key, pay);
  (void)n;
  return cudaGetLastError();
}

cudaError_t launch_pair_hist(const StepArgs &a, const uint32_t *key, const uint32_t *pay,
                             int *start, int64_t n, double r_max, int nbins,
                             unsigned long long *counts, int sms, cudaStream_t st) {
  const int64_t ncell = (int64_t)a.geo.N * a.geo.N * a.geo.N;
  const int cg = (int)std::min<int64_t>((ncell + 256) / 256, (int64_t)sms * 16);
  k_cell_starts<<<cg, 256, 0, st>>>(key, n, ncell, start);
  const int pg = (int)std::max<int64_t>(1, std::min<int64_t>((n + PAIR_BLOCK - 1) / PAIR_BLOCK,
                                                             (int64_t)sms * 8));
  k_pair_hist<<<pg, PAIR_BLOCK, 0, st>>>(a, key, pay, start, n, r_max, (double)nbins / r_max,
                                         nbins, counts);
  return cudaGetLastError();
}

}  // namespace lcs
