// lcs_partition_noalloc: the stable partition of lcs_partition without any
// device allocation.
//
// Who needs it: callers that must not allocate device memory at the point
// where they partition -- for example code that runs while its stream is
// being captured into a CUDA graph (an allocation there fails or turns into
// a graph-owned memory node), code that runs under a fixed device-memory
// budget reserved up front, and latency-critical loops that cannot afford
// the implicit synchronisation of cudaMalloc / cudaFree.  They still pass
// their own input and output buffers; only the internal scratch moves.
//
// The scratch is one file-scope __device__ array of NOALLOC_BYTES bytes
// (about 13.6 MB), sized for n <= LCS_PARTITION_NOALLOC_MAX_N keys.  Every
// GPU that loads the library holds it until the process exits.  Host code
// must not pass the array's name to a kernel (on the host it is only a
// stand-in symbol); the device address is obtained with cudaGetSymbolAddress
// during the first call on a device, and again whenever that device's
// current context has changed since (after cudaDeviceReset the module is
// loaded anew and the array may sit elsewhere).
#include <algorithm>
#include <mutex>

#include <cuda.h>  // CUcontext / CUresult types; the functions come through the runtime

#include "lcs_internal.cuh"

namespace lcs {
__global__ void k_bin_bounds(const uint32_t *key, const int64_t *cs1, int shift, int nbins,
                             int64_t *start);
__global__ void k_partition_in(const uint32_t *keys, int64_t n, uint32_t nbins, uint32_t *k,
                               uint32_t *p, int32_t *status);
__global__ void k_partition_tables(int64_t n, int64_t *cs1, int *to1, int32_t *status);
}  // namespace lcs

namespace {

using namespace lcs;

constexpr int64_t MAX_N = LCS_PARTITION_NOALLOC_MAX_N;
constexpr int MAX_TILES = (int)(MAX_N / SORT_TILE + 2);
constexpr int64_t HIST_INTS = (int64_t)MAX_TILES * SORT_MAX_D;
constexpr int64_t BLOCK_INTS = HIST_INTS / 4096 + 2;

constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }
constexpr size_t OFF_KEY0 = 0;
constexpr size_t OFF_KEY1 = OFF_KEY0 + align16(MAX_N * 4);
constexpr size_t OFF_PAY0 = OFF_KEY1 + align16(MAX_N * 4);
constexpr size_t OFF_HIST = OFF_PAY0 + align16(MAX_N * 4);
constexpr size_t OFF_HSCAN = OFF_HIST + align16(HIST_INTS * 4);
constexpr size_t OFF_BLOCKS = OFF_HSCAN + align16(HIST_INTS * 4);
constexpr size_t OFF_CS1 = OFF_BLOCKS + align16(BLOCK_INTS * 4);
constexpr size_t OFF_TO1 = OFF_CS1 + 16;
constexpr size_t NOALLOC_BYTES = OFF_TO1 + 16;

__device__ __align__(256) unsigned char g_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void *g_scratch_addr[MAX_DEVICES] = {};
unsigned long long g_scratch_ctx[MAX_DEVICES] = {};  // context id the address belongs to

using CtxGetCurrent = CUresult (*)(CUcontext *);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (cuCtxGetId, reached
// through the runtime's driver entry points; ids are never reused within a
// process), or 0 if it cannot be read.  Call with g_mutex held.
unsigned long long current_context_id() {
  static CtxGetCurrent get_current = nullptr;
  static CtxGetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    resolved = true;
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1{}, q2{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = (CtxGetCurrent)f;
      get_id = (CtxGetId)g;
    }
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of g_scratch in the current device's current context:
// looked up on the first call on a device and again when the context has
// changed since (or its id cannot be read).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = current_context_id();  // the lookup may have created the context
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

int ceil_log2_i(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}

}  // namespace

extern "C" lcs_status lcs_partition_noalloc(const uint32_t *keys, int64_t n, int nbins,
                                            uint32_t *perm, int64_t *bin_off, int32_t *status,
                                            void *stream) {
  if (n < 0 || n > MAX_N || nbins < 1 || nbins > 65536 || (n > 0 && (!keys || !perm)) ||
      !bin_off)
    return LCS_ERR_ARG;
  void *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return LCS_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *p = (unsigned char *)base;
  SortArgs s{};
  s.key[0] = (uint32_t *)(p + OFF_KEY0);
  s.key[1] = (uint32_t *)(p + OFF_KEY1);
  s.pay[0] = (uint32_t *)(p + OFF_PAY0);
  s.pay[1] = perm;
  s.hist = (int *)(p + OFF_HIST);
  s.hist_scan = (int *)(p + OFF_HSCAN);
  s.scan_blocks = (int *)(p + OFF_BLOCKS);
  int64_t *cs1 = (int64_t *)(p + OFF_CS1);
  int *to1 = (int *)(p + OFF_TO1);
  s.nseg = 1, s.cstart = cs1, s.tile_off = to1;
  s.max_tiles = (int)(n / SORT_TILE + 2);
  // Nothing in the scratch needs to start at zero: the tables, histograms,
  // scans and key/payload buffers are fully written before they are read.
  const int gs = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, device_sms() * 8));
  k_partition_tables<<<1, 1, 0, st>>>(n, cs1, to1, status);
  if (n > 0) k_partition_in<<<gs, 256, 0, st>>>(keys, n, (uint32_t)nbins, s.key[0], s.pay[0], status);
  int ob = 0;
  cudaError_t err = radix_sort(s, ceil_log2_i(nbins), &ob, st, nullptr);
  if (err == cudaSuccess) {
    if (ob == 0 && n > 0) err = cudaMemcpyAsync(perm, s.pay[0], n * 4, cudaMemcpyDeviceToDevice, st);
  }
  if (err == cudaSuccess) {
    k_bin_bounds<<<gs, 256, 0, st>>>(s.key[ob], cs1, 0, nbins, bin_off);
    err = cudaGetLastError();
  }
  return err == cudaSuccess ? LCS_OK : LCS_ERR_CUDA;
}
