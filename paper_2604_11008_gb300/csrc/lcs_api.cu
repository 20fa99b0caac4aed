// C ABI of liblcs: context creation, the captured step loop, standalone
// migration / sort passes, state I/O and the stateless partition.
// See include/lcs.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lcs_internal.cuh"

using namespace lcs;

namespace lcs {
// kernels defined in lcs_sort.cu
__global__ void k_keys_cell(StepArgs a, uint32_t *key, uint32_t *pay, int B, int nbx, int nby);
__global__ void k_keys_dest(StepArgs a, uint32_t *key, uint32_t *pay);
__global__ void k_one_segment(const int64_t *cstart, int P, int64_t *cs1, int *to1);
__global__ void k_bin_bounds(const uint32_t *key, const int64_t *cs1, int shift, int nbins,
                             int64_t *start);
__global__ void k_relayout(StepArgs a, int from_starts);
__global__ void k_gather(StepArgs a, const uint32_t *pay);
__global__ void k_set_phase(StepArgs a);
__global__ void k_input_meta(StepArgs a, const int64_t *seg_dev);
__global__ void k_iota(uint32_t *p, const int64_t *cstart, int P);
__global__ void k_compact(StepArgs a, Rec out);
__global__ void k_import(Rec R, int64_t n, Geom g, int *status);
__global__ void k_export(Rec R, int64_t n, Geom g);
__global__ void k_id_keys(Rec R, int64_t n, uint32_t *key, uint32_t *pay);
__global__ void k_by_id(Rec S, const uint32_t *pay, int64_t n, Rec D, double L);
__global__ void k_partition_in(const uint32_t *keys, int64_t n, uint32_t nbins, uint32_t *k,
                               uint32_t *p, int32_t *status);
__global__ void k_partition_tables(int64_t n, int64_t *cs1, int *to1, int32_t *status);
}  // namespace lcs

namespace {

int ceil_log2(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}

struct Ens {
  lcs_desc d{};
  FieldKind kind = FK_F64;
  int64_t np = 0, cap = 0;
  int brick = 8, nb[3] = {1, 1, 1}, key_bits = 0, mig_bits = 1;
  int max_tiles = 0, max_stiles = 0, step_grid = 1;
  void *field = nullptr;
  void *field_b = nullptr;  // second snapshot (evolving field) or nullptr
  void *bricks = nullptr;   // owned-field mode: the subdomains' field bricks
  void *bricks_b = nullptr; // the same for the second snapshot (evolving field)
  double t_a = 0.0, t_b = 1.0;
  StepArgs a{};
  SortArgs s{};
  int64_t *cs1 = nullptr;
  int *to1 = nullptr;
  int64_t steps = 0;
  int id_bits = 32;  // key width of the id sort (ceil log2 np for the default ids)
  // cell sort computed but not applied: its permutation sits in s.pay[perm],
  // and the next step reads the records through it (-1: none pending)
  int perm = -1;
  // adjoint tape: checkpoint k holds the state after k*ckpt_every steps
  std::vector<TapeSlot> tape;
  bool tape_ok = false;
  unsigned long long *states = nullptr;  // recomputed states of one segment (k_recompute)
  double *lam_id = nullptr, *lam_s = nullptr;
};

// Step-kernel configuration: threads per block, particles per thread, mode.
struct StepCfg {
  int block = 256, items = 1, mode = LCS_STEP_DEFERRED;
};

// One step-kernel launch: its ensembles (at most GROUP_ENS) and configuration.
struct Group {
  std::vector<int> ens;
  StepCfg cfg;
  int64_t tiles = 0;  // look-back array size of the launch
};

}  // namespace

struct lcs_ctx {
  std::vector<Ens> ens;
  cudaStream_t st = nullptr;      // the caller's stream: all work runs here
  cudaStream_t cap_st = nullptr;  // private stream used only to record graphs
  int failed = 0;  // latched host-side status (LCS_ERR_*)
  std::string err;
  std::vector<void *> allocs;
  // Step period Q: the least common multiple of the ensembles' sort_every and
  // ckpt_every (0 when it exceeds MAX_PERIOD).  With Q > 0 lcs_step records
  // runs of consecutive steps that end at multiples of Q, checkpoint steps
  // or the end of the call as one graph each: the same run of sorts repeats
  // every Q steps.  Without a period every step is its own graph.
  int64_t period = 0;
  struct RunGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int> perm_out;  // pending permutations a replay leaves
    int64_t launches = 0;       // kernel launches of one replay
  };
  // Recorded runs, keyed by (step count mod Q at the start, or -1 without a
  // period; number of steps; the pending permutation of every ensemble at
  // the start; without a period, which ensembles sort after the step).
  using RunKey = std::tuple<int64_t, int64_t, std::vector<int>, std::vector<bool>>;
  std::map<RunKey, RunGraph> chunk_graphs;
  int64_t launches = 0;
  int64_t graph_launches = 0;  // cudaGraphLaunch calls of lcs_step
  int sms = 0;  // streaming multiprocessors of the context's device
  // batched step over all ensembles (one launch per kernel per step)
  FieldKind kind = FK_F64;
  bool pf_tau = false, pf_img = false;  // some ensemble has per-particle tau / images
  bool evolve = false;  // some ensemble has an evolving field (mode-3 kernels only)
  bool per_stage = false;  // migration after each Runge-Kutta stage (modes 3 and 4 only)
  bool owned = false;      // owned-field mode (mode-4 kernels only)
  int step_grid = 1, total_P = 0;
  int64_t total_tiles = 0;      // sum of the ensembles' look-back array sizes
  unsigned long long *tile_status = nullptr;
  BatchArgs bt{};
  StepArgs *d_args = nullptr;
  int *d_ens_P_off = nullptr;
  unsigned *d_counter = nullptr;  // one tile counter per step group (n_ens + 1 of them)
  std::vector<StepCfg> cfg;       // step-kernel configuration of every ensemble
  std::vector<Group> groups;      // the step-kernel launches of one step
};

namespace {

thread_local std::string g_last_init_error = "no error";

// Ensembles that share a step-kernel configuration are advanced by one
// launch per GROUP_ENS of them; during lcs_tune also split by class.
void regroup(lcs_ctx *c, const std::vector<int> *cls) {
  const int n = (int)c->ens.size();
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  auto key = [&](int k) {
    return std::make_tuple(cls ? (*cls)[k] : 0, c->cfg[k].mode, c->cfg[k].block,
                           c->cfg[k].items);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key(a) < key(b); });
  c->groups.clear();
  for (int i = 0; i < n;) {
    Group g;
    g.cfg = c->cfg[order[i]];
    int j = i;
    while (j < n && key(order[j]) == key(order[i]) && (int)g.ens.size() < GROUP_ENS) {
      g.ens.push_back(order[j]);
      g.tiles += c->ens[order[j]].max_tiles;
      ++j;
    }
    c->groups.push_back(std::move(g));
    i = j;
  }
  c->bt.ngroups = (int)c->groups.size();
}

lcs_status fail(lcs_ctx *c, lcs_status s, const std::string &msg) {
  if (c) {
    if (!c->failed) c->failed = s;
    c->err = msg;
  }
  g_last_init_error = msg;
  return s;
}

// An argument error of a call on a live context: the call does nothing and
// the context stays usable (no error is latched).
lcs_status reject(lcs_ctx *c, const std::string &msg) {
  c->err = msg;
  g_last_init_error = msg;
  return LCS_ERR_ARG;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, e_ == cudaErrorMemoryAllocation ? LCS_ERR_OOM : LCS_ERR_CUDA,       \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

template <class T>
cudaError_t dalloc(lcs_ctx *c, T **p, int64_t n) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) {
    c->allocs.push_back(q);
    *p = (T *)q;
  }
  return e;
}

// For every destination subdomain d, the (source, direction) pairs whose
// leavers arrive in d, by ascending source id (each source appears once;
// -1 pads the row of 26).  Fixed by the subdomain grid alone.
std::vector<int> finish_table(const int Pd[3]) {
  const int P = Pd[0] * Pd[1] * Pd[2];
  std::vector<int> tab((size_t)P * (NBIN - 1), -1);
  for (int d = 0; d < P; ++d) {
    const int pd[3] = {d % Pd[0], (d / Pd[0]) % Pd[1], d / (Pd[0] * Pd[1])};
    std::vector<std::pair<int, int>> in;
    for (int b = 0; b < NBIN; ++b) {
      if (b == BIN_STAY) continue;
      const int dir[3] = {b % 3 - 1, (b / 3) % 3 - 1, b / 9 - 1};
      int ps[3], ok = 1;
      for (int q = 0; q < 3; ++q) {
        ps[q] = ((pd[q] - dir[q]) % Pd[q] + Pd[q]) % Pd[q];
        if (dir_comp(ps[q], pd[q], Pd[q]) != dir[q]) ok = 0;
      }
      if (!ok) continue;
      const int src = ps[0] + Pd[0] * (ps[1] + Pd[1] * ps[2]);
      if (src != d) in.push_back({src, b});
    }
    std::sort(in.begin(), in.end());
    for (size_t j = 0; j < in.size(); ++j)
      tab[(size_t)d * (NBIN - 1) + j] = in[j].first * NBIN + in[j].second;
  }
  return tab;
}

// Record arrays get 4 elements (>= 16 bytes) of slack: the step kernel's bulk
// copies round a tile's rows out to 16-byte boundaries.
lcs_status alloc_rec(lcs_ctx *c, Rec &r, int64_t cap, bool has_tau, bool has_img, bool has_vs) {
  cap += 4;
  for (int s = 0; s < 3; ++s) {
    r.vs[s] = nullptr;
    if (has_vs) CK(dalloc(c, &r.vs[s], cap));
    CK(dalloc(c, &r.x[s], cap));
    CK(dalloc(c, &r.v[s], cap));
    r.img[s] = nullptr;
    if (has_img) CK(dalloc(c, &r.img[s], cap));
  }
  r.tau = nullptr;
  if (has_tau) CK(dalloc(c, &r.tau, cap));
  CK(dalloc(c, &r.id, cap));
  return LCS_OK;
}

int grid_for(int64_t n, int block, int cap_blocks) {
  int64_t g = (n + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap_blocks));
}

// The standalone migration: stable sort of the whole live set by
// 2*dest + (dest != source), new counts from the bin starts, gather.
lcs_status enqueue_migrate(lcs_ctx *c, Ens &e) {
  cudaStream_t st = c->st;  // never captured
  const int gs = grid_for(e.np, 256, c->sms * 8);
  k_keys_dest<<<gs, 256, 0, st>>>(e.a, e.s.key[0], e.s.pay[0]);
  k_one_segment<<<1, 1, 0, st>>>(e.a.m.cstart, e.a.geo.Ptot, e.cs1, e.to1);
  SortArgs s = e.s;
  s.nseg = 1, s.cstart = e.cs1, s.tile_off = e.to1;
  int ob = 0;
  CK(radix_sort(s, e.mig_bits, &ob, st, &c->launches));
  k_bin_bounds<<<gs, 256, 0, st>>>(s.key[ob], e.cs1, 1, e.a.geo.Ptot, e.a.m.cstart);
  k_relayout<<<1, 1024, 0, st>>>(e.a, 1);
  k_gather<<<gs, 256, 0, st>>>(e.a, s.pay[ob]);
  k_set_phase<<<1, 1024, 0, st>>>(e.a);
  c->launches += 7;
  CK(cudaGetLastError());
  return LCS_OK;
}

// The cell sort, first half: keys and the stable per-segment radix sort by
// brick-major cell key; *ob receives the payload buffer holding the
// permutation (sorted rank -> input slot).
lcs_status enqueue_sort_keys(lcs_ctx *c, Ens &e, cudaStream_t st, int *ob) {
  const int gs = grid_for(e.np, 256, c->sms * 8);
  k_keys_cell<<<gs, 256, 0, st>>>(e.a, e.s.key[0], e.s.pay[0], e.brick, e.nb[0], e.nb[1]);
  *ob = 0;
  CK(radix_sort(e.s, e.key_bits, ob, st, &c->launches));
  c->launches += 1;
  CK(cudaGetLastError());
  return LCS_OK;
}

// The second half: the records permuted into the other buffer, which becomes
// the input.
lcs_status enqueue_apply_perm(lcs_ctx *c, Ens &e, cudaStream_t st, int ob) {
  const int gs = grid_for(e.np, 256, c->sms * 8);
  k_relayout<<<1, 1024, 0, st>>>(e.a, 0);
  k_gather<<<gs, 256, 0, st>>>(e.a, e.s.pay[ob]);
  k_set_phase<<<1, 1024, 0, st>>>(e.a);
  c->launches += 3;
  CK(cudaGetLastError());
  return LCS_OK;
}

// The whole cell sort.
lcs_status enqueue_sort(lcs_ctx *c, Ens &e, cudaStream_t st) {
  int ob = 0;
  lcs_status r = enqueue_sort_keys(c, e, st, &ob);
  return r == LCS_OK ? enqueue_apply_perm(c, e, st, ob) : r;
}

// Apply every pending sort permutation (before anything but the step kernel
// reads the records, or before a configuration change).
lcs_status materialize(lcs_ctx *c) {
  for (auto &e : c->ens) {
    if (e.perm < 0) continue;
    lcs_status r = enqueue_apply_perm(c, e, c->st, e.perm);
    if (r != LCS_OK) return r;
    e.perm = -1;
  }
  return LCS_OK;
}

struct Prof;
void prof_mark(Prof *pf, cudaStream_t st, int cls);

// The step kernel of every group of ensembles (one launch per group; with
// pf, an event pair around each launch, class 1000 + group index).
lcs_status launch_steps(lcs_ctx *c, cudaStream_t st, int stage, Prof *pf = nullptr) {
  static thread_local StepGroup<GROUP_ENS> big;
  for (size_t gi = 0; gi < c->groups.size(); ++gi) {
    const Group &gr = c->groups[gi];
    const StepCfg &k = gr.cfg;
    const int cnt = (int)gr.ens.size();
    const int occ = std::max(
        1, step_kernel_occupancy(c->kind, k.mode, k.block, k.items, c->evolve, stage,
                                 c->pf_tau, c->pf_img, c->per_stage));
    const int grid =
        (int)std::max<int64_t>(1, std::min<int64_t>(gr.tiles, (int64_t)occ * c->sms));
    if (pf) prof_mark(pf, st, 1000 + (int)gi);
    if (cnt == 1) {
      StepGroup<1> one;
      one.a[0] = c->ens[gr.ens[0]].a;
      one.n = 1;
      one.pf_tau = c->pf_tau;
      one.pf_img = c->pf_img;
      one.pf_vs = c->per_stage;
      one.counter = c->d_counter + gi;
      CK(launch_step_group<1>(one, c->kind, k.mode, k.block, k.items, c->evolve, stage, grid,
                              st));
    } else {
      for (int j = 0; j < cnt; ++j) big.a[j] = c->ens[gr.ens[j]].a;
      big.n = cnt;
      big.pf_tau = c->pf_tau;
      big.pf_img = c->pf_img;
      big.pf_vs = c->per_stage;
      big.counter = c->d_counter + gi;
      CK(launch_step_group<GROUP_ENS>(big, c->kind, k.mode, k.block, k.items, c->evolve, stage,
                                      grid, st));
    }
    c->launches += 1;
  }
  return LCS_OK;
}

// Whether the step kernel of ensemble k reads its records through a pending
// cell-sort permutation (the modes that read every record by its slot).
bool fuses_sort(const lcs_ctx *c, size_t k) {
  const int m = c->cfg[k].mode;
  return m == LCS_STEP_DEFERRED || m == LCS_STEP_OWNED_FIELD;
}

// Before a step: a pending permutation is handed to the step kernel where
// its mode reads through it, else applied first.
lcs_status take_pending(lcs_ctx *c, cudaStream_t st) {
  for (size_t k = 0; k < c->ens.size(); ++k) {
    Ens &e = c->ens[k];
    e.a.perm = nullptr;
    if (e.perm < 0) continue;
    if (fuses_sort(c, k)) {
      e.a.perm = e.s.pay[e.perm];
    } else {
      lcs_status r = enqueue_apply_perm(c, e, st, e.perm);
      if (r != LCS_OK) return r;
    }
    e.perm = -1;
  }
  return LCS_OK;
}

void clear_step_perm(lcs_ctx *c) {
  for (auto &e : c->ens) e.a.perm = nullptr;
}

// After a step: the cell sort of the ensembles in `sorts`; where the next
// step kernel can read through the permutation, only the keys and the radix
// passes run now.
lcs_status enqueue_sorts(lcs_ctx *c, const std::vector<bool> &sorts, cudaStream_t st) {
  for (size_t k = 0; k < c->ens.size(); ++k) {
    if (!sorts[k]) continue;
    Ens &e = c->ens[k];
    lcs_status r;
    if (fuses_sort(c, k)) {
      int ob = 0;
      r = enqueue_sort_keys(c, e, st, &ob);
      e.perm = ob;
    } else {
      r = enqueue_sort(c, e, st);
    }
    if (r != LCS_OK) return r;
  }
  return LCS_OK;
}

// One step of every ensemble: (launch groups + 1) launches -- the step
// kernel of every group, then the step tail (unpack, next layout, buffer
// swap, look-back words cleared for the next step) -- whatever the number
// of ensembles; twice that with migration per stage (the predictor pass,
// then the corrector).  A pending sort permutation is consumed by the first
// pass.
lcs_status enqueue_step(lcs_ctx *c, cudaStream_t st) {
  lcs_status r = take_pending(c, st);
  if (r != LCS_OK) return r;
  const int passes = c->per_stage ? 2 : 1;
  for (int p = 0; p < passes; ++p) {
    const int stage = c->per_stage ? p + 1 : 0;
    lcs_status rs = launch_steps(c, st, stage);
    clear_step_perm(c);
    if (rs != LCS_OK) return rs;
    CK(launch_tail(c->bt, c->total_P, st, p == passes - 1));
    c->launches += 1;
  }
  return LCS_OK;
}

// Un-graphed step with an event pair around each kernel class.
struct Prof {
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls;
  cudaEvent_t get() {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    ev.push_back(e);
    return e;
  }
};

// Record an event opening the interval of class `cls` (up to the next mark).
void prof_mark(Prof *pf, cudaStream_t st, int cls) {
  cudaEventRecord(pf->get(), st);
  pf->cls.push_back(cls);
}

lcs_status enqueue_step_profiled(lcs_ctx *c, const std::vector<bool> &sorts, Prof &pf) {
  cudaStream_t st = c->st;
  auto mark = [&](int cls) {
    cudaEvent_t e0 = pf.get();
    cudaEventRecord(e0, st);
    pf.cls.push_back(cls);
  };
  bool pending = false;
  for (auto &e : c->ens) pending |= e.perm >= 0;
  if (pending) mark(LCS_PROF_SORT);  // a permutation applied before the step
  lcs_status r = take_pending(c, st);
  if (r != LCS_OK) return r;
  const int passes = c->per_stage ? 2 : 1;
  for (int p = 0; p < passes; ++p) {
    lcs_status rs = launch_steps(c, st, c->per_stage ? p + 1 : 0, &pf);
    clear_step_perm(c);
    if (rs != LCS_OK) return rs;
    mark(LCS_PROF_TAIL);
    CK(launch_tail(c->bt, c->total_P, st, p == passes - 1));
    c->launches += 1;
  }
  bool any = false;
  for (bool b : sorts) any |= b;
  if (any) {
    mark(LCS_PROF_SORT);
    r = enqueue_sorts(c, sorts, st);
    if (r != LCS_OK) return r;
  }
  mark(-1);
  return LCS_OK;
}

std::vector<bool> sort_set(lcs_ctx *c, int64_t next);

// Record `len` consecutive steps of every ensemble as one CUDA graph, the
// first of them step number first_step (1-based), each followed by the cell
// sort of the ensembles that sort after it.  The pending permutations of the
// context move on as if the steps had run (the graph starts from the ones
// given at capture and leaves the ones the context then holds); *nlaunch
// receives the kernel launches of one replay.
lcs_status capture(lcs_ctx *c, int64_t first_step, int64_t len, cudaGraphExec_t *out,
                   int64_t *nlaunch) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal));
  lcs_status r = LCS_OK;
  const int64_t l0 = c->launches;
  for (int64_t j = 0; j < len && r == LCS_OK; ++j) {
    const std::vector<bool> sorts = sort_set(c, first_step + j);
    r = enqueue_step(c, c->cap_st);
    if (r == LCS_OK) r = enqueue_sorts(c, sorts, c->cap_st);
  }
  *nlaunch = c->launches - l0;
  c->launches = l0;  // counted again at each replay
  cudaError_t ee = cudaStreamEndCapture(c->cap_st, &g);
  if (r != LCS_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  CK(ee);
  cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(ie);
  return LCS_OK;
}

// Which ensembles sort after step number `next` (1-based).
std::vector<bool> sort_set(lcs_ctx *c, int64_t next) {
  std::vector<bool> s(c->ens.size());
  for (size_t k = 0; k < c->ens.size(); ++k) {
    const int se = c->ens[k].d.sort_every;
    s[k] = se > 0 && next % se == 0;
  }
  return s;
}

void drop_graphs(lcs_ctx *c) {
  for (auto &kv : c->chunk_graphs) cudaGraphExecDestroy(kv.second.exec);
  c->chunk_graphs.clear();
}

// Record checkpoint k of ensemble e (allocating its slot on first use).
lcs_status tape_store(lcs_ctx *c, Ens &e, int64_t k) {
  while ((int64_t)e.tape.size() <= k) {
    TapeSlot t{};
    CK(dalloc(c, &t.x, 3 * std::max<int64_t>(e.np, 1)));
    CK(dalloc(c, &t.v, 3 * std::max<int64_t>(e.np, 1)));
    if (e.d.tau) CK(dalloc(c, &t.tau, std::max<int64_t>(e.np, 1)));
    CK(dalloc(c, &t.id, std::max<int64_t>(e.np, 1)));
    e.tape.push_back(t);
  }
  if (e.np > 0) CK(launch_tape_store(e.a, e.tape[k], e.np, c->st));
  c->launches += 1;
  return LCS_OK;
}

lcs_status check_ctx(lcs_ctx *c) {
  if (!c) return LCS_ERR_ARG;
  if (c->failed) return LCS_ERR_STATE;
  return LCS_OK;
}

lcs_status read_status(lcs_ctx *c) {
  int dev_status = 0;
  for (auto &e : c->ens) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, e.a.m.status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (v && !dev_status) dev_status = v;
  }
  if (dev_status) {
    static const char *names[] = {"ok", "argument", "cuda", "out of memory", "capacity",
                                  "timeout", "non-finite state", "displacement", "state"};
    return fail(c, (lcs_status)dev_status,
                std::string("device reported: ") + names[dev_status < 9 ? dev_status : 0]);
  }
  return LCS_OK;
}

// Copy every ensemble's StepArgs to the device array the batched kernels read.
lcs_status upload_args(lcs_ctx *c) {
  std::vector<StepArgs> h(c->ens.size());
  for (size_t k = 0; k < c->ens.size(); ++k) h[k] = c->ens[k].a;
  CK(cudaMemcpyAsync(c->d_args, h.data(), sizeof(StepArgs) * h.size(), cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  return LCS_OK;
}

// Step-tile tables of every ensemble for the current tile size.
lcs_status retile(lcs_ctx *c) {
  for (size_t k = 0; k < c->ens.size(); ++k) {
    Ens &e = c->ens[k];
    e.a.step_tile = c->cfg[k].block * c->cfg[k].items;
    k_relayout<<<1, 1024, 0, c->st>>>(e.a, 0);
    c->launches += 1;
  }
  CK(cudaGetLastError());
  return upload_args(c);
}

// The batched view of the ensembles: one look-back status array, one tile
// counter, the device copy of every ensemble's arguments.
lcs_status setup_batch(lcs_ctx *c) {
  const int n = (int)c->ens.size();
  if (n > MAX_ENS) return fail(c, LCS_ERR_ARG, "too many ensembles in one context");
  c->kind = c->ens[0].kind;
  for (auto &e : c->ens) {
    if (e.kind != c->kind)
      return fail(c, LCS_ERR_ARG, "all ensembles of a context need the same field storage");
    c->pf_tau |= e.a.buf[0].tau != nullptr;
    c->pf_img |= e.a.buf[0].img[0] != nullptr;
    c->evolve |= e.field_b != nullptr;
    if (e.d.migrate_per_stage != c->ens[0].d.migrate_per_stage)
      return fail(c, LCS_ERR_ARG, "all ensembles of a context need the same migration schedule");
    if (e.d.owned_field != c->ens[0].d.owned_field)
      return fail(c, LCS_ERR_ARG, "all ensembles of a context need the same owned_field");
  }
  c->per_stage = c->ens[0].d.migrate_per_stage != 0;
  // step period of the recorded runs: lcm of the sort and checkpoint
  // intervals, stretched to at least 8 steps (a multiple of a period is a
  // period), none above MAX_PERIOD
  {
    constexpr int64_t MAX_PERIOD = 64;
    int64_t q = 1;
    auto lcm = [](int64_t a, int64_t b) {
      int64_t x = a, y = b;
      while (y) {
        const int64_t t = x % y;
        x = y;
        y = t;
      }
      return a / x * b;
    };
    for (auto &e : c->ens) {
      if (e.d.sort_every > 0 && q <= MAX_PERIOD) q = lcm(q, e.d.sort_every);
      if (e.d.ckpt_every > 0 && q <= MAX_PERIOD) q = lcm(q, e.d.ckpt_every);
    }
    if (q < 8) q *= (8 + q - 1) / q;
    c->period = q <= MAX_PERIOD ? q : 0;
  }
  c->owned = c->ens[0].d.owned_field != 0;
  // default step kernel (lcs_tune / lcs_set_step_config change it): the
  // deferred scatter, one particle per thread (two for FP32 and BF16
  // fields), the fastest of the configurations on the 16.8M-particle workload
  c->cfg.assign(c->ens.size(),
                StepCfg{256, c->kind == FK_BF16 || c->kind == FK_F32 ? 2 : 1,
                        c->owned ? LCS_STEP_OWNED_FIELD : LCS_STEP_DEFERRED});
  c->total_tiles = 0;
  c->total_P = 0;
  std::vector<int> poff(n + 1, 0);
  for (int k = 0; k < n; ++k) {
    c->total_tiles += c->ens[k].max_tiles;
    poff[k + 1] = poff[k] + c->ens[k].a.geo.Ptot;
  }
  c->total_P = poff[n];
  CK(dalloc(c, &c->tile_status, c->total_tiles));
  // zero once: after that every step tail clears the words its step used
  CK(cudaMemsetAsync(c->tile_status, 0, sizeof(unsigned long long) * c->total_tiles, c->st));
  int64_t off = 0;
  for (auto &e : c->ens) {
    e.a.m.tile_status = c->tile_status + off;
    off += e.max_tiles;
  }
  CK(dalloc(c, &c->d_args, n));
  CK(dalloc(c, &c->d_ens_P_off, n + 1));
  CK(dalloc(c, &c->d_counter, n + 1));  // at most one launch group per ensemble
  CK(cudaMemcpyAsync(c->d_ens_P_off, poff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned) * (n + 1), c->st));
  c->bt = BatchArgs{c->d_args, n, c->d_ens_P_off, c->d_counter, 0};
  regroup(c, nullptr);
  return retile(c);
}

}  // namespace

extern "C" {

// An NVTX range around a public entry point: the library's calls appear as
// named spans on an Nsight timeline (header-only NVTX; no cost without a tool).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

lcs_status lcs_init(const lcs_desc *ens, int n_ens, void *stream, lcs_ctx **out) {
  NvtxRange nvtx_range("lcs_init");
  if (!out) return LCS_ERR_ARG;
  *out = nullptr;
  if (!ens || n_ens < 1) return LCS_ERR_ARG;
  lcs_ctx *c = new lcs_ctx();
  c->st = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return LCS_ERR_CUDA;
  }
  c->sms = device_sms();
  c->ens.resize(n_ens);
  lcs_status r = LCS_OK;
  for (int k = 0; k < n_ens && r == LCS_OK; ++k) {
    Ens &e = c->ens[k];
    e.d = ens[k];
    const lcs_desc &d = e.d;
    const int P = d.sub[0] * d.sub[1] * d.sub[2];
    if (d.n < 2 || d.n > 1024 || !(d.box > 0) || d.np < 0 || d.np >= (int64_t(1) << 31) ||
        d.sub[0] < 1 || d.sub[1] < 1 || d.sub[2] < 1 || d.n % d.sub[0] || d.n % d.sub[1] ||
        d.n % d.sub[2] || P > 4096 || !(d.dt > 0) || !d.field || (d.np > 0 && (!d.x0 || !d.v0)) ||
        (!d.tau && !(d.tau_const >= d.dt)) || d.sort_every < 0 || d.sort_brick < 0 ||
        d.ckpt_every < 0) {
      r = fail(c, LCS_ERR_ARG, "invalid lcs_desc for ensemble " + std::to_string(k));
      break;
    }
    if (d.drag != LCS_DRAG_STOKES &&
        (d.drag != LCS_DRAG_NONLINEAR || !(d.nu > 0) || !(d.density_ratio >= 0) ||
         !std::isfinite(d.nu) || !std::isfinite(d.density_ratio))) {
      r = fail(c, LCS_ERR_ARG, "invalid drag parameters for ensemble " + std::to_string(k));
      break;
    }
    if (d.drag != LCS_DRAG_STOKES && d.ckpt_every > 0) {
      r = fail(c, LCS_ERR_ARG, "lcs_backward supports the Stokes drag only (ckpt_every > 0)");
      break;
    }
    if (d.field_next && (!(d.t_field[1] > d.t_field[0]) || !std::isfinite(d.t_field[0]) ||
                         !std::isfinite(d.t_field[1]) || !std::isfinite(d.t_start))) {
      r = fail(c, LCS_ERR_ARG, "evolving field: needs t_field[1] > t_field[0], finite times");
      break;
    }
    if (d.field_next && d.ckpt_every > 0) {
      r = fail(c, LCS_ERR_ARG, "lcs_backward supports a frozen field only (ckpt_every > 0)");
      break;
    }
    if (d.migrate_per_stage && (d.migrate_per_stage != 1 || d.ckpt_every > 0)) {
      r = fail(c, LCS_ERR_ARG, "migrate_per_stage: not with ckpt_every");
      break;
    }
    if (d.owned_field &&
        (d.owned_field != 1 || d.ckpt_every > 0 ||
         (d.field_dtype == LCS_F64 && d.field_kernel == LCS_KERNEL_FP64))) {
      r = fail(c, LCS_ERR_ARG, "owned_field: not with LCS_KERNEL_FP64 or ckpt_every");
      break;
    }
    switch (d.field_dtype) {
      case LCS_F64:
        e.kind = d.field_kernel == LCS_KERNEL_FP64 ? FK_F64 : FK_DF;
        break;
      case LCS_F32: e.kind = FK_F32; break;
      case LCS_BF16: e.kind = FK_BF16; break;
      default: r = fail(c, LCS_ERR_ARG, "unknown field dtype");
    }
    if (r != LCS_OK) break;
    e.np = d.np;
    e.cap = d.np + d.np / 16 + (int64_t)SLACK_MIN * P + 1024;
    Geom &g = e.a.geo;
    g.N = d.n;
    g.L = d.box;
    g.inv_dx = (double)d.n / d.box;
    g.fix_dx = d.box / (double)d.n / 4503599627370496.0;  // L / N / 2^52
    g.qL = (int64_t)d.n << 52;
    g.Ptot = P;
    for (int s = 0; s < 3; ++s) {
      g.P[s] = d.sub[s];
      g.W[s] = d.n / d.sub[s];
      g.Wrcp[s] = g.W[s] > 1 ? (unsigned)(((uint64_t(1) << 32) + g.W[s] - 1) / g.W[s]) : 0u;
    }
    e.brick = d.sort_brick ? d.sort_brick : 8;
    int64_t space = (int64_t)e.brick * e.brick * e.brick;
    for (int s = 0; s < 3; ++s) {
      e.nb[s] = (g.W[s] + e.brick - 1) / e.brick;
      space *= e.nb[s];
    }
    if (space > (int64_t(1) << 32)) {
      r = fail(c, LCS_ERR_ARG, "cell key space exceeds 32 bits");
      break;
    }
    e.key_bits = ceil_log2(space);
    e.mig_bits = std::max(1, ceil_log2(2 * (int64_t)P));
    e.max_tiles = (int)(e.np / 32 + P + 2);  // 32 = smallest step tile of any config
    e.a.step_tile = 256;  // the configuration's tile, set by setup_batch (retile)
    e.max_stiles = (int)(e.np / SORT_TILE + P + 2);
    e.a.dt = d.dt;
    e.a.half_dt = 0.5 * d.dt;
    e.a.drag = d.drag == LCS_DRAG_NONLINEAR ? 1 : 0;
    e.a.drag_c = e.a.drag ? 18.0 / (d.nu * (d.density_ratio > 0 ? d.density_ratio : 843.0)) : 0.0;
    e.a.tau_const = d.tau ? 0.0 : d.tau_const;
    for (int s = 0; s < 3; ++s) e.a.g[s] = d.g[s];
    {
      // exact float-pair splits of the DF step's constants
      auto split = [](double v, float *o) {
        o[0] = (float)v;
        o[1] = (float)(v - (double)o[0]);
      };
      split(d.dt, e.a.dfk + 0);
      split(0.5 * d.dt, e.a.dfk + 2);
      split(d.dt * g.inv_dx, e.a.dfk + 4);
      for (int s = 0; s < 3; ++s) split(d.dt * d.g[s], e.a.dfk + 6 + 2 * s);
    }
    const bool has_tau = d.tau != nullptr, has_img = d.track_images != 0;
    const bool has_vs = d.migrate_per_stage != 0;
    for (int b = 0; b < 2 && r == LCS_OK; ++b)
      r = alloc_rec(c, e.a.buf[b], e.cap, has_tau, has_img, has_vs);
    if (r == LCS_OK) r = alloc_rec(c, e.a.pack, e.cap, has_tau, has_img, has_vs);
    if (r != LCS_OK) break;
    Meta &m = e.a.m;
    auto A = [&](cudaError_t err) {
      if (err != cudaSuccess && r == LCS_OK)
        r = fail(c, err == cudaErrorMemoryAllocation ? LCS_ERR_OOM : LCS_ERR_CUDA,
                 std::string("allocation: ") + cudaGetErrorString(err));
    };
    A(dalloc(c, &e.a.pack_bin, e.cap));
    for (int b = 0; b < 2; ++b) {
      A(dalloc(c, &m.lay_base[b], P));
      A(dalloc(c, &m.lay_cap[b], P));
    }
    A(dalloc(c, &m.next_base, P));
    A(dalloc(c, &m.next_cap, P));
    A(dalloc(c, &m.cnt, P));
    A(dalloc(c, &m.cstart, P + 1));
    A(dalloc(c, &m.tile_off, P + 1));
    A(dalloc(c, &m.stile_off, P + 1));
    A(dalloc(c, &m.phase, 1));
    A(dalloc(c, &m.status, 1));
    A(dalloc(c, &m.tile_counter, 1));
    A(dalloc(c, &m.staged, 1));
    A(dalloc(c, &m.fin_tab, (int64_t)P * (NBIN - 1)));
    A(dalloc(c, &m.bincnt, (int64_t)P * NBIN));
    A(dalloc(c, &m.tail_done, 1));
    A(dalloc(c, &m.stay_tot, P));
    A(dalloc(c, &m.mig_tot, P));
    for (int b = 0; b < 2; ++b) {
      A(dalloc(c, &e.s.key[b], std::max<int64_t>(e.np, 1)));
      A(dalloc(c, &e.s.pay[b], std::max<int64_t>(e.np, 1)));
    }
    A(dalloc(c, &e.s.hist, (int64_t)e.max_stiles * SORT_MAX_D));
    A(dalloc(c, &e.s.hist_scan, (int64_t)e.max_stiles * SORT_MAX_D));
    A(dalloc(c, &e.s.scan_blocks, (int64_t)e.max_stiles * SORT_MAX_D / 4096 + 2));
    A(dalloc(c, &e.cs1, 2));
    A(dalloc(c, &e.to1, 2));
    const int64_t ncell = (int64_t)d.n * d.n * d.n;
    const int64_t fbytes = e.kind == FK_BF16 ? 8 : e.kind == FK_F32 ? 16 : 32;
    A(dalloc(c, (char **)&e.field, ncell * fbytes));
    if (d.field_next) A(dalloc(c, (char **)&e.field_b, ncell * fbytes));
    if (d.owned_field) {
      const int64_t bcell = (int64_t)(g.W[0] + 4) * (g.W[1] + 4) * (g.W[2] + 4);
      A(dalloc(c, (char **)&e.bricks, (int64_t)P * bcell * fbytes));
      if (d.field_next) A(dalloc(c, (char **)&e.bricks_b, (int64_t)P * bcell * fbytes));
    }
    A(dalloc(c, &m.nstep, 1));
    if (r != LCS_OK) break;
    e.a.field = e.field;
    e.a.field_b = e.field_b;
    e.a.bricks = e.bricks;
    e.a.bricks_b = e.bricks_b;
    e.t_a = d.t_field[0];
    e.t_b = d.t_field[1];
    if (e.field_b) {
      e.a.th0 = (d.t_start - e.t_a) / (e.t_b - e.t_a);
      e.a.dth = d.dt / (e.t_b - e.t_a);
    }
    e.a.max_tiles = e.max_tiles;
    e.a.cap = e.cap;
    e.s.nseg = P;
    e.s.cstart = m.cstart;
    e.s.tile_off = m.stile_off;
    e.s.max_tiles = e.max_stiles;
    e.s.status = m.status;
    cudaStream_t st = c->st;
    auto C2 = [&](cudaError_t err) {
      if (err != cudaSuccess && r == LCS_OK)
        r = fail(c, LCS_ERR_CUDA, std::string("init: ") + cudaGetErrorString(err));
    };
    C2(cudaMemsetAsync(m.status, 0, sizeof(int), st));
    C2(cudaMemsetAsync(m.tile_counter, 0, sizeof(unsigned), st));
    C2(cudaMemsetAsync(m.staged, 0, sizeof(unsigned long long), st));
    {
      const std::vector<int> tab = finish_table(e.a.geo.P);
      C2(cudaMemcpy(m.fin_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice));
    }
    C2(cudaMemsetAsync(m.bincnt, 0, sizeof(int) * P * NBIN, st));
    C2(cudaMemsetAsync(m.tail_done, 0, sizeof(unsigned), st));
    C2(cudaMemsetAsync(m.stay_tot, 0, sizeof(int64_t) * P, st));
    C2(cudaMemsetAsync(m.mig_tot, 0, sizeof(int64_t) * P, st));
    C2(launch_field_convert(d.field, d.n, e.kind, e.field, st));
    if (e.field_b) C2(launch_field_convert(d.field_next, d.n, e.kind, e.field_b, st));
    if (e.bricks) C2(launch_build_bricks(e.field, e.a.geo, e.kind, e.bricks, st));
    if (e.bricks_b) C2(launch_build_bricks(e.field_b, e.a.geo, e.kind, e.bricks_b, st));
    C2(cudaMemsetAsync(m.nstep, 0, sizeof(int64_t), st));
    // particles -> buffer 1 compacted as one input segment, then migrate
    Rec &B1 = e.a.buf[1];
    for (int s = 0; s < 3 && e.np > 0; ++s) {
      C2(cudaMemcpyAsync(B1.x[s], d.x0 + s * e.np, e.np * 8, cudaMemcpyDefault, st));
      C2(cudaMemcpyAsync(B1.v[s], d.v0 + s * e.np, e.np * 8, cudaMemcpyDefault, st));
      if (B1.img[s]) C2(cudaMemsetAsync(B1.img[s], 0, e.np * 4, st));
    }
    if (B1.tau && e.np > 0) C2(cudaMemcpyAsync(B1.tau, d.tau, e.np * 8, cudaMemcpyDefault, st));
    if (e.np > 0)  // FP64 positions and velocities -> fixed point and float pairs
      k_import<<<grid_for(e.np, 256, c->sms * 8), 256, 0, st>>>(B1, e.np, e.a.geo, m.status);
    std::vector<int64_t> seg(P + 1, e.np);
    seg[0] = 0;
    int64_t *seg_dev = nullptr;
    C2(cudaMallocAsync((void **)&seg_dev, sizeof(int64_t) * (P + 1), st));
    C2(cudaMemcpyAsync(seg_dev, seg.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, st));
    k_input_meta<<<1, 1024, 0, st>>>(e.a, seg_dev);
    e.id_bits = d.ids ? 32 : std::max(1, ceil_log2(e.np));
    if (d.ids && e.np > 0) {
      C2(cudaMemcpyAsync(B1.id, d.ids, e.np * 4, cudaMemcpyDefault, st));
    } else {
      k_iota<<<grid_for(e.np, 256, c->sms * 8), 256, 0, st>>>(B1.id, m.cstart, P);
    }
    C2(cudaFreeAsync(seg_dev, st));
    C2(cudaGetLastError());
    if (r == LCS_OK) r = enqueue_migrate(c, e);
    if (r == LCS_OK && d.ckpt_every > 0) {
      r = tape_store(c, e, 0);
      e.tape_ok = true;
    }
    if (r == LCS_OK) {
      // tau >= dt and finite tau are checked on the host copy
      if (d.tau && e.np > 0) {
        std::vector<double> t(e.np);
        C2(cudaMemcpy(t.data(), d.tau, e.np * 8, cudaMemcpyDefault));
        for (int64_t i = 0; i < e.np && r == LCS_OK; ++i)
          if (!(t[i] >= d.dt) || !std::isfinite(t[i]))
            r = fail(c, LCS_ERR_ARG, "tau_p must be finite and >= dt");
      }
    }
  }
  if (r == LCS_OK) r = read_status(c);
  if (r == LCS_OK) r = setup_batch(c);
  if (r != LCS_OK) {
    const lcs_status rr = r;
    lcs_destroy(c);
    return rr;
  }
  *out = c;
  return LCS_OK;
}

lcs_status lcs_step(lcs_ctx *c, int64_t nsteps) {
  NvtxRange nvtx_range("lcs_step");
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (nsteps < 0) return reject(c, "nsteps < 0");
  int64_t done = 0;
  while (done < nsteps) {
    // all ensembles of a context share the step count
    const int64_t S = c->ens[0].steps;
    int64_t len = 1;
    std::vector<int> pend(c->ens.size());
    for (size_t k = 0; k < c->ens.size(); ++k) pend[k] = c->ens[k].perm;
    lcs_ctx::RunKey key;
    if (c->period > 0) {
      // a run of steps up to the next multiple of the period, the next
      // checkpoint step of any ensemble, or the end of the call
      const int64_t Q = c->period, phase = S % Q;
      len = std::min(nsteps - done, Q - phase);
      for (auto &e : c->ens)
        if (e.d.ckpt_every > 0)
          len = std::min<int64_t>(len, e.d.ckpt_every - S % e.d.ckpt_every);
      key = lcs_ctx::RunKey(phase, len, pend, std::vector<bool>());
    } else {
      key = lcs_ctx::RunKey(-1, 1, pend, sort_set(c, S + 1));
    }
    auto it = c->chunk_graphs.find(key);
    if (it == c->chunk_graphs.end()) {
      lcs_ctx::RunGraph rg;
      r = capture(c, S + 1, len, &rg.exec, &rg.launches);
      for (size_t k = 0; k < c->ens.size(); ++k) rg.perm_out.push_back(c->ens[k].perm);
      for (size_t k = 0; k < c->ens.size(); ++k) c->ens[k].perm = pend[k];  // not run yet
      if (r != LCS_OK) return r;
      it = c->chunk_graphs.emplace(key, rg).first;
    }
    CK(cudaGraphLaunch(it->second.exec, c->st));
    c->graph_launches += 1;
    c->launches += it->second.launches;
    for (size_t k = 0; k < c->ens.size(); ++k) c->ens[k].perm = it->second.perm_out[k];
    done += len;
    for (auto &e : c->ens) {
      e.steps += len;
      if (e.d.ckpt_every > 0 && e.steps % e.d.ckpt_every == 0) {
        r = materialize(c);  // a checkpoint holds the sorted records
        if (r == LCS_OK) r = tape_store(c, e, e.steps / e.d.ckpt_every);
        if (r != LCS_OK) return r;
      }
    }
  }
  return LCS_OK;
}

lcs_status lcs_migrate(lcs_ctx *c) {
  NvtxRange nvtx_range("lcs_migrate");
  lcs_status r = check_ctx(c);
  if (r == LCS_OK) r = materialize(c);  // the migration sort reuses the sort buffers
  if (r != LCS_OK) return r;
  for (auto &e : c->ens) {
    r = enqueue_migrate(c, e);
    if (r != LCS_OK) return r;
  }
  return LCS_OK;
}

lcs_status lcs_sort(lcs_ctx *c) {
  NvtxRange nvtx_range("lcs_sort");
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  for (auto &e : c->ens) {
    // a stable sort of the unsorted records gives the order a pending
    // permutation stands for: that permutation is simply recomputed
    e.perm = -1;
    r = enqueue_sort(c, e, c->st);
    if (r != LCS_OK) return r;
  }
  return LCS_OK;
}

lcs_status lcs_set_state(lcs_ctx *c, int ens, const double *x, const double *v,
                         const double *tau, const uint32_t *ids, const int32_t *img,
                         const int64_t *seg) {
  NvtxRange nvtx_range("lcs_set_state");
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (ens < 0 || ens >= (int)c->ens.size() || !x || !v || !ids || !seg)
    return reject(c, "lcs_set_state: bad argument");
  Ens &e = c->ens[ens];
  const int P = e.a.geo.Ptot;
  if (seg[0] != 0 || seg[P] != e.np) return reject(c, "lcs_set_state: bad segments");
  for (int s = 0; s < P; ++s)
    if (seg[s + 1] < seg[s]) return reject(c, "lcs_set_state: bad segments");
  if (e.a.buf[1].tau && e.np > 0 && !tau)
    return reject(c, "lcs_set_state: tau required (per-particle tau_p)");
  e.tape_ok = false;  // the recorded trajectory no longer leads to this state
  e.perm = -1;        // and a pending sort of the old records is void
  cudaStream_t st = c->st;
  // Place into buffer 1 with the given segments as windows; a relayout copy
  // moves it to the other buffer with a fresh layout.
  Rec &B1 = e.a.buf[1];
  for (int s = 0; s < 3 && e.np > 0; ++s) {
    CK(cudaMemcpyAsync(B1.x[s], x + s * e.np, e.np * 8, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(B1.v[s], v + s * e.np, e.np * 8, cudaMemcpyDefault, st));
    if (B1.img[s]) {
      if (img) CK(cudaMemcpyAsync(B1.img[s], img + s * e.np, e.np * 4, cudaMemcpyDefault, st));
      else CK(cudaMemsetAsync(B1.img[s], 0, e.np * 4, st));
    }
  }
  if (B1.tau && e.np > 0) {
    CK(cudaMemcpyAsync(B1.tau, tau, e.np * 8, cudaMemcpyDefault, st));
  }
  if (e.np > 0) CK(cudaMemcpyAsync(B1.id, ids, e.np * 4, cudaMemcpyDefault, st));
  if (e.np > 0) {
    k_import<<<grid_for(e.np, 256, c->sms * 8), 256, 0, st>>>(B1, e.np, e.a.geo, e.a.m.status);
    c->launches += 1;
  }
  int64_t *seg_dev = nullptr;
  CK(cudaMallocAsync((void **)&seg_dev, sizeof(int64_t) * (P + 1), st));
  CK(cudaMemcpyAsync(seg_dev, seg, sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, st));
  k_input_meta<<<1, 1024, 0, st>>>(e.a, seg_dev);
  k_relayout<<<1, 1024, 0, st>>>(e.a, 0);
  const int gs = grid_for(e.np, 256, c->sms * 8);
  k_iota<<<gs, 256, 0, st>>>(e.s.pay[0], e.a.m.cstart, P);
  k_gather<<<gs, 256, 0, st>>>(e.a, e.s.pay[0]);
  k_set_phase<<<1, 1024, 0, st>>>(e.a);
  c->launches += 5;
  CK(cudaFreeAsync(seg_dev, st));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return read_status(c);
}

lcs_status lcs_get_state(lcs_ctx *c, int ens, double *x, double *v, double *tau,
                         uint32_t *ids, int32_t *img, int64_t *seg) {
  NvtxRange nvtx_range("lcs_get_state");
  if (!c) return LCS_ERR_ARG;
  if (c->failed) return LCS_ERR_STATE;
  if (ens < 0 || ens >= (int)c->ens.size()) return reject(c, "bad ensemble");
  Ens &e = c->ens[ens];
  cudaStream_t st = c->st;
  const int P = e.a.geo.Ptot;
  Rec tmp = e.a.pack;
  // the records in their sorted order: a pending sort permutation is read
  // through (and stays pending for the next step)
  StepArgs ea = e.a;
  ea.perm = e.perm >= 0 ? e.s.pay[e.perm] : nullptr;
  k_compact<<<grid_for(e.np, 256, c->sms * 8), 256, 0, st>>>(ea, tmp);
  k_export<<<grid_for(e.np, 256, c->sms * 8), 256, 0, st>>>(tmp, e.np, e.a.geo);
  c->launches += 2;
  CK(cudaGetLastError());
  for (int s = 0; s < 3 && e.np > 0; ++s) {
    if (x) CK(cudaMemcpyAsync(x + s * e.np, tmp.x[s], e.np * 8, cudaMemcpyDefault, st));
    if (v) CK(cudaMemcpyAsync(v + s * e.np, tmp.v[s], e.np * 8, cudaMemcpyDefault, st));
    if (img && tmp.img[s])
      CK(cudaMemcpyAsync(img + s * e.np, tmp.img[s], e.np * 4, cudaMemcpyDefault, st));
  }
  if (tau && e.np > 0) {
    if (tmp.tau) {
      CK(cudaMemcpyAsync(tau, tmp.tau, e.np * 8, cudaMemcpyDefault, st));
    } else {
      std::vector<double> t(e.np, e.d.tau_const);
      CK(cudaMemcpyAsync(tau, t.data(), e.np * 8, cudaMemcpyDefault, st));
      CK(cudaStreamSynchronize(st));
    }
  }
  if (img && !tmp.img[0] && e.np > 0) {
    // images not tracked: zeros, written on the side of the pointer
    cudaPointerAttributes pa{};
    CK(cudaPointerGetAttributes(&pa, img));
    if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) {
      CK(cudaMemsetAsync(img, 0, 3 * e.np * 4, st));
    } else {
      CK(cudaStreamSynchronize(st));
      std::memset(img, 0, 3 * e.np * 4);
    }
  }
  if (ids && e.np > 0) CK(cudaMemcpyAsync(ids, tmp.id, e.np * 4, cudaMemcpyDefault, st));
  if (seg) CK(cudaMemcpyAsync(seg, e.a.m.cstart, sizeof(int64_t) * (P + 1), cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return read_status(c);
}

lcs_status lcs_get_state_by_id(lcs_ctx *c, int ens, double *x, double *v, uint32_t *ids) {
  NvtxRange nvtx_range("lcs_get_state_by_id");
  if (!c) return LCS_ERR_ARG;
  if (c->failed) return LCS_ERR_STATE;
  if (ens < 0 || ens >= (int)c->ens.size()) return reject(c, "bad ensemble");
  lcs_status mr = materialize(c);  // the id sort reuses the sort buffers
  if (mr != LCS_OK) return mr;
  Ens &e = c->ens[ens];
  cudaStream_t st = c->st;
  if (e.np > 0) {
    // the output buffer of the next step is free between steps: it stages
    // the id-ordered rows (the input buffer is the one the phase names)
    int ph = 0;
    CK(cudaMemcpyAsync(&ph, e.a.m.phase, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    Rec tmp = e.a.pack, out = e.a.buf[ph ^ 1];
    const int gs = grid_for(e.np, 256, c->sms * 8);
    k_compact<<<gs, 256, 0, st>>>(e.a, tmp);
    k_export<<<gs, 256, 0, st>>>(tmp, e.np, e.a.geo);
    k_id_keys<<<gs, 256, 0, st>>>(tmp, e.np, e.s.key[0], e.s.pay[0]);
    k_one_segment<<<1, 1, 0, st>>>(e.a.m.cstart, e.a.geo.Ptot, e.cs1, e.to1);
    SortArgs s = e.s;
    s.nseg = 1, s.cstart = e.cs1, s.tile_off = e.to1;
    int ob = 0;
    CK(radix_sort(s, e.id_bits, &ob, st, &c->launches));
    k_by_id<<<gs, 256, 0, st>>>(tmp, s.pay[ob], e.np, out, e.a.geo.L);
    c->launches += 5;
    CK(cudaGetLastError());
    for (int q = 0; q < 3; ++q) {
      if (x) CK(cudaMemcpyAsync(x + q * e.np, out.x[q], e.np * 8, cudaMemcpyDefault, st));
      if (v) CK(cudaMemcpyAsync(v + q * e.np, out.v[q], e.np * 8, cudaMemcpyDefault, st));
    }
    if (ids) CK(cudaMemcpyAsync(ids, out.id, e.np * 4, cudaMemcpyDefault, st));
  }
  CK(cudaStreamSynchronize(st));
  return read_status(c);
}

lcs_status lcs_get_field(lcs_ctx *c, int ens, double *out) {
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (ens < 0 || ens >= (int)c->ens.size() || !out) return reject(c, "bad argument");
  Ens &e = c->ens[ens];
  const int64_t ncell = (int64_t)e.d.n * e.d.n * e.d.n;
  double *tmp = nullptr;
  CK(cudaMallocAsync((void **)&tmp, ncell * 3 * sizeof(double), c->st));
  CK(launch_field_expand(e.field, e.d.n, e.kind, tmp, c->st));
  CK(cudaMemcpyAsync(out, tmp, ncell * 3 * sizeof(double), cudaMemcpyDefault, c->st));
  CK(cudaFreeAsync(tmp, c->st));
  c->launches += 1;
  CK(cudaStreamSynchronize(c->st));
  return LCS_OK;
}

lcs_status lcs_pair_histogram(lcs_ctx *c, int ens, double r_max, int nbins, int64_t *counts) {
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (ens < 0 || ens >= (int)c->ens.size() || !counts || nbins < 1 || nbins > 4096)
    return reject(c, "lcs_pair_histogram: bad argument");
  Ens &e = c->ens[ens];
  const Geom &g = e.a.geo;
  if (g.N < 3 || !(r_max > 0) || !(r_max <= g.L / g.N))
    return reject(c, "lcs_pair_histogram: needs N >= 3 and 0 < r_max <= L/N");
  r = materialize(c);  // the cell sort of the pairs reuses the sort buffers
  if (r != LCS_OK) return r;
  cudaStream_t st = c->st;
  const int64_t n = e.np;
  std::vector<unsigned long long> h(nbins, 0ull);
  if (n > 1) {
    const int64_t ncell = (int64_t)g.N * g.N * g.N;
    char *mem = nullptr;
    const size_t bytes = sizeof(int) * (ncell + 1) + sizeof(unsigned long long) * nbins + 64;
    CK(cudaMallocAsync((void **)&mem, bytes, st));
    int *start = (int *)mem;
    unsigned long long *dcount =
        (unsigned long long *)(mem + ((sizeof(int) * (ncell + 1) + 15) & ~size_t(15)));
    CK(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long) * nbins, st));
    const int gs = grid_for(n, 256, c->sms * 8);
    CK(launch_pair_keys(e.a, e.s.key[0], e.s.pay[0], n, gs, st));
    k_one_segment<<<1, 1, 0, st>>>(e.a.m.cstart, g.Ptot, e.cs1, e.to1);
    SortArgs s = e.s;
    s.nseg = 1, s.cstart = e.cs1, s.tile_off = e.to1;
    int ob = 0;
    CK(radix_sort(s, ceil_log2(ncell), &ob, st, &c->launches));
    CK(launch_pair_hist(e.a, s.key[ob], s.pay[ob], start, n, r_max, nbins, dcount, c->sms, st));
    c->launches += 4;
    CK(cudaMemcpyAsync(h.data(), dcount, sizeof(unsigned long long) * nbins,
                       cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(mem, st));
  }
  CK(cudaStreamSynchronize(st));
  for (int b = 0; b < nbins; ++b) counts[b] = (int64_t)h[b];
  return read_status(c);
}

lcs_status lcs_pair_rdf(lcs_ctx *c, int ens, double r_max, int nbins, double *r, double *g,
                        int64_t *counts) {
  lcs_status st = check_ctx(c);
  if (st != LCS_OK) return st;
  if (!g || nbins < 1 || nbins > 4096) return reject(c, "lcs_pair_rdf: bad argument");
  std::vector<int64_t> cnt(nbins);
  st = lcs_pair_histogram(c, ens, r_max, nbins, cnt.data());
  if (st != LCS_OK) return st;
  const double n = (double)c->ens[ens].np, L = c->ens[ens].d.box;
  const double pairs = n * (n - 1.0) / 2.0, pi = 3.14159265358979323846;
  for (int b = 0; b < nbins; ++b) {
    const double r0 = r_max * b / nbins, r1 = r_max * (b + 1) / nbins;
    const double expected = pairs * (4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0)) / (L * L * L);
    g[b] = expected > 0.0 ? (double)cnt[b] / expected : 0.0;
    if (r) r[b] = 0.5 * (r0 + r1);
    if (counts) counts[b] = cnt[b];
  }
  return LCS_OK;
}

lcs_status lcs_set_field(lcs_ctx *c, int ens, const double *field, double t) {
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (ens < 0 || ens >= (int)c->ens.size() || !field)
    return reject(c, "lcs_set_field: bad argument");
  Ens &e = c->ens[ens];
  if (!e.field_b) return reject(c, "lcs_set_field: ensemble was created with a frozen field");
  if (!(t > e.t_b) || !std::isfinite(t)) return reject(c, "lcs_set_field: t must exceed t_b");
  CK(cudaStreamSynchronize(c->st));
  std::swap(e.field, e.field_b);  // the newer snapshot becomes the first
  CK(launch_field_convert(field, e.d.n, e.kind, e.field_b, c->st));
  c->launches += 1;
  if (e.bricks_b) {  // owned field: the bricks follow their snapshots
    std::swap(e.bricks, e.bricks_b);
    CK(launch_build_bricks(e.field_b, e.a.geo, e.kind, e.bricks_b, c->st));
    c->launches += 1;
    e.a.bricks = e.bricks;
    e.a.bricks_b = e.bricks_b;
  }
  e.t_a = e.t_b;
  e.t_b = t;
  e.a.field = e.field;
  e.a.field_b = e.field_b;
  e.a.th0 = (e.d.t_start - e.t_a) / (e.t_b - e.t_a);
  e.a.dth = e.d.dt / (e.t_b - e.t_a);
  r = upload_args(c);
  if (r != LCS_OK) return r;
  drop_graphs(c);  // the graphs carry the snapshot pointers and times
  CK(cudaStreamSynchronize(c->st));
  return read_status(c);
}

lcs_status lcs_backward(lcs_ctx *c, const double *gx, const double *gv, double *gU,
                        double *gx0, double *gv0) {
  NvtxRange nvtx_range("lcs_backward");
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (c->ens.size() != 1) return reject(c, "lcs_backward: one ensemble only");
  Ens &e = c->ens[0];
  const int K = e.d.ckpt_every;
  if (K <= 0 || !e.d.track_images || !e.tape_ok)
    return reject(c, "lcs_backward: needs ckpt_every > 0, track_images = 1 and no "
                     "lcs_set_state since lcs_init");
  if (!gx || !gv || !gU || !gx0 || !gv0) return reject(c, "lcs_backward: null pointer");
  const int64_t np = e.np, T = e.steps;
  cudaStream_t st = c->st;
  if (!e.lam_id) {
    CK(dalloc(c, &e.lam_id, 6 * std::max<int64_t>(np, 1)));
    CK(dalloc(c, &e.lam_s, 6 * std::max<int64_t>(np, 1)));
    CK(dalloc(c, &e.states, (int64_t)K * 6 * std::max<int64_t>(np, 1)));
  }
  if (np > 0) {
    CK(cudaMemcpyAsync(e.lam_id, gx, 3 * np * 8, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(e.lam_id + 3 * np, gv, 3 * np * 8, cudaMemcpyDefault, st));
    for (int64_t k = (T - 1) / K; T > 0 && k >= 0; --k) {
      const int64_t s0 = k * K;
      const int len = (int)std::min<int64_t>(K, T - s0);
      const TapeSlot &t = e.tape[k];
      CK(launch_recompute(e.a, e.kind, t, e.states, len, np, st));
      CK(launch_lam_permute(t.id, e.lam_id, e.lam_s, np, 1, e.a.m.status, st));
      for (int j = len - 1; j >= 0; --j)
        CK(launch_adjoint(e.a, e.kind, e.states + (int64_t)j * 6 * np, t.tau, e.lam_s, gU, np,
                          st));
      CK(launch_lam_permute(t.id, e.lam_s, e.lam_id, np, 0, e.a.m.status, st));
      c->launches += 3 + len;
    }
    CK(cudaMemcpyAsync(gx0, e.lam_id, 3 * np * 8, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(gv0, e.lam_id + 3 * np, 3 * np * 8, cudaMemcpyDefault, st));
  }
  CK(cudaStreamSynchronize(st));
  return read_status(c);
}

}  // extern "C"

namespace {
// lcs_profile_steps with, when group_ms is given, the step-kernel time of
// every launch group accumulated per group.
lcs_status profile_steps(lcs_ctx *c, int64_t nsteps, double *ms, int64_t *count,
                         std::vector<double> *group_ms) {
  for (int k = 0; k < LCS_PROF_N; ++k) {
    ms[k] = 0.0;
    if (count) count[k] = 0;
  }
  if (group_ms) group_ms->assign(c->groups.size(), 0.0);
  lcs_status r = LCS_OK;
  for (int64_t k = 0; k < nsteps; ++k) {
    const std::vector<bool> sorts = sort_set(c, c->ens[0].steps + 1);
    {
      Prof pf;
      r = enqueue_step_profiled(c, sorts, pf);
      if (r == LCS_OK) {
        CK(cudaStreamSynchronize(c->st));
        for (size_t i = 0; i + 1 < pf.ev.size(); ++i) {
          float t = 0.f;
          cudaEventElapsedTime(&t, pf.ev[i], pf.ev[i + 1]);
          int cls = pf.cls[i];
          if (cls >= 1000) {  // one step-kernel launch group
            if (group_ms && cls - 1000 < (int)group_ms->size()) (*group_ms)[cls - 1000] += t;
            cls = LCS_PROF_STEP;
          }
          if (cls >= 0 && cls < LCS_PROF_N) {
            ms[cls] += t;
            if (count) count[cls] += 1;
          }
        }
      }
      for (auto ev : pf.ev) cudaEventDestroy(ev);
      if (r != LCS_OK) return r;
    }
    for (auto &e : c->ens) {
      ++e.steps;
      if (e.d.ckpt_every > 0 && e.steps % e.d.ckpt_every == 0) {
        r = tape_store(c, e, e.steps / e.d.ckpt_every);
        if (r != LCS_OK) return r;
      }
    }
  }
  return read_status(c);
}
}  // namespace

extern "C" {

lcs_status lcs_profile_steps(lcs_ctx *c, int64_t nsteps, double *ms, int64_t *count) {
  NvtxRange nvtx_range("lcs_profile_steps");
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (nsteps < 0 || !ms) return reject(c, "lcs_profile_steps: bad argument");
  return profile_steps(c, nsteps, ms, count, nullptr);
}

// Step-kernel configurations: (threads per block, particles per thread, kernel mode)
// Whether a context may use a step-kernel configuration: no staged-field
// form of the all-FP64 kernel; an evolving field or migration per stage only
// with the deferred scatter (256 threads for migration per stage); an
// owned-field context only with mode LCS_STEP_OWNED_FIELD, which no other
// context uses.
static bool step_config_allowed(const lcs_ctx *c, int block, int mode) {
  if (mode == LCS_STEP_STAGED_FIELD && c->kind == FK_F64) return false;
  const int deferred = c->owned ? LCS_STEP_OWNED_FIELD : LCS_STEP_DEFERRED;
  if (c->owned != (mode == LCS_STEP_OWNED_FIELD)) return false;
  if (c->evolve && mode != deferred) return false;
  if (c->per_stage && (mode != deferred || block != 256)) return false;
  return true;
}

static const int kStepConfigs[LCS_TUNE_CONFIGS][3] = {
    {256, 2, 0}, {256, 1, 0}, {128, 2, 0}, {256, 2, 1}, {128, 2, 1}, {256, 2, 2},
    {128, 2, 2}, {256, 1, 2}, {256, 2, 3}, {128, 2, 3}, {256, 1, 3}, {128, 1, 3},
    {256, 1, 4}, {256, 2, 4}};

lcs_status lcs_set_step_config(lcs_ctx *c, int block, int items, int mode) {
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  bool known = false;
  for (const auto &k : kStepConfigs) known |= k[0] == block && k[1] == items && k[2] == mode;
  if (!known || !step_config_allowed(c, block, mode))
    return reject(c, "lcs_set_step_config: configuration not available");
  CK(cudaStreamSynchronize(c->st));
  for (auto &k : c->cfg) k = StepCfg{block, items, mode};
  regroup(c, nullptr);
  r = retile(c);
  if (r != LCS_OK) return r;
  drop_graphs(c);
  return read_status(c);
}

lcs_status lcs_step_config_of(lcs_ctx *c, int ens, int *block, int *items, int *mode) {
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (ens < 0 || ens >= (int)c->ens.size()) return reject(c, "lcs_step_config_of: bad ensemble");
  if (block) *block = c->cfg[ens].block;
  if (items) *items = c->cfg[ens].items;
  if (mode) *mode = c->cfg[ens].mode;
  return LCS_OK;
}

lcs_status lcs_staged_tiles(lcs_ctx *c, int64_t *count) {
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (!count) return reject(c, "lcs_staged_tiles: count is NULL");
  CK(cudaStreamSynchronize(c->st));
  int64_t tot = 0;
  for (auto &e : c->ens) {
    unsigned long long v = 0;
    CK(cudaMemcpy(&v, e.a.m.staged, sizeof(v), cudaMemcpyDeviceToHost));
    tot += (int64_t)v;
  }
  *count = tot;
  return read_status(c);
}

lcs_status lcs_tune(lcs_ctx *c, int steps_per_trial, int *block, int *items, int *mode,
                    double *trial_ms) {
  NvtxRange nvtx_range("lcs_tune");
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  if (steps_per_trial < 1) return reject(c, "lcs_tune: steps_per_trial < 1");
  // ensemble classes: grid size and decade of the particle count
  const int n = (int)c->ens.size();
  std::vector<int> cls(n);
  {
    std::map<std::pair<int, int>, int> ids;
    for (int k = 0; k < n; ++k) {
      int dec = 0;
      for (int64_t v = c->ens[k].np; v >= 10; v /= 10) ++dec;
      const auto key = std::make_pair(c->ens[k].d.n, dec);
      auto it = ids.find(key);
      if (it == ids.end()) it = ids.emplace(key, (int)ids.size()).first;
      cls[k] = it->second;
    }
  }
  int ncls = 0;
  for (int v : cls) ncls = std::max(ncls, v + 1);
  std::vector<double> best(ncls, 1e300);
  std::vector<int> pick(ncls, -1);
  const auto &cfg = kStepConfigs;
  for (int k = 0; k < LCS_TUNE_CONFIGS; ++k) {
    if (trial_ms) trial_ms[k] = -1.0;
    if (!step_config_allowed(c, cfg[k][0], cfg[k][2])) continue;
    // every class in launches of its own, so that each is timed alone
    for (auto &q : c->cfg) q = StepCfg{cfg[k][0], cfg[k][1], cfg[k][2]};
    regroup(c, &cls);
    r = retile(c);
    if (r != LCS_OK) return r;
    double ms[LCS_PROF_N];
    std::vector<double> gms;
    r = profile_steps(c, steps_per_trial, ms, nullptr, &gms);
    if (r != LCS_OK) return r;
    if (trial_ms) trial_ms[k] = ms[LCS_PROF_STEP];
    std::vector<double> per(ncls, 0.0);
    for (size_t g = 0; g < c->groups.size(); ++g) per[cls[c->groups[g].ens[0]]] += gms[g];
    for (int q = 0; q < ncls; ++q)
      if (per[q] < best[q]) best[q] = per[q], pick[q] = k;
  }
  for (int k = 0; k < n; ++k) {
    const int b = pick[cls[k]] >= 0 ? pick[cls[k]] : 0;
    c->cfg[k] = StepCfg{cfg[b][0], cfg[b][1], cfg[b][2]};
  }
  regroup(c, nullptr);  // ensembles that share a configuration share launches again
  r = retile(c);
  if (r != LCS_OK) return r;
  drop_graphs(c);  // graphs recorded with the old configuration are rebuilt
  if (block) *block = c->cfg[0].block;
  if (items) *items = c->cfg[0].items;
  if (mode) *mode = c->cfg[0].mode;
  return LCS_OK;
}

lcs_status lcs_sync(lcs_ctx *c) {
  lcs_status r = check_ctx(c);
  if (r != LCS_OK) return r;
  CK(cudaStreamSynchronize(c->st));
  return read_status(c);
}

const char *lcs_last_error(lcs_ctx *c) {
  if (!c) return g_last_init_error.c_str();
  return c->err.c_str();
}

void lcs_destroy(lcs_ctx *c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  drop_graphs(c);
  for (void *p : c->allocs) cudaFree(p);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  delete c;
}

int64_t lcs_launch_count(lcs_ctx *c) { return c ? c->launches : 0; }

int64_t lcs_graph_launch_count(lcs_ctx *c) { return c ? c->graph_launches : 0; }

lcs_status lcs_partition(const uint32_t *keys, int64_t n, int nbins, uint32_t *perm,
                         int64_t *bin_off, int32_t *status, void *stream) {
  if (n < 0 || n >= (int64_t(1) << 31) || nbins < 1 || nbins > 65536 ||
      (n > 0 && (!keys || !perm)) || !bin_off)
    return LCS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int max_tiles = (int)(n / SORT_TILE + 2);
  const int64_t nn = std::max<int64_t>(n, 1);
  char *mem = nullptr;
  // layout: key[2], pay[2] (n each), hist, hist_scan (tiles * 512), blocks, cs1, to1
  const int64_t hn = (int64_t)max_tiles * SORT_MAX_D;
  const int64_t nblk = hn / 4096 + 2;
  const size_t bytes = 4 * nn * 4 + 2 * hn * 4 + nblk * 4 + 2 * 8 + 2 * 4 + 64;
  if (cudaMallocAsync((void **)&mem, bytes, st) != cudaSuccess) return LCS_ERR_OOM;
  SortArgs s{};
  char *p = mem;
  auto take = [&](size_t b) { char *q = p; p += (b + 15) / 16 * 16; return q; };
  s.key[0] = (uint32_t *)take(nn * 4);
  s.key[1] = (uint32_t *)take(nn * 4);
  s.pay[0] = (uint32_t *)take(nn * 4);
  s.pay[1] = perm;
  s.hist = (int *)take(hn * 4);
  s.hist_scan = (int *)take(hn * 4);
  s.scan_blocks = (int *)take(nblk * 4);
  int64_t *cs1 = (int64_t *)take(16);
  int *to1 = (int *)take(8);
  s.nseg = 1, s.cstart = cs1, s.tile_off = to1, s.max_tiles = max_tiles;
  (void)take(0);
  const int gs = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, device_sms() * 8));
  k_partition_tables<<<1, 1, 0, st>>>(n, cs1, to1, status);
  if (n > 0) k_partition_in<<<gs, 256, 0, st>>>(keys, n, (uint32_t)nbins, s.key[0], s.pay[0], status);
  int ob = 0;
  cudaError_t err = radix_sort(s, ceil_log2(nbins), &ob, st, nullptr);
  if (err == cudaSuccess) {
    if (ob == 0 && n > 0)
      cudaMemcpyAsync(perm, s.pay[0], n * 4, cudaMemcpyDeviceToDevice, st);
    k_bin_bounds<<<gs, 256, 0, st>>>(s.key[ob], cs1, 0, nbins, bin_off);
    err = cudaGetLastError();
  }
  cudaFreeAsync(mem, st);
  return err == cudaSuccess ? LCS_OK : LCS_ERR_CUDA;
}

}  // extern "C"
