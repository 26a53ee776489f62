// C ABI of the library (declared in include/pma.h): handle lifetime, argument
// checks, the per-call launch sequence and status read-back.
//
// One call of pma_merge enqueues, on the caller's stream and without any host
// synchronisation:
//   hist / scan             Step 1: per-cell counts and first positions
//   radix prep / passes     Step 1 for ungrouped input: stable sort by cell
//   cluster_kernel          cells too large for shared memory: top cuts in
//                           global memory by a 4-CTA cluster per cell
//                           (partial sums through distributed shared
//                           memory) until every piece fits
//   team_kernel (3 launches) Steps 2-6 in shared memory: cells of up to
//                           1024 particles (4-warp teams), larger cells and
//                           the pieces of big cells (8-warp teams)
//   count / tiles / emit    Step 7: centroids, compacted, canonical order
// and a 1-line status copy (count, error bits, counters) to pinned memory.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lookback.cuh"
#include "pma.h"
#include "pma_launch.h"

using namespace pma;

namespace {

struct Ctl {
  unsigned err;
  int32_t unsorted;
  int32_t big_count;
  int32_t big_next;
  int32_t piece_count;
  int32_t unit_next[2];
  int32_t warp_count;
  int32_t warp_next;
  int32_t tiny_count;
  int32_t tiny_next;
  int32_t block_count;
  int32_t bin_ticket;
  int32_t emit_ticket;
  int32_t radix_ticket[kRadixMaxPasses];
  int32_t pad;
  int64_t count;
  unsigned long long stats[kStCount];
  double energy[2];  // kinetic energy in and out (PMA_FLAG_ENERGY_STATS)
  unsigned long long check;  // first failed bounds check (checked build), site << 48 | index
};

constexpr int kRing = 64;  // timed calls kept for pma_get_timing

struct Staging {
  int32_t *cells = nullptr;
  void *q[kMaxD] = {};
  void *w = nullptr;
  int32_t *out_cell = nullptr;
  void *out_pos[3] = {};
  double *out_mom[3] = {};
  double *out_w = nullptr;
  int32_t *out_index = nullptr;
  bool ready = false;
};

}  // namespace

struct pma_handle {
  pma_config cfg;
  int device = 0;
  int sms = 0;
  int smem_optin = 0;
  int D = 0;
  int mixed = 0;
  int cap = 0;
  int unit_grid = 0;
  int unit_team = 8;               // warps of the large-cell and piece teams
  int cap_w = 0;
  int cap_t = 0;
  int class_base = kClassBaseMin;  // size classes of pending subsets
  int widen_groups = 0;            // more lanes per set in sparse rounds
  int tiny_grid = 0;
  int warp_grid = 0;
  int64_t capacity = 0;
  int bin_tiles = 0;
  int emit_tiles_max = 0;
  int max_pieces = 0;
  // workspace
  int32_t *counts = nullptr, *cell_begin = nullptr, *radix_count = nullptr;
  unsigned long long *radix_status = nullptr;
  int32_t *perm = nullptr, *perm_tmp = nullptr, *perm_final = nullptr, *big_list = nullptr;
  int32_t *warp_list = nullptr, *block_list = nullptr, *tiny_list = nullptr;
  void *fin = nullptr;  // staging: D + 1 columns of fin_stride entries
  int64_t fin_stride = 0;  // capacity rounded up to 16 entries (bulk-copy alignment)
  uint8_t *head = nullptr;
  uint32_t *cell_flags = nullptr;  // near-tie bits per cell when the caller gives none
  unsigned long long *bin_status = nullptr;
  int32_t *tile_count = nullptr;
  long long *tile_prefix = nullptr;
  double *energy_tiles = nullptr;  // [2][emit tiles] partial energy sums
  int4 *pieces = nullptr;
  Ctl *ctl = nullptr;
  Ctl *ctl_host = nullptr;
  cudaStream_t last_stream = nullptr;
  bool pending = false;
  Staging stage;
  bool timing = false;
  int timed = 0;     // calls recorded since timing was enabled
  int nvtx_depth = 0;  // NVTX ranges of the current call still open
  unsigned long long wait_ns = 0;  // limit of the bounded device waits (0: default)
  int withhold_tile = -1;          // failure-detection test hook (see pma.h)
  cudaEvent_t ev[kRing][PMA_N_STAGES] = {};  // PMA_N_STAGES events per call
  cudaEvent_t *cur_ev = nullptr;
  std::string last_error;
  pma_stats stats{};
  // the counts of the handle's last call that completed without error: a
  // work source that was empty then gets a small grid now (see enqueue)
  bool have_prev = false;
  unsigned long long check_first = 0;  // the last synced call's first failed bounds check
  pma_stats prev{};
};

namespace {

int fail(pma_handle *h, int code, const std::string &msg) {
  if (h) h->last_error = msg;
  return code;
}

int cuda_fail(pma_handle *h, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, PMA_ERR_CUDA, m);
}

#define PMA_CUDA(h, call)                                     \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);  \
  } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void free_all(pma_handle *h) {
  void *ptrs[] = {h->counts, h->cell_begin, h->radix_count, h->radix_status, h->perm, h->perm_tmp, h->perm_final,
                  h->big_list, h->head, h->bin_status, h->tile_count, h->tile_prefix,
                  h->energy_tiles,
                  h->pieces, h->ctl, h->warp_list, h->block_list, h->tiny_list, h->fin, h->cell_flags,
                  h->stage.cells, h->stage.w, h->stage.out_cell,
                  h->stage.out_w, h->stage.out_index};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int l = 0; l < kMaxD; ++l)
    if (h->stage.q[l]) cudaFree(h->stage.q[l]);
  for (int l = 0; l < 3; ++l) {
    if (h->stage.out_pos[l]) cudaFree(h->stage.out_pos[l]);
    if (h->stage.out_mom[l]) cudaFree(h->stage.out_mom[l]);
  }
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  for (auto &row : h->ev)
    for (auto &e : row)
      if (e) cudaEventDestroy(e);
}

// NVTX ranges of a call and of its stages, for profilers that show host
// ranges beside the kernels (no-ops unless a profiler is attached)
const char *const kStageRange[PMA_N_STAGES - 1] = {
    "pma Step 1 binning", "pma big-cell cuts", "pma small-cell teams",
    "pma large-cell teams", "pma big-cell pieces", "pma Step 7 emit"};

// event i of the current call: 0 before binning, 1..6 after each stage
// (stage k spans events k..k+1, the whole call 0..6); the NVTX range of the
// call opens at 0 and closes at 6, one stage range at a time in between
void mark(pma_handle *h, int i, cudaStream_t st) {
  if (h->timing && h->cur_ev) cudaEventRecord(h->cur_ev[i], st);
  if (i == 0) {
    // ranges that an earlier call left open when it returned an error
    for (; h->nvtx_depth > 0; --h->nvtx_depth) nvtxRangePop();
    nvtxRangePushA("pma_merge");
    nvtxRangePushA(kStageRange[0]);
    h->nvtx_depth = 2;
  } else if (h->nvtx_depth == 2) {
    nvtxRangePop();
    if (i < PMA_N_STAGES - 1) {
      nvtxRangePushA(kStageRange[i]);
    } else {
      nvtxRangePop();
      h->nvtx_depth = 0;
    }
  }
}

// status code of a device error word: bad particle data first, then a wait
// that gave up, then an internal bound
int status_of_bits(unsigned err) {
  if (err & kErrInput) return PMA_ERR_INPUT;
  if (err & kErrTimeout) return PMA_ERR_TIMEOUT;
  if (err & kErrInternal) return PMA_ERR_INTERNAL;
  return PMA_OK;
}

int status_from_ctl(pma_handle *h) {
  const Ctl &c = *h->ctl_host;
  pma_stats &s = h->stats;
  h->check_first = c.check;
  s.n_out = c.count;
  s.cells_merged = (int64_t)c.stats[kStCellsMerged];
  s.cells_passthrough = (int64_t)c.stats[kStCellsPass];
  s.splits = (int64_t)c.stats[kStSplits];
  s.leaves = (int64_t)c.stats[kStLeaves];
  s.depth_sum = (int64_t)c.stats[kStDepth];
  s.degenerate_cuts = (int64_t)c.stats[kStDegenerate];
  s.big_cells = (int64_t)c.stats[kStBig];
  s.sorted_input = c.unsorted ? 0 : 1;
  s.near_stop = (int64_t)c.stats[kStNearStop];
  s.near_argmax = (int64_t)c.stats[kStNearArgmax];
  s.near_cut = (int64_t)c.stats[kStNearCut];
  s.fp64_rechecks = (int64_t)c.stats[kStRecheck];
  s.cells_flagged = (int64_t)c.stats[kStCellsFlagged];
  s.cells_tiny = c.tiny_count;
  s.cells_small = c.warp_count;
  s.cells_large = c.block_count;
  s.energy_in = c.energy[0];
  s.energy_out = c.energy[1];
  switch (status_of_bits(c.err)) {
    case PMA_ERR_INPUT:
      return fail(h, PMA_ERR_INPUT,
                  "invalid particle data (cell id out of range, w <= 0 or non-finite value)");
    case PMA_ERR_TIMEOUT: return fail(h, PMA_ERR_TIMEOUT, "a bounded device wait gave up");
    case PMA_ERR_INTERNAL:
      return fail(h, PMA_ERR_INTERNAL, "an internal device bound was exceeded");
    default: return PMA_OK;
  }
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

// The regions a call must clear, zeroed by one kernel on the call's stream
// instead of one memset per region.  Every region is a whole number of
// 4-byte words.
constexpr int kZeroRegions = 5;
struct ZeroArgs {
  uint32_t *p[kZeroRegions];
  int64_t words[kZeroRegions];
};

__global__ void zero_kernel(ZeroArgs z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kZeroRegions; ++r)
    for (int64_t i = t; i < z.words[r]; i += stride) z.p[r][i] = 0u;
}

// ------------------------------------------------------ population classes
//
// Cells of at most cap_t particles go to one-warp teams (a small tile, many
// cells in flight per SM, no warp waits for another), cells of at most
// cap_w to 4-warp teams (several CTAs per SM), cells of at most cap to
// 8-warp teams with a large tile; larger cells are cut in global memory
// first and their pieces join the 8-warp class.

struct Classes {
  int cap_t, cap_w, cap, base, widen;
};

// largest tile of at most `hi` particles whose team fits the CTA's shared memory
int largest_tile(const pma_handle *h, int hi, int lo) {
  int c = hi;
  while (c > lo && team_smem(h->mixed, h->D, c) > (size_t)h->smem_optin) c -= 64;
  return c;
}

Classes default_classes(const pma_handle *h) {
  Classes c;
  c.cap_w = largest_tile(h, 1024, 128);
  c.cap_t = 256;
  c.cap = largest_tile(h, 8191, c.cap_w);
  c.base = kClassBaseMin;
  c.widen = 0;
  return c;
}

bool classes_valid(const pma_handle *h, const Classes &c) {
  return c.cap_t >= 2 && c.cap_t <= 1024 && c.cap_t <= c.cap_w && c.cap_w <= 1024 &&
         c.cap_w <= c.cap && c.cap <= 8191 && c.base >= kClassBaseMin &&
         c.base <= kClassBaseMax && (c.widen == 0 || c.widen == 1) &&
         team_smem(h->mixed, h->D, c.cap) <= (size_t)h->smem_optin &&
         team_smem(h->mixed, h->D, c.cap_w) <= (size_t)h->smem_optin;
}

// set the classes and the grids of the team launches (CTAs resident per SM,
// from the shared memory of one tile)
void apply_classes(pma_handle *h, const Classes &c) {
  const size_t smem_sm = (size_t)h->smem_optin + 1024;
  h->cap_t = c.cap_t;
  h->cap_w = c.cap_w;
  h->cap = c.cap;
  h->class_base = c.base;
  h->widen_groups = c.widen;
  h->have_prev = false;  // the last call's counts per class no longer apply
  h->warp_grid =
      h->sms * std::max<int>(1, (int)(smem_sm / (team_smem(h->mixed, h->D, c.cap_w) + 1024)));
  // (about 24 one-warp CTAs per SM are resident at the kernel's register use)
  h->tiny_grid = h->sms * std::min<int>(24, std::max<int>(1, (int)(smem_sm / (team_smem(
                                                                     h->mixed, h->D, c.cap_t) +
                                                                 1024))));
  // large cells and pieces: 8-warp teams, or 12-warp teams when only one
  // 8-warp CTA fits an SM (registers or shared memory): more warps to hide
  // latency, where two 8-warp CTAs would give more if they fitted
  const int b8 = team_blocks(h->mixed, h->D, 8, c.cap, h->smem_optin);
  h->unit_team = b8 == 1 ? 12 : 8;
  h->unit_grid =
      h->sms * (b8 == 1 ? team_blocks(h->mixed, h->D, 12, c.cap, h->smem_optin) : b8);
}

// the candidates the tuner times: tiny-class limit x small-class tile x
// large tile (the largest that fits, or smaller so that more CTAs fit and
// more cells are first cut in global memory)
std::vector<Classes> class_candidates(const pma_handle *h) {
  std::vector<Classes> v;
  const int wmax = largest_tile(h, 1024, 128);
  const int cmax = largest_tile(h, 8191, wmax);
  const int ts[] = {128, 256, 512};
  const int ws[] = {512, wmax};
  const int cs[] = {cmax, 4096, 2048};
  for (int t : ts)
    for (int w : ws)
      for (int c : cs) {
        Classes k{std::min(t, w), w, std::min(c, cmax), kClassBaseMin, 0};
        if (!classes_valid(h, k)) continue;
        bool dup = false;
        for (const Classes &o : v) dup |= o.cap_t == k.cap_t && o.cap_w == k.cap_w && o.cap == k.cap;
        if (!dup) v.push_back(k);
      }
  return v;
}

// population histogram of the cells (fractions of the particles in cells of
// 1-64, 65-256, 257-1024, 1025-4096, 4097-8191 and more particles, in
// twentieths): the part of the tuning key that describes the input
std::string histogram_signature(const std::vector<int32_t> &counts) {
  const int64_t edges[6] = {64, 256, 1024, 4096, 8191, INT64_MAX};
  double f[6] = {0, 0, 0, 0, 0, 0}, tot = 0;
  for (int32_t c : counts) {
    if (c <= 0) continue;
    int b = 0;
    while (c > edges[b]) ++b;
    f[b] += c;
    tot += c;
  }
  char buf[96];
  int k[6];
  for (int b = 0; b < 6; ++b) k[b] = tot > 0 ? (int)std::lround(20.0 * f[b] / tot) : 0;
  snprintf(buf, sizeof buf, "h=%d,%d,%d,%d,%d,%d", k[0], k[1], k[2], k[3], k[4], k[5]);
  return buf;
}

}  // namespace

extern "C" {

const char *pma_error_string(int code) {
  switch (code) {
    case PMA_OK: return "ok";
    case PMA_ERR_INVALID_ARG: return "invalid argument";
    case PMA_ERR_INPUT: return "invalid particle data";
    case PMA_ERR_CUDA: return "CUDA error";
    case PMA_ERR_NOMEM: return "out of memory";
    case PMA_ERR_CAPACITY: return "n exceeds the handle capacity";
    case PMA_ERR_TIMEOUT: return "device wait timed out";
    case PMA_ERR_INTERNAL: return "internal bound exceeded";
    default: return "unknown status";
  }
}

const char *pma_last_error(const pma_handle *h) { return h ? h->last_error.c_str() : ""; }

int pma_create(const pma_config *cfg, pma_handle **out) {
  if (!cfg || !out) return PMA_ERR_INVALID_ARG;
  if (cfg->dx < 1 || cfg->dx > 3 || cfg->dp < 1 || cfg->dp > 3) return PMA_ERR_INVALID_ARG;
  if (cfg->n_cells < 1 || cfg->n_cells > INT32_MAX - 1) return PMA_ERR_INVALID_ARG;
  if (cfg->n_min < 0) return PMA_ERR_INVALID_ARG;
  if (cfg->precision != PMA_FP64 && cfg->precision != PMA_MIXED) return PMA_ERR_INVALID_ARG;
  if (cfg->capacity < 0 || cfg->capacity > INT32_MAX) return PMA_ERR_INVALID_ARG;
  if (cfg->flags & ~(PMA_FLAG_NO_INDEX | PMA_FLAG_SPLIT_NORMALIZED | PMA_FLAG_MOMENTUM_NORM |
                     PMA_FLAG_CONSERVE_ENERGY | PMA_FLAG_ENERGY_STATS))
    return PMA_ERR_INVALID_ARG;
  for (int a = 0; a < cfg->dx; ++a)
    if (!(cfg->cell_size[a] > 0.0) || !std::isfinite(cfg->cell_size[a]))
      return PMA_ERR_INVALID_ARG;
  pma_handle *h = new (std::nothrow) pma_handle();
  if (!h) return PMA_ERR_NOMEM;
  h->cfg = *cfg;
  h->D = cfg->dx + cfg->dp;
  h->mixed = cfg->precision == PMA_MIXED;
  h->capacity = cfg->capacity;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  int smem_optin = 0;
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e != cudaSuccess) {
    delete h;
    return PMA_ERR_CUDA;
  }
  h->smem_optin = smem_optin;
  // population classes (default, or as pma_tune / pma_set_classes choose)
  apply_classes(h, default_classes(h));
  const int64_t N = std::max<int64_t>(cfg->capacity, 1);
  const int64_t C = cfg->n_cells;
  h->bin_tiles = scan_tiles_for(C);
  h->emit_tiles_max = emit_tiles_for(N);
  h->max_pieces = (int)std::min<int64_t>(N, N / 64 + 4096);
  const int64_t Npad = (N + 15) / 16 * 16;
  bool ok = dalloc(&h->counts, C) == cudaSuccess && dalloc(&h->cell_begin, C + 1) == cudaSuccess &&
            dalloc(&h->radix_count, kRadixMaxPasses * kRadixBins) == cudaSuccess &&
            dalloc(&h->radix_status, (size_t)2 * radix_tiles_for(N) * kRadixBins) == cudaSuccess &&
            dalloc(&h->perm, N) == cudaSuccess &&
            dalloc(&h->perm_tmp, N) == cudaSuccess && dalloc(&h->perm_final, Npad) == cudaSuccess &&
            dalloc(&h->big_list, C) == cudaSuccess && dalloc(&h->head, Npad) == cudaSuccess &&
            dalloc(&h->warp_list, C) == cudaSuccess && dalloc(&h->block_list, C) == cudaSuccess &&
            dalloc(&h->tiny_list, C) == cudaSuccess && dalloc(&h->cell_flags, C) == cudaSuccess &&
            cudaMalloc(&h->fin, (size_t)Npad * (h->D + 1) * (h->mixed ? 4 : 8)) == cudaSuccess &&
            dalloc(&h->bin_status, h->bin_tiles) == cudaSuccess &&
            dalloc(&h->tile_count, h->emit_tiles_max) == cudaSuccess &&
            dalloc(&h->tile_prefix, h->emit_tiles_max) == cudaSuccess &&
            dalloc(&h->energy_tiles, 2 * (size_t)h->emit_tiles_max) == cudaSuccess &&
            dalloc(&h->pieces, h->max_pieces) == cudaSuccess && dalloc(&h->ctl, 1) == cudaSuccess &&
            cudaMallocHost(reinterpret_cast<void **>(&h->ctl_host), sizeof(Ctl)) == cudaSuccess;
  h->fin_stride = Npad;
  if (!ok) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return PMA_ERR_NOMEM;
  }
  memset(h->ctl_host, 0, sizeof(Ctl));
  *out = h;
  return PMA_OK;
}

int pma_destroy(pma_handle *h) {
  if (!h) return PMA_OK;
  if (h->pending && h->last_stream) cudaStreamSynchronize(h->last_stream);
  free_all(h);
  delete h;
  return PMA_OK;
}

static int check_common(pma_handle *h, int64_t n, const int32_t *cells, const void *const *pos,
                        const void *const *mom, const void *weights, double tol_x,
                        double tol_p, const pma_output *out) {
  if (!h) return PMA_ERR_INVALID_ARG;
  h->last_error.clear();
  if (n < 0) return fail(h, PMA_ERR_INVALID_ARG, "n < 0");
  if (n > h->capacity) return fail(h, PMA_ERR_CAPACITY, "n exceeds the handle capacity");
  if (!finite_nonneg(tol_x) || !finite_nonneg(tol_p))
    return fail(h, PMA_ERR_INVALID_ARG, "tolerances must be finite and >= 0");
  if (!out) return fail(h, PMA_ERR_INVALID_ARG, "out is NULL");
  if (n == 0) return PMA_OK;
  if (!cells || !pos || !mom || !weights) return fail(h, PMA_ERR_INVALID_ARG, "NULL input");
  for (int a = 0; a < h->cfg.dx; ++a)
    if (!pos[a] || !out->pos[a]) return fail(h, PMA_ERR_INVALID_ARG, "NULL position array");
  for (int a = 0; a < h->cfg.dp; ++a)
    if (!mom[a] || !out->mom[a]) return fail(h, PMA_ERR_INVALID_ARG, "NULL momentum array");
  if (!out->cell || !out->w) return fail(h, PMA_ERR_INVALID_ARG, "NULL output array");
  return PMA_OK;
}

static int enqueue(pma_handle *h, int64_t n, const int32_t *cells, const void *const *pos,
                   const void *const *mom, const void *weights, double tol_x, double tol_p,
                   const pma_output *out, cudaStream_t st) {
  const int64_t C = h->cfg.n_cells;
  uint32_t *cell_flags = out->cell_flags ? out->cell_flags : h->cell_flags;
  if (n == 0) {
    PMA_CUDA(h, cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), st));
    if (out->count_dev) PMA_CUDA(h, cudaMemsetAsync(out->count_dev, 0, sizeof(int64_t), st));
    if (out->cell_flags) PMA_CUDA(h, cudaMemsetAsync(out->cell_flags, 0, C * sizeof(uint32_t), st));
    return PMA_OK;
  }
  {
    static_assert(sizeof(Ctl) % 4 == 0, "Ctl is cleared in 4-byte words");
    ZeroArgs z;
    z.p[0] = reinterpret_cast<uint32_t *>(h->ctl);
    z.words[0] = sizeof(Ctl) / 4;
    z.p[1] = reinterpret_cast<uint32_t *>(h->counts);
    z.words[1] = C;
    z.p[2] = reinterpret_cast<uint32_t *>(h->radix_count);
    z.words[2] = kRadixMaxPasses * kRadixBins;
    z.p[3] = reinterpret_cast<uint32_t *>(h->bin_status);
    z.words[3] = (int64_t)h->bin_tiles * 2;
    z.p[4] = cell_flags;
    z.words[4] = C;
    const int64_t most = std::max<int64_t>(C, (int64_t)h->bin_tiles * 2);
    const int grid =
        (int)std::max<int64_t>(1, std::min<int64_t>((most + 255) / 256, (int64_t)h->sms * 4));
    zero_kernel<<<grid, 256, 0, st>>>(z);
    PMA_CUDA(h, cudaGetLastError());
  }
  const int tiles = emit_tiles_for(n);

  BinArgs b{};
  b.n = n;
  b.cells = cells;
  b.n_cells = (int32_t)C;
  b.cap = h->cap;
  b.n_min = h->cfg.n_min;
  b.counts = h->counts;
  b.cell_begin = h->cell_begin;
  b.perm = h->perm;
  b.unsorted = &h->ctl->unsorted;
  b.big_list = h->big_list;
  b.big_count = &h->ctl->big_count;
  b.cap_w = h->cap_w;
  b.warp_list = h->warp_list;
  b.warp_count = &h->ctl->warp_count;
  b.cap_t = h->cap_t;
  b.tiny_list = h->tiny_list;
  b.tiny_count = &h->ctl->tiny_count;
  b.block_list = h->block_list;
  b.block_count = &h->ctl->block_count;
  b.err = &h->ctl->err;
  b.wait_ns = h->wait_ns ? h->wait_ns : kWaitNs;
  b.withhold_tile = h->withhold_tile;
  b.scan_status = h->bin_status;
  b.scan_ticket = &h->ctl->bin_ticket;
  b.scan_tiles = h->bin_tiles;
  radix_plan(b);
  b.radix_tiles = radix_tiles_for(n);
  b.radix_count = h->radix_count;
  b.radix_ticket = h->ctl->radix_ticket;
  b.radix_status = h->radix_status;
  {
    // intermediate keys in the first two staging columns (written only after
    // Step 1), intermediate indices in the two spare permutation arrays
    const size_t es = h->mixed ? 4 : 8;
    b.radix_keys[0] = reinterpret_cast<int32_t *>(h->fin);
    b.radix_keys[1] = reinterpret_cast<int32_t *>(static_cast<char *>(h->fin) + (size_t)h->fin_stride * es);
    b.radix_vals[0] = h->perm_tmp;
    b.radix_vals[1] = h->perm_final;
  }
  h->cur_ev = h->timing ? h->ev[h->timed % kRing] : nullptr;
  mark(h, 0, st);
  cudaError_t e = launch_binning(b, h->sms, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "binning launch");

  Problem P{};
  P.n = n;
  P.check = &h->ctl->check;
  P.n_cells = (int32_t)C;
  P.dx = h->cfg.dx;
  P.D = h->D;
  P.n_min = h->cfg.n_min;
  P.variant = ((h->cfg.flags & PMA_FLAG_SPLIT_NORMALIZED) ? kVarNormalized : 0) |
              ((h->cfg.flags & PMA_FLAG_MOMENTUM_NORM) ? kVarPNorm : 0);
  P.cap = h->cap;
  P.unsorted = &h->ctl->unsorted;
  P.tol2_x = tol_x * tol_x;
  P.tol2_p = tol_p * tol_p;
  P.tol2_xf = (float)P.tol2_x;
  P.tol2_pf = (float)P.tol2_p;
  for (int a = 0; a < 3; ++a) {
    double L = a < h->cfg.dx ? h->cfg.cell_size[a] : 1.0;
    P.L2[a] = L * L;
    P.L2f[a] = (float)P.L2[a];
  }
  for (int a = 0; a < h->cfg.dx; ++a) P.q[a] = pos[a];
  for (int a = 0; a < h->cfg.dp; ++a) P.q[h->cfg.dx + a] = mom[a];
  P.w = weights;
  P.cells = cells;
  {
    const size_t es = h->mixed ? 4 : 8;
    for (int l = 0; l <= h->D; ++l)
      P.fin[l] = static_cast<char *>(h->fin) + (size_t)l * h->fin_stride * es;
  }
  P.cell_begin = h->cell_begin;
  P.perm = h->perm;
  P.head = h->head;
  P.perm_final = h->perm_final;
  P.err = &h->ctl->err;
  P.stats = h->ctl->stats;
  P.cell_flags = cell_flags;
  P.big_list = h->big_list;
  P.big_count = &h->ctl->big_count;
  P.big_next = &h->ctl->big_next;
  P.pieces = h->pieces;
  P.piece_count = &h->ctl->piece_count;
  P.perm_tmp = h->perm_tmp;
  P.max_pieces = h->max_pieces;
  P.unit_next = h->ctl->unit_next;
  P.cap_w = h->cap_w;
  P.warp_list = h->warp_list;
  P.warp_count = &h->ctl->warp_count;
  P.warp_next = &h->ctl->warp_next;
  P.cap_t = h->cap_t;
  P.class_base = h->class_base;
  P.widen_groups = h->widen_groups;
  P.tiny_list = h->tiny_list;
  P.tiny_count = &h->ctl->tiny_count;
  P.tiny_next = &h->ctl->tiny_next;
  P.block_list = h->block_list;
  P.block_count = &h->ctl->block_count;

  // Launch sizes.  Every kernel below takes its work by ticket or in a
  // grid-stride loop, so any grid of at least one CTA gives the same result.
  // A work source that was empty in the handle's last completed call (for
  // a PIC code, the previous time step) gets a quarter of a CTA per SM: a
  // launch that finds nothing to do then costs less, and one that does find
  // work still does it, only with fewer CTAs.
  auto grid_for = [&](bool was_empty, int grid) {
    return (h->have_prev && was_empty) ? std::min(grid, std::max(1, h->sms / 4)) : grid;
  };
  const pma_stats &pv = h->prev;
  e = launch_gather(P, n, h->mixed, grid_for(pv.sorted_input != 0, h->sms * 8), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "gather launch");
  mark(h, 1, st);  // Step 1 done: binned (and, for ungrouped input, copied in sorted order)
  e = launch_big(P, h->mixed, grid_for(pv.big_cells == 0, h->sms * 4), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "big-cell launch");
  mark(h, 2, st);
  e = launch_team(P, h->mixed, 3, 1, h->cap_t, grid_for(pv.cells_tiny == 0, h->tiny_grid), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "team launch (tiny cells)");
  e = launch_team(P, h->mixed, 0, 4, h->cap_w, grid_for(pv.cells_small == 0, h->warp_grid), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "team launch (small cells)");
  mark(h, 3, st);
  e = launch_team(P, h->mixed, 1, h->unit_team, h->cap,
                  grid_for(pv.cells_large == 0, h->unit_grid), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "team launch (large cells)");
  mark(h, 4, st);
  e = launch_team(P, h->mixed, 2, h->unit_team, h->cap,
                  grid_for(pv.big_cells == 0, h->unit_grid), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "team launch (pieces)");
  mark(h, 5, st);

  EmitArgs m{};
  m.n = n;
  m.check = &h->ctl->check;
  m.dx = h->cfg.dx;
  m.dp = h->cfg.dp;
  m.mixed = h->mixed;
  m.ec = (h->cfg.flags & PMA_FLAG_CONSERVE_ENERGY) ? 1 : 0;
  m.head = h->head;
  m.perm_final = h->perm_final;
  m.cells = cells;
  m.unsorted = &h->ctl->unsorted;
  for (int l = 0; l <= h->D; ++l) m.fin[l] = P.fin[l];
  m.out_cell = out->cell;
  for (int a = 0; a < 3; ++a) {
    m.out_pos[a] = out->pos[a];
    m.out_mom[a] = out->mom[a];
  }
  m.out_w = out->w;
  m.out_index = (h->cfg.flags & PMA_FLAG_NO_INDEX) ? nullptr : out->index;
  m.out_count = out->count_dev;
  m.out_count2 = &h->ctl->count;
  m.err = &h->ctl->err;
  m.tile_count = h->tile_count;
  m.tile_prefix = h->tile_prefix;
  m.tiles = tiles;
  m.energy = (h->cfg.flags & PMA_FLAG_ENERGY_STATS) ? h->ctl->energy : nullptr;
  m.energy_tiles = h->energy_tiles;
  m.energy_ticket = &h->ctl->emit_ticket;
  e = launch_emit(m, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "emit launch");
  mark(h, 6, st);
  if (h->timing) ++h->timed;
  return PMA_OK;
}

int pma_merge(pma_handle *h, int64_t n, const int32_t *cells, const void *const *pos,
              const void *const *mom, const void *weights, double tol_x, double tol_p,
              const pma_output *out, int64_t *count_host, void *stream) {
  int rc = check_common(h, n, cells, pos, mom, weights, tol_x, tol_p, out);
  if (rc != PMA_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = -1;
  PMA_CUDA(h, cudaGetDevice(&dev));
  if (dev != h->device) return fail(h, PMA_ERR_INVALID_ARG, "handle belongs to another device");
  rc = enqueue(h, n, cells, pos, mom, weights, tol_x, tol_p, out, st);
  if (rc != PMA_OK) return rc;
  h->stats = pma_stats{};
  h->stats.n_in = n;
  PMA_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  h->last_stream = st;
  h->pending = true;
  if (!count_host) return PMA_OK;
  rc = pma_sync(h);
  *count_host = h->stats.n_out;
  return rc;
}

int pma_sync(pma_handle *h) {
  if (!h) return PMA_ERR_INVALID_ARG;
  if (!h->pending) return PMA_OK;
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  h->pending = false;
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
  int64_t n_in = h->stats.n_in;
  int rc = status_from_ctl(h);
  h->stats.n_in = n_in;
  if (rc == PMA_OK) {
    h->prev = h->stats;
    h->have_prev = true;
  }
  return rc;
}

int pma_set_timing(pma_handle *h, int enable) {
  if (!h) return PMA_ERR_INVALID_ARG;
  if (enable && !h->ev[0][0]) {
    for (auto &row : h->ev)
      for (auto &e : row)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(h, PMA_ERR_CUDA, "cudaEventCreate");
  }
  h->timing = enable != 0;
  h->timed = 0;
  return PMA_OK;
}

int pma_get_timing(const pma_handle *h, float *ms, int n) {
  if (!h || !ms || h->timed == 0) return PMA_ERR_INVALID_ARG;
  static const int from[PMA_N_STAGES] = {0, 1, 2, 3, 4, 5, 0};
  static const int to[PMA_N_STAGES] = {1, 2, 3, 4, 5, 6, 6};
  const int calls = h->timed < kRing ? h->timed : kRing;
  for (int i = 0; i < n && i < PMA_N_STAGES; ++i) {
    double sum = 0.0;
    for (int c = 0; c < calls; ++c) {
      float t = 0.f;
      if (cudaEventSynchronize(h->ev[c][to[i]]) != cudaSuccess ||
          cudaEventElapsedTime(&t, h->ev[c][from[i]], h->ev[c][to[i]]) != cudaSuccess)
        return PMA_ERR_CUDA;
      sum += t;
    }
    ms[i] = (float)(sum / calls);
  }
  return PMA_OK;
}

int pma_checked_build(void) { return kChecked ? 1 : 0; }

int pma_check_first(const pma_handle *h, uint64_t *site_index) {
  if (!h || !site_index) return PMA_ERR_INVALID_ARG;
  *site_index = h->check_first;
  return PMA_OK;
}

int pma_set_wait_limit(pma_handle *h, int64_t wait_ns) {
  if (!h || wait_ns < 0 || (wait_ns > 0 && wait_ns < 1000)) return PMA_ERR_INVALID_ARG;
  h->wait_ns = (unsigned long long)wait_ns;
  return PMA_OK;
}

int pma_test_status_of_bits(unsigned bits) { return status_of_bits(bits); }

int pma_test_withhold_status(pma_handle *h, int tile) {
  if (!h) return PMA_ERR_INVALID_ARG;
  h->withhold_tile = tile < 0 ? -1 : tile;
  return PMA_OK;
}

int pma_get_stats(const pma_handle *h, pma_stats *out) {
  if (!h || !out) return PMA_ERR_INVALID_ARG;
  *out = h->stats;
  return PMA_OK;
}

// ---------------------------------------------------------------- tuning

int pma_get_classes(const pma_handle *h, int32_t caps[5]) {
  if (!h || !caps) return PMA_ERR_INVALID_ARG;
  caps[0] = h->cap_t;
  caps[1] = h->cap_w;
  caps[2] = h->cap;
  caps[3] = h->class_base;
  caps[4] = h->widen_groups;
  return PMA_OK;
}

int pma_set_classes(pma_handle *h, const int32_t caps[5]) {
  if (!h || !caps) return PMA_ERR_INVALID_ARG;
  const Classes c{caps[0], caps[1], caps[2], caps[3], caps[4]};
  if (!classes_valid(h, c)) return fail(h, PMA_ERR_INVALID_ARG, "invalid population classes");
  if (h->pending) {
    const int rc = pma_sync(h);
    if (rc != PMA_OK) return rc;
  }
  apply_classes(h, c);
  return PMA_OK;
}

namespace {

constexpr int kCaps = 5;

struct CacheEntry {
  std::string key;
  int caps[kCaps];
  double ms;
};

// the cache file: a JSON object, one entry per line,
//   "key": [cap_t, cap_w, cap, base, widen, ms],
std::vector<CacheEntry> read_cache(const char *path) {
  std::vector<CacheEntry> v;
  FILE *f = fopen(path, "r");
  if (!f) return v;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    const char *a = strchr(line, '"');
    if (!a) continue;
    const char *b = strchr(a + 1, '"');
    if (!b) continue;
    const char *br = strchr(b + 1, '[');
    if (!br) continue;
    CacheEntry e;
    e.key.assign(a + 1, b);
    if (sscanf(br + 1, "%d , %d , %d , %d , %d , %lf", &e.caps[0], &e.caps[1], &e.caps[2],
               &e.caps[3], &e.caps[4], &e.ms) == 6)
      v.push_back(e);
  }
  fclose(f);
  return v;
}

bool write_cache(const char *path, const std::vector<CacheEntry> &v) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return false;
  fprintf(f, "{\n");
  for (size_t i = 0; i < v.size(); ++i)
    fprintf(f, "  \"%s\": [%d, %d, %d, %d, %d, %.6g]%s\n", v[i].key.c_str(), v[i].caps[0],
            v[i].caps[1], v[i].caps[2], v[i].caps[3], v[i].caps[4], v[i].ms,
            i + 1 < v.size() ? "," : "");
  fprintf(f, "}\n");
  const bool ok = fclose(f) == 0;
  return ok && rename(tmp.c_str(), path) == 0;
}

}  // namespace

int pma_tune_cache_lookup(const char *path, const char *key, int32_t caps[5]) {
  if (!path || !key || !caps) return PMA_ERR_INVALID_ARG;
  for (const CacheEntry &e : read_cache(path))
    if (e.key == key) {
      for (int i = 0; i < kCaps; ++i) caps[i] = e.caps[i];
      return PMA_OK;
    }
  return PMA_ERR_INVALID_ARG;
}

int pma_tune_cache_store(const char *path, const char *key, const int32_t caps[5], double ms) {
  if (!path || !key || !caps || strchr(key, '"') || strchr(key, '\n')) return PMA_ERR_INVALID_ARG;
  std::vector<CacheEntry> v = read_cache(path);
  bool found = false;
  for (CacheEntry &e : v)
    if (e.key == key) {
      for (int i = 0; i < kCaps; ++i) e.caps[i] = caps[i];
      e.ms = ms;
      found = true;
    }
  if (!found) {
    CacheEntry e;
    e.key = key;
    for (int i = 0; i < kCaps; ++i) e.caps[i] = caps[i];
    e.ms = ms;
    v.push_back(e);
  }
  return write_cache(path, v) ? PMA_OK : PMA_ERR_INVALID_ARG;
}

int pma_tune(pma_handle *h, int64_t n, const int32_t *cells, const void *const *pos,
             const void *const *mom, const void *weights, double tol_x, double tol_p,
             const pma_output *out, void *stream) {
  int rc = check_common(h, n, cells, pos, mom, weights, tol_x, tol_p, out);
  if (rc != PMA_OK) return rc;
  if (n == 0) return PMA_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a prefix of the input (at most 2^26 particles) stands for the whole
  const int64_t ns = std::min<int64_t>(n, (int64_t)1 << 26);
  pma_output o = *out;
  o.cell_flags = nullptr;
  int64_t M = 0;
  rc = pma_merge(h, ns, cells, pos, mom, weights, tol_x, tol_p, &o, &M, stream);
  if (rc != PMA_OK) return rc;
  std::vector<int32_t> counts((size_t)h->cfg.n_cells);
  PMA_CUDA(h, cudaMemcpy(counts.data(), h->counts, counts.size() * sizeof(int32_t),
                         cudaMemcpyDeviceToHost));
  char key[256];
  snprintf(key, sizeof key, "D=%d %s flags=%u sms=%d %s", h->D, h->mixed ? "mixed" : "fp64",
           h->cfg.flags, h->sms, histogram_signature(counts).c_str());
  const char *cache = getenv("PMA_TUNE_CACHE");
  int32_t caps[kCaps];
  if (cache && *cache && pma_tune_cache_lookup(cache, key, caps) == PMA_OK &&
      pma_set_classes(h, caps) == PMA_OK)
    return PMA_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PMA_CUDA(h, cudaEventCreate(&e0));
  PMA_CUDA(h, cudaEventCreate(&e1));
  Classes best = default_classes(h);
  double best_ms = 1e300;
  // median of three timed calls after one untimed
  auto time_one = [&](const Classes &c) {
    apply_classes(h, c);
    float t[3];
    for (int r = -1; r < 3 && rc == PMA_OK; ++r) {
      if (r >= 0) cudaEventRecord(e0, st);
      rc = pma_merge(h, ns, cells, pos, mom, weights, tol_x, tol_p, &o, nullptr, stream);
      if (rc != PMA_OK) break;
      if (r >= 0) cudaEventRecord(e1, st);
      rc = pma_sync(h);
      if (r >= 0 && rc == PMA_OK) cudaEventElapsedTime(&t[r], e0, e1);
    }
    if (rc != PMA_OK) return;
    std::sort(t, t + 3);
    if (t[1] < best_ms) {
      best_ms = t[1];
      best = c;
    }
  };
  // the population limits with the default class base, then the class base
  for (const Classes &c : class_candidates(h)) {
    time_one(c);
    if (rc != PMA_OK) break;
  }
  const Classes limits = best;
  for (int b : {16, 24, 32}) {
    if (rc != PMA_OK) break;
    Classes c = limits;
    c.base = b;
    time_one(c);
  }
  // then wider groups in sparse rounds, with the best class base and with
  // base 24 (their best partner on the measured workloads)
  const Classes narrow = best;
  for (int b : {narrow.base, 24}) {
    if (rc != PMA_OK) break;
    if (b == 24 && narrow.base == 24) continue;
    Classes c = narrow;
    c.base = b;
    c.widen = 1;
    time_one(c);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply_classes(h, best);
  if (rc != PMA_OK) return rc;
  if (cache && *cache) {
    caps[0] = best.cap_t;
    caps[1] = best.cap_w;
    caps[2] = best.cap;
    caps[3] = best.base;
    caps[4] = best.widen;
    pma_tune_cache_store(cache, key, caps, best_ms);
  }
  return PMA_OK;
}

int pma_merge_host(pma_handle *h, int64_t n, const int32_t *cells, const void *const *pos,
                   const void *const *mom, const void *weights, double tol_x, double tol_p,
                   const pma_output *out_host, int64_t *count_host, void *stream) {
  int rc = check_common(h, n, cells, pos, mom, weights, tol_x, tol_p, out_host);
  if (rc != PMA_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Staging &S = h->stage;
  const size_t N = (size_t)std::max<int64_t>(h->capacity, 1);
  const size_t ts = h->mixed ? sizeof(float) : sizeof(double);
  if (!S.ready) {
    bool ok = dalloc(&S.cells, N) == cudaSuccess && dalloc(&S.out_cell, N) == cudaSuccess &&
              dalloc(&S.out_w, N) == cudaSuccess && dalloc(&S.out_index, N) == cudaSuccess &&
              cudaMalloc(&S.w, N * ts) == cudaSuccess;
    for (int l = 0; ok && l < h->D; ++l) ok = cudaMalloc(&S.q[l], N * ts) == cudaSuccess;
    for (int a = 0; ok && a < h->cfg.dx; ++a) ok = cudaMalloc(&S.out_pos[a], N * ts) == cudaSuccess;
    for (int a = 0; ok && a < h->cfg.dp; ++a) ok = dalloc(&S.out_mom[a], N) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return fail(h, PMA_ERR_NOMEM, "staging buffers");
    }
    S.ready = true;
  }
  if (n > 0) {
    PMA_CUDA(h, cudaMemcpyAsync(S.cells, cells, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    for (int a = 0; a < h->cfg.dx; ++a)
      PMA_CUDA(h, cudaMemcpyAsync(S.q[a], pos[a], n * ts, cudaMemcpyHostToDevice, st));
    for (int a = 0; a < h->cfg.dp; ++a)
      PMA_CUDA(h, cudaMemcpyAsync(S.q[h->cfg.dx + a], mom[a], n * ts, cudaMemcpyHostToDevice, st));
    PMA_CUDA(h, cudaMemcpyAsync(S.w, weights, n * ts, cudaMemcpyHostToDevice, st));
  }
  pma_output dout{};
  dout.cell = S.out_cell;
  for (int a = 0; a < 3; ++a) {
    dout.pos[a] = S.out_pos[a];
    dout.mom[a] = S.out_mom[a];
  }
  dout.w = S.out_w;
  dout.index = out_host->index ? S.out_index : nullptr;
  const void *dq[3], *dm[3];
  for (int a = 0; a < h->cfg.dx; ++a) dq[a] = S.q[a];
  for (int a = 0; a < h->cfg.dp; ++a) dm[a] = S.q[h->cfg.dx + a];
  int64_t M = 0;
  rc = pma_merge(h, n, S.cells, dq, dm, S.w, tol_x, tol_p, &dout, &M, stream);
  if (rc != PMA_OK) return rc;
  if (M > 0) {
    PMA_CUDA(h, cudaMemcpyAsync(out_host->cell, S.out_cell, M * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st));
    for (int a = 0; a < h->cfg.dx; ++a)
      PMA_CUDA(h, cudaMemcpyAsync(out_host->pos[a], S.out_pos[a], M * ts, cudaMemcpyDeviceToHost, st));
    for (int a = 0; a < h->cfg.dp; ++a)
      PMA_CUDA(h, cudaMemcpyAsync(out_host->mom[a], S.out_mom[a], M * sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
    PMA_CUDA(h, cudaMemcpyAsync(out_host->w, S.out_w, M * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (out_host->index && n > 0)
    PMA_CUDA(h, cudaMemcpyAsync(out_host->index, S.out_index, n * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st));
  if (out_host->cell_flags)
    PMA_CUDA(h, cudaMemcpyAsync(out_host->cell_flags, h->cell_flags,
                                h->cfg.n_cells * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  PMA_CUDA(h, cudaStreamSynchronize(st));
  if (count_host) *count_host = M;
  return PMA_OK;
}

}  // extern "C"
