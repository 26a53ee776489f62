// Host-side launchers shared by the translation units of the library.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "pma_device.cuh"

namespace pma {

// the class base B of the team kernels' subset size classes (the largest
// subset a single lane takes) ranges over [kClassBaseMin, kClassBaseMax]: at
// most 32 terms per lane in every class of a 1024-particle tile, and shared
// memory is sized for the smallest B
constexpr int kClassBaseMin = 12;
constexpr int kClassBaseMax = 32;

// split.cu
size_t unit_smem(int mixed, int D, int cap);
cudaError_t launch_big(const Problem &P, int mixed, int grid, cudaStream_t st);
// warp.cu: a team of `team` (4 or 8) warps per unit of up to `cap` particles;
// mode 0 small-class cells, 1 large-class cells, 2 pieces of big cells
size_t team_smem(int mixed, int D, int cap);
// CTAs per SM of the large-cell team kernel (8 or 12 warps) at tile size cap
int team_blocks(int mixed, int D, int team, int cap, int smem_optin);
cudaError_t launch_team(const Problem &P, int mixed, int mode, int team, int cap, int grid,
                        cudaStream_t st);

// bin.cu
struct BinArgs {
  int64_t n;
  const int32_t *cells;
  int32_t n_cells;
  int32_t cap;
  int32_t n_min;
  int32_t *counts;      // [n_cells]
  int32_t *cell_begin;  // [n_cells + 1]
  int32_t *perm;        // [n]
  int32_t *unsorted;    // device flag
  int32_t *big_list;
  int32_t *big_count;
  int32_t cap_w;
  int32_t *warp_list;
  int32_t *warp_count;
  int32_t cap_t;          // cells of at most cap_t particles: the tiny class
  int32_t *tiny_list;
  int32_t *tiny_count;
  int32_t *block_list;
  int32_t *block_count;
  unsigned *err;
  unsigned long long wait_ns;       // limit of every bounded wait
  int32_t withhold_tile;            // failure-detection test: this scan tile never
                                    // publishes its status (-1: none)
  unsigned long long *scan_status;  // [scan tiles]
  int32_t *scan_ticket;
  int32_t scan_tiles;
  // stable LSD radix sort of ungrouped input by cell id (Step 1)
  int32_t radix_passes;             // <= kRadixMaxPasses
  int32_t radix_shift[4];           // first key bit of each pass
  int32_t radix_bits[4];            // key bits of each pass (<= 8)
  int32_t radix_tiles;              // tiles of kRadixTile keys
  int32_t *radix_count;             // [kRadixMaxPasses][256] digit counts (zeroed by the caller)
  int32_t *radix_ticket;            // [kRadixMaxPasses] tile tickets (zeroed by the caller)
  unsigned long long *radix_status; // [2][radix_tiles][256] look-back words
  int32_t *radix_keys[2];           // [n] intermediate keys
  int32_t *radix_vals[2];           // [n] intermediate input indices
};
constexpr int kRadixMaxPasses = 4;
constexpr int kRadixBins = 256;
cudaError_t launch_binning(const BinArgs &a, int sms, cudaStream_t st);
// ungrouped input: the particles in sorted order into the staging columns
// (grid-stride: any grid of at least one CTA is correct)
cudaError_t launch_gather(const Problem &P, int64_t n, int mixed, int grid_max, cudaStream_t st);
int scan_tiles_for(int64_t n);
int radix_tiles_for(int64_t n);
// passes and bit split of the cell-id keys (values 0..n_cells, n_cells marks
// an invalid id); fills a.radix_passes / radix_shift / radix_bits
void radix_plan(BinArgs &a);

// emit.cu
struct EmitArgs {
  int64_t n;
  unsigned long long *check;  // first failed bounds check (checked build)
  int32_t dx, dp, mixed;
  int32_t ec;  // energy-conserving replacement (PMA_FLAG_CONSERVE_ENERGY)
  const uint8_t *head;
  const int32_t *perm_final;
  const int32_t *cells;
  const int32_t *unsorted;  // device flag: cell ids of final positions are cells[p] when 0
  const void *fin[kMaxD + 1];  // staged coordinates and weight in final order
  int32_t *out_cell;
  void *out_pos[3];
  double *out_mom[3];
  double *out_w;
  int32_t *out_index;
  int64_t *out_count;   // device word(s) receiving M
  int64_t *out_count2;
  unsigned *err;
  int32_t *tile_count;    // [tiles] heads per tile
  long long *tile_prefix; // [tiles] heads before each tile
  int32_t tiles;
  double *energy;         // [2] kinetic energy in and out, or null
  double *energy_tiles;   // [2][tiles] per-tile partial sums (workspace)
  int32_t *energy_ticket; // CTAs done (zeroed by the caller); the last one sums
};
int emit_tiles_for(int64_t n);
cudaError_t launch_emit(const EmitArgs &a, cudaStream_t st);

}  // namespace pma
