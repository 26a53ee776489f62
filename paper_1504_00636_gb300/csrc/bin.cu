// Step 1 of the method: collect the particles of every simulation cell.
//
// hist_kernel   validates the cell ids, counts particles per cell (warp-
//               aggregated atomics) and detects input that is already
//               grouped by cell (non-decreasing ids).
// scan_kernel   exclusive prefix of the counts -> first sorted position of
//               every cell (single pass, decoupled look-back), and the list of
//               cells too large for one CTA's shared memory.
// scatter_kernel  (only for ungrouped input) writes the permutation
//               sorted position -> input index.
#include "lookback.cuh"
#include "pma_launch.h"

namespace pma {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

int scan_tiles_for(int64_t n) { return (int)((n + kScanTile - 1) / kScanTile); }

__global__ void hist_kernel(BinArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int unsorted = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n;
       base += stride) {
    int64_t i = base + lane;
    int c = -1;
    if (i < a.n) {
      c = a.cells[i];
      if (c < 0 || c >= a.n_cells) {
        atomicOr(a.err, kErrInput);
        c = -1;
      } else if (i > 0 && a.cells[i - 1] > c) {
        unsorted = 1;
      }
    }
    unsigned grp = __match_any_sync(0xffffffffu, c);
    if (c >= 0 && lane == __ffs(grp) - 1) atomicAdd(&a.counts[c], __popc(grp));
  }
  if (__any_sync(0xffffffffu, unsorted) && lane == 0) atomicExch(a.unsorted, 1);
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(BinArgs a) {
  __shared__ int s_tile;
  __shared__ int s_warp[32];
  __shared__ long long s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(a.scan_ticket, 1);
  __syncthreads();
  const int tile = s_tile;
  const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t i = base + j;
    v[j] = i < a.n_cells ? a.counts[i] : 0;
    sum += v[j];
    if (v[j] > 0) {
      // population class of the cell
      if (v[j] <= a.n_min || v[j] <= a.cap_w)
        a.warp_list[atomicAdd(a.warp_count, 1)] = (int)i;
      else if (v[j] <= a.cap)
        a.block_list[atomicAdd(a.block_count, 1)] = (int)i;
      else
        a.big_list[atomicAdd(a.big_count, 1)] = (int)i;
    }
  }
  int total;
  int ex = block_exclusive_scan(sum, s_warp, &total);
  if (threadIdx.x < 32) {
    const long long pre = warp_exclusive_prefix(a.scan_status, tile, total, a.err);
    if (threadIdx.x == 0) s_prefix = pre;
  }
  __syncthreads();
  long long run = s_prefix + ex;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t i = base + j;
    if (i < a.n_cells) a.cell_begin[i] = (int32_t)run;
    run += v[j];
    if (i == a.n_cells - 1) a.cell_begin[a.n_cells] = (int32_t)run;
  }
}

__global__ void scatter_kernel(BinArgs a) {
  if (*a.unsorted == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n;
       base += stride) {
    int64_t i = base + lane;
    int c = -1;
    if (i < a.n) {
      c = a.cells[i];
      if (c < 0 || c >= a.n_cells) c = -1;
    }
    unsigned grp = __match_any_sync(0xffffffffu, c);
    int leader = __ffs(grp) - 1;
    int off = 0;
    if (c >= 0 && lane == leader) off = atomicAdd(&a.fill[c], __popc(grp));
    off = __shfl_sync(0xffffffffu, off, leader);
    if (c >= 0) a.perm[a.cell_begin[c] + off + __popc(grp & lt)] = (int32_t)i;
  }
}

cudaError_t launch_binning(const BinArgs &a, int sms, cudaStream_t st) {
  if (a.n > 0) {
    int grid = (int)std::min<int64_t>((a.n + 255) / 256, (int64_t)sms * 8);
    hist_kernel<<<grid, 256, 0, st>>>(a);
  }
  scan_kernel<<<a.scan_tiles, kScanThreads, 0, st>>>(a);
  if (a.n > 0) {
    int grid = (int)std::min<int64_t>((a.n + 255) / 256, (int64_t)sms * 8);
    scatter_kernel<<<grid, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace pma
