// Step 1 of the method: collect the particles of every simulation cell.
//
// hist_kernel   validates the cell ids, counts particles per cell (one
//               atomic per run of equal ids, in shared memory when the cells
//               are few) and detects input that is already grouped by cell
//               (non-decreasing ids).
// scan_kernel   exclusive prefix of the counts -> first sorted position of
//               every cell (single pass, decoupled look-back), and the list of
//               cells too large for one CTA's shared memory.
// radix_prep_kernel, radix_pass_kernel
//               (only for ungrouped input) a stable least-significant-digit
//               radix sort of the cell ids, one pass per digit of up to 8
//               bits, gives the permutation sorted position -> input index
//               in (cell, input index) order, so the result does not depend
//               on how the GPU schedules the work.
#include <climits>

#include "lookback.cuh"
#include "pma_launch.h"

namespace pma {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

int scan_tiles_for(int64_t n) { return (int)((n + kScanTile - 1) / kScanTile); }

constexpr int kHistRows = 4;  // rows of 32 ids a warp loads per step

// Each warp reads kHistRows rows of 32 consecutive ids at a time.  Inside a
// row, every run of equal valid ids adds its length to the cell's count with
// one atomic (run starts from a neighbour shuffle and one ballot), so ids
// grouped by cell cost one atomic per run; ungrouped ids stay correct (runs
// of one).  A pair of neighbours in decreasing order marks the input as not
// grouped.  With few cells (SMEM) the CTA counts in shared memory and adds
// its non-zero counts to the global ones at the end: ungrouped ids then cost
// one global atomic per cell and CTA instead of one per particle.
constexpr int kHistSmemCells = 12288;  // 48 KB of shared counters
constexpr int kHistSmemThreads = 1024;

template <bool SMEM>
__global__ void __launch_bounds__(SMEM ? kHistSmemThreads : 256) hist_kernel(BinArgs a) {
  extern __shared__ int s_count[];  // SMEM: [n_cells]
  if (SMEM) {
    for (int k = threadIdx.x; k < a.n_cells; k += blockDim.x) s_count[k] = 0;
    __syncthreads();
  }
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t step = 32 * kHistRows;
  bool unsorted = false, bad = false;
  for (int64_t w0 = warp * step; w0 < a.n; w0 += warps * step) {  // warp-uniform
    int c[kHistRows];
#pragma unroll
    for (int j = 0; j < kHistRows; ++j) {
      const int64_t i = w0 + j * 32 + lane;
      c[j] = i < a.n ? a.cells[i] : -1;
    }
    int carry = (lane == 0 && w0 > 0) ? a.cells[w0 - 1] : INT_MIN;  // the id before the row
#pragma unroll
    for (int j = 0; j < kHistRows; ++j) {
      const int64_t i = w0 + j * 32 + lane;
      const int v = c[j];
      const bool in = i < a.n;
      const bool valid = in && v >= 0 && v < a.n_cells;
      bad |= in && !valid;
      int prev = __shfl_up_sync(full, v, 1);
      if (lane == 0) prev = carry;
      if (valid && prev > v) unsorted = true;
      carry = __shfl_sync(full, v, 31);
      const int key = valid ? v : -1;
      const int kprev = __shfl_up_sync(full, key, 1);
      const bool start = lane == 0 || kprev != key;
      const unsigned starts = __ballot_sync(full, start);
      if (start && key >= 0) {
        const unsigned later = starts & ~((2u << lane) - 1u);
        const int end = later ? __ffs(later) - 1 : 32;
        atomicAdd(SMEM ? &s_count[key] : &a.counts[key], end - lane);
      }
    }
  }
  if (__any_sync(full, bad) && lane == 0) atomicOr(a.err, kErrInput);
  if (__any_sync(full, unsorted) && lane == 0) atomicExch(a.unsorted, 1);
  if (SMEM) {
    __syncthreads();
    for (int k = threadIdx.x; k < a.n_cells; k += blockDim.x)
      if (s_count[k]) atomicAdd(&a.counts[k], s_count[k]);
  }
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
      if (v[j] <= a.cap_t)
        a.tiny_list[atomicAdd(a.tiny_count, 1)] = (int)i;
      else if (v[j] <= a.n_min || v[j] <= a.cap_w)
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
    const long long pre = warp_exclusive_prefix(a.scan_status, tile, total, a.err, a.wait_ns,
                                                tile != a.withhold_tile);
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

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;
static_assert(kRadixThreads == kRadixBins, "one thread per digit");

int radix_tiles_for(int64_t n) { return (int)((n + kRadixTile - 1) / kRadixTile); }

void radix_plan(BinArgs &a) {
  // keys 0..n_cells (n_cells = invalid id), so bits for the value n_cells
  int bits = 1;
  while (bits < 32 && ((int64_t)1 << bits) <= (int64_t)a.n_cells) ++bits;
  const int passes = (bits + 7) / 8;
  const int per = (bits + passes - 1) / passes;
  a.radix_passes = passes;
  for (int p = 0; p < kRadixMaxPasses; ++p) {
    a.radix_shift[p] = p * per;
    a.radix_bits[p] = p < passes ? std::min(per, bits - p * per) : 0;
  }
}

__device__ __forceinline__ unsigned radix_key(const BinArgs &a, int c) {
  return (c < 0 || c >= a.n_cells) ? (unsigned)a.n_cells : (unsigned)c;
}

// digit counts of every pass, and the first pass's look-back words cleared
__global__ void __launch_bounds__(kRadixThreads) radix_prep_kernel(BinArgs a) {
  if (*a.unsorted == 0 || timed_out(a.err)) return;
  __shared__ int s_count[kRadixMaxPasses][kRadixBins];
  for (int k = threadIdx.x; k < kRadixMaxPasses * kRadixBins; k += blockDim.x)
    (&s_count[0][0])[k] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const unsigned key = radix_key(a, a.cells[i]);
    for (int p = 0; p < a.radix_passes; ++p)
      atomicAdd(&s_count[p][(key >> a.radix_shift[p]) & ((1u << a.radix_bits[p]) - 1u)], 1);
  }
  const int64_t words = (int64_t)a.radix_tiles * kRadixBins;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < words; k += stride)
    a.radix_status[k] = 0ull;
  __syncthreads();
  for (int p = 0; p < a.radix_passes; ++p) {
    const int v = s_count[p][threadIdx.x];
    if (v) atomicAdd(&a.radix_count[p * kRadixBins + threadIdx.x], v);
  }
}

// One stable counting pass over key bits [shift, shift + bits).  Every warp
// ranks a contiguous run of 32 * kRadixItems keys in input order (match on
// the digit, running per-warp counts), the CTA combines its warps, and each
// digit's offset across tiles comes from a per-digit decoupled look-back.
__global__ void __launch_bounds__(kRadixThreads) radix_pass_kernel(BinArgs a, int p) {
  if (*a.unsorted == 0 || timed_out(a.err)) return;
  __shared__ int s_tile;
  __shared__ int s_hist[kRadixWarps][kRadixBins];
  __shared__ int s_base[kRadixBins];
  __shared__ int s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = tid; k < kRadixWarps * kRadixBins; k += kRadixThreads) (&s_hist[0][0])[k] = 0;
  if (tid == 0) s_tile = atomicAdd(&a.radix_ticket[p], 1);
  // first sorted position of every digit of this pass
  int total;
  const int digit_base = block_exclusive_scan(a.radix_count[p * kRadixBins + tid], s_warp, &total);
  const int tile = s_tile;  // published by the scan's barriers
  const size_t region = (size_t)a.radix_tiles * kRadixBins;
  unsigned long long *status = a.radix_status + (size_t)(p & 1) * region;
  // the next pass uses the other region: clear this tile's words of it
  if (p + 1 < a.radix_passes) a.radix_status[(size_t)((p + 1) & 1) * region +
                                             (size_t)tile * kRadixBins + tid] = 0ull;
  const bool first = p == 0, last = p + 1 == a.radix_passes;
  const int32_t *keys_in = first ? nullptr : a.radix_keys[(p - 1) & 1];
  const int32_t *vals_in = first ? nullptr : a.radix_vals[(p - 1) & 1];
  const unsigned shift = a.radix_shift[p], mask = (1u << a.radix_bits[p]) - 1u;
  const int64_t seg = (int64_t)tile * kRadixTile + (int64_t)warp * (32 * kRadixItems);
  unsigned key[kRadixItems];
  int val[kRadixItems], rank[kRadixItems];
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const int64_t i = seg + j * 32 + lane;
    key[j] = 0xffffffffu;  // beyond n
    val[j] = -1;
    if (i < a.n) {
      if (first) {
        key[j] = radix_key(a, a.cells[i]);
        val[j] = (int)i;
      } else {
        key[j] = (unsigned)keys_in[i];
        val[j] = vals_in[i];
      }
    }
  }
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const int d = key[j] == 0xffffffffu ? kRadixBins : (int)((key[j] >> shift) & mask);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = d < kRadixBins ? s_hist[warp][d] : 0;
    __syncwarp();
    if (d < kRadixBins && lane == __ffs(peers) - 1) s_hist[warp][d] = before + __popc(peers);
    __syncwarp();
    rank[j] = before + __popc(peers & lt);
  }
  __syncthreads();
  // digit tid: offsets of the warps inside the tile, then across tiles
  int run = 0;
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) {
    const int t = s_hist[w][tid];
    s_hist[w][tid] = run;
    run += t;
  }
  const long long before_tile =
      tile_exclusive_prefix_batched(status + tid, tile, run, a.err, kRadixBins, a.wait_ns);
  s_base[tid] = digit_base + (int)before_tile;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    if (key[j] == 0xffffffffu) continue;
    const int d = (int)((key[j] >> shift) & mask);
    const int64_t pos = (int64_t)s_base[d] + s_hist[warp][d] + rank[j];
    if ((uint64_t)pos >= (uint64_t)a.n) {  // only after a failed look-back
      atomicOr(a.err, kErrInternal);
      continue;
    }
    if (last) {
      a.perm[pos] = val[j];
    } else {
      a.radix_keys[p & 1][pos] = (int32_t)key[j];
      a.radix_vals[p & 1][pos] = val[j];
    }
  }
}

// Ungrouped input only (returns at once otherwise): every particle's
// coordinates and weight in sorted (cell, input index) order, copied into
// the staging columns, so that the partition kernels read each cell
// contiguously instead of gathering it through the permutation (they later
// overwrite the columns of a cell with its final order).  One sorted
// position per thread and step: the permutation and the stores are
// coalesced, the loads scattered.
constexpr int kGatherUnroll = 4;

template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(Problem P, int64_t n) {
  if (*P.unsorted == 0 || timed_out(P.err)) return;
  const int D = P.D;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n;
       i0 += stride * kGatherUnroll) {
    int src[kGatherUnroll];
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
      const int64_t i = i0 + u * stride;
      src[u] = i < n ? P.perm[i] : -1;
      if ((unsigned)src[u] >= (unsigned)n) src[u] = -1;  // never after a complete sort
    }
#pragma unroll
    for (int l = 0; l <= kMaxD; ++l) {
      if (l > D) break;
      const T *col = static_cast<const T *>(l < D ? P.q[l] : P.w);
      T v[kGatherUnroll];
#pragma unroll
      for (int u = 0; u < kGatherUnroll; ++u) v[u] = src[u] >= 0 ? col[src[u]] : T(0);
#pragma unroll
      for (int u = 0; u < kGatherUnroll; ++u)
        if (src[u] >= 0) static_cast<T *>(P.fin[l])[i0 + u * stride] = v[u];
    }
  }
}

cudaError_t launch_gather(const Problem &P, int64_t n, int mixed, int grid_max, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, grid_max));
  if (mixed)
    gather_kernel<float><<<grid, 256, 0, st>>>(P, n);
  else
    gather_kernel<double><<<grid, 256, 0, st>>>(P, n);
  return cudaGetLastError();
}

cudaError_t launch_binning(const BinArgs &a, int sms, cudaStream_t st) {
  if (a.n > 0) {
    if (a.n_cells <= kHistSmemCells) {
      const int grid = (int)std::min<int64_t>(
          (a.n + kHistSmemThreads * kHistRows - 1) / (kHistSmemThreads * kHistRows),
          (int64_t)sms * 2);
      hist_kernel<true><<<grid, kHistSmemThreads, (size_t)a.n_cells * sizeof(int), st>>>(a);
    } else {
      const int grid = (int)std::min<int64_t>((a.n + 256 * kHistRows - 1) / (256 * kHistRows),
                                              (int64_t)sms * 8);
      hist_kernel<false><<<grid, 256, 0, st>>>(a);
    }
  }
  scan_kernel<<<a.scan_tiles, kScanThreads, 0, st>>>(a);
  if (a.n > 0) {
    // the radix kernels return at once when the input is grouped by cell
    int grid = (int)std::min<int64_t>((a.n + kRadixThreads - 1) / kRadixThreads, (int64_t)sms * 4);
    radix_prep_kernel<<<grid, kRadixThreads, 0, st>>>(a);
    for (int p = 0; p < a.radix_passes; ++p)
      radix_pass_kernel<<<radix_tiles_for(a.n), kRadixThreads, 0, st>>>(a, p);
  }
  return cudaGetLastError();
}

}  // namespace pma
