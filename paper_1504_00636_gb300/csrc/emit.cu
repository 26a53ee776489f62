// Step 7: replace every final set by its centroid, compacted in canonical
// order; the centroid (W, X, P) of a merged set is summed here from its
// members, in FP64.  The final sets of all cells are contiguous position ranges marked by
// a head byte at their first position; cells are laid out in ascending order
// and the sets of a cell in V1-first depth-first order, so the output slot of
// a set is the number of heads before it.  One pass: each tile counts its
// heads, gets its exclusive prefix by decoupled look-back, and writes the
// merged particles and the input->output index.
#include "lookback.cuh"
#include "pma_launch.h"

namespace pma {

constexpr int kEmitThreads = 256;
constexpr int kEmitChunk = 4;  // consecutive positions per chunk
constexpr int kEmitTile = kEmitThreads * kEmitChunk;

int emit_tiles_for(int64_t n) { return (int)((n + kEmitTile - 1) / kEmitTile); }

template <typename T>
__device__ __forceinline__ double to_f64(T x);
template <>
__device__ __forceinline__ double to_f64<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ double to_f64<float>(float x) {
  return f2d_exact(x);
}

template <typename T>
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(EmitArgs a) {
  __shared__ int s_tile;
  __shared__ int s_warp[32];
  __shared__ long long s_prefix;
  __shared__ unsigned short s_mask[kEmitThreads];
  __shared__ int s_chunk[kEmitThreads];
  __shared__ __align__(16) uint8_t s_head[kEmitTile];
  __shared__ int s_nmerged;
  __shared__ int2 s_merged[kEmitTile / 2 + 1];  // (offset in tile, output slot)
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_tile = atomicAdd(a.scan_ticket, 1);
    s_nmerged = 0;
  }
  __syncthreads();
  const int tile = s_tile;
  const int64_t t0 = (int64_t)tile * kEmitTile;
  // heads of my chunk of 4 consecutive positions
  const int64_t c0 = t0 + (int64_t)tid * kEmitChunk;
  unsigned hw = 0;
  if (c0 + kEmitChunk <= a.n) {
    hw = *reinterpret_cast<const unsigned *>(a.head + c0);
  } else {
    for (int j = 0; j < kEmitChunk; ++j)
      if (c0 + j < a.n) hw |= (unsigned)a.head[c0 + j] << (8 * j);
  }
  unsigned mask = 0;
#pragma unroll
  for (int j = 0; j < kEmitChunk; ++j)
    if ((hw >> (8 * j)) & 0xffu) mask |= 1u << j;
  reinterpret_cast<unsigned *>(s_head)[tid] = hw;
  int total;
  const int ex = block_exclusive_scan(__popc(mask), s_warp, &total);
  s_mask[tid] = (unsigned short)mask;
  s_chunk[tid] = ex;
  if (tid < 32) {
    const long long pre = warp_exclusive_prefix(a.scan_status, tile, total, a.err);
    if (tid == 0) {
      s_prefix = pre;
      if (tile == a.tiles - 1) {
        if (a.out_count) *a.out_count = pre + total;
        if (a.out_count2) *a.out_count2 = pre + total;
      }
    }
  }
  __syncthreads();
  const long long prefix = s_prefix;
  const int32_t *__restrict__ perm_final = a.perm_final;
  const int32_t *__restrict__ cells = a.cells;
  const bool sorted = *a.unsorted == 0;
  const int D = a.dx + a.dp;
  bool bad = false, internal = false;
  // positions in strided order: consecutive threads, consecutive positions;
  // all loads of a thread's positions are issued before its stores
  int orig[kEmitChunk], hh[kEmitChunk], cc[kEmitChunk];
  long long slot[kEmitChunk];
  T xv[kEmitChunk][kMaxD + 1];
#pragma unroll
  for (int j = 0; j < kEmitChunk; ++j) {
    const int off = j * kEmitThreads + tid;
    const int64_t p = t0 + off;
    orig[j] = -1;
    hh[j] = -1;  // beyond n
    cc[j] = 0;
    slot[j] = 0;
#pragma unroll
    for (int l = 0; l <= kMaxD; ++l) xv[j][l] = T(1);
    if (p < a.n) {
      const int ch = off / kEmitChunk, in = off % kEmitChunk;
      const unsigned m = s_mask[ch];
      slot[j] = prefix + s_chunk[ch] + __popc(m & ((2u << in) - 1u)) - 1;
      orig[j] = perm_final[p];
      hh[j] = s_head[off];
      if (hh[j]) {
        cc[j] = cells[sorted ? p : (int64_t)max(orig[j], 0)];
        if (hh[j] == kHeadSingle) {
#pragma unroll
          for (int l = 0; l <= kMaxD; ++l)
            if (l <= D) xv[j][l] = static_cast<const T *>(a.fin[l])[p];
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kEmitChunk; ++j) {
    if (hh[j] < 0) continue;
    if ((unsigned)orig[j] >= (unsigned)a.n) {
      // a position left unwritten by an earlier failure: never follow it
      internal = true;
      continue;
    }
    if (a.out_index) a.out_index[orig[j]] = (int32_t)slot[j];
    if (!hh[j]) continue;
    a.out_cell[slot[j]] = cc[j];
    if (hh[j] == kHeadSingle) {
      // one-particle set: the particle itself (Step 7)
      for (int l = 0; l < a.dx; ++l) {
        bad |= !isfinite(xv[j][l]);
        static_cast<T *>(a.out_pos[l])[slot[j]] = xv[j][l];
      }
      for (int l = 0; l < a.dp; ++l) {
        bad |= !isfinite(xv[j][a.dx + l]);
        a.out_mom[l][slot[j]] = to_f64<T>(xv[j][a.dx + l]);
      }
      const T w = xv[j][D];
      bad |= !(w > T(0)) || !isfinite(w);
      a.out_w[slot[j]] = to_f64<T>(w);
    } else {
      // merged set: summed below, densely, by the whole CTA
      const int k = atomicAdd(&s_nmerged, 1);
      s_merged[k] = make_int2(j * kEmitThreads + tid, (int)slot[j]);
    }
  }
  __syncthreads();
  // merged sets of this tile: members are the staged positions up to the next
  // head; W, W X and W P are FP64 sums (a product of two floats is exact in
  // FP64)
  for (int k = tid; k < s_nmerged; k += kEmitThreads) {
    const int64_t p = t0 + s_merged[k].x;
    const long long slot = s_merged[k].y;
    double W = 0.0, S1[kMaxD];
#pragma unroll
    for (int l = 0; l < kMaxD; ++l) S1[l] = 0.0;
    for (int64_t r = p; r < a.n; ++r) {
      if (r > p && a.head[r]) break;
      const double w = to_f64<T>(static_cast<const T *>(a.fin[D])[r]);
      W += w;
#pragma unroll
      for (int l = 0; l < kMaxD; ++l)
        if (l < D) S1[l] = fma(w, to_f64<T>(static_cast<const T *>(a.fin[l])[r]), S1[l]);
    }
    const double inv = 1.0 / W;
    a.out_w[slot] = W;
    for (int l = 0; l < a.dx; ++l) static_cast<T *>(a.out_pos[l])[slot] = (T)(S1[l] * inv);
    for (int l = 0; l < a.dp; ++l) a.out_mom[l][slot] = S1[a.dx + l] * inv;
  }
  if (bad) atomicOr(a.err, kErrInput);
  if (internal) atomicOr(a.err, kErrInternal);
}

cudaError_t launch_emit(const EmitArgs &a, cudaStream_t st) {
  if (a.tiles <= 0) return cudaSuccess;
  if (a.mixed)
    emit_kernel<float><<<a.tiles, kEmitThreads, 0, st>>>(a);
  else
    emit_kernel<double><<<a.tiles, kEmitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pma
