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
constexpr int kEmitChunk = 16;  // consecutive positions per chunk
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
  // heads of my chunk of 16 consecutive positions
  const int64_t c0 = t0 + (int64_t)tid * kEmitChunk;
  unsigned mask = 0;
  uint4 hv = make_uint4(0u, 0u, 0u, 0u);
  if (c0 + kEmitChunk <= a.n) {
    hv = *reinterpret_cast<const uint4 *>(a.head + c0);
  } else {
    uint8_t hb[kEmitChunk];
    for (int j = 0; j < kEmitChunk; ++j) hb[j] = (c0 + j < a.n) ? a.head[c0 + j] : (uint8_t)0;
    hv.x = hb[0] | (hb[1] << 8) | (hb[2] << 16) | ((unsigned)hb[3] << 24);
    hv.y = hb[4] | (hb[5] << 8) | (hb[6] << 16) | ((unsigned)hb[7] << 24);
    hv.z = hb[8] | (hb[9] << 8) | (hb[10] << 16) | ((unsigned)hb[11] << 24);
    hv.w = hb[12] | (hb[13] << 8) | (hb[14] << 16) | ((unsigned)hb[15] << 24);
  }
  {
    const unsigned wv[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if ((wv[j >> 2] >> (8 * (j & 3))) & 0xffu) mask |= 1u << j;
    *reinterpret_cast<uint4 *>(s_head + tid * kEmitChunk) = hv;
  }
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
  // staged values, final positions and output slots all advance together
#pragma unroll 4
  for (int j = 0; j < kEmitChunk; ++j) {
    const int off = j * kEmitThreads + tid;
    const int64_t p = t0 + off;
    if (p >= a.n) break;
    const int ch = off / kEmitChunk, in = off % kEmitChunk;
    const unsigned m = s_mask[ch];
    const long long slot = prefix + s_chunk[ch] + __popc(m & ((2u << in) - 1u)) - 1;
    const int orig = perm_final[p];
    if ((unsigned)orig >= (unsigned)a.n) {
      // a position left unwritten by an earlier failure: never follow it
      internal = true;
      continue;
    }
    if (a.out_index) a.out_index[orig] = (int32_t)slot;
    const int h = s_head[off];
    if (!h) continue;
    a.out_cell[slot] = cells[sorted ? p : (int64_t)orig];
    if (h == kHeadSingle) {
      // one-particle set: the particle itself (Step 7)
      for (int l = 0; l < a.dx; ++l) {
        const T x = static_cast<const T *>(a.fin[l])[p];
        bad |= !isfinite(x);
        static_cast<T *>(a.out_pos[l])[slot] = x;
      }
      for (int l = 0; l < a.dp; ++l) {
        const T x = static_cast<const T *>(a.fin[a.dx + l])[p];
        bad |= !isfinite(x);
        a.out_mom[l][slot] = to_f64<T>(x);
      }
      const T w = static_cast<const T *>(a.fin[D])[p];
      bad |= !(w > T(0)) || !isfinite(w);
      a.out_w[slot] = to_f64<T>(w);
    } else {
      // merged set: summed below, densely, by the whole CTA
      const int k = atomicAdd(&s_nmerged, 1);
      s_merged[k] = make_int2(off, (int)slot);
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
