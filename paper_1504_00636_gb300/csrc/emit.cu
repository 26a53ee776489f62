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
  if (tid == 0) {
    const long long pre = tile_exclusive_prefix(a.scan_status, tile, total, a.err);
    s_prefix = pre;
    if (tile == a.tiles - 1) {
      if (a.out_count) *a.out_count = pre + total;
      if (a.out_count2) *a.out_count2 = pre + total;
    }
  }
  __syncthreads();
  const long long prefix = s_prefix;
  const int32_t *__restrict__ perm_final = a.perm_final;
  const int32_t *__restrict__ cells = a.cells;
  const T *__restrict__ win = static_cast<const T *>(a.w);
  bool bad = false, internal = false;
  // positions in strided order (consecutive threads, consecutive positions),
  // in batches whose loads are issued before their stores
  constexpr int kB = 4;
  for (int jb = 0; jb < kEmitChunk; jb += kB) {
    int orig[kB], hh[kB];
    long long slot[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int off = (jb + u) * kEmitThreads + tid;
      const int64_t p = t0 + off;
      orig[u] = -1;
      hh[u] = 0;
      slot[u] = 0;
      if (p < a.n) {
        const int ch = off / kEmitChunk, in = off % kEmitChunk;
        const unsigned m = s_mask[ch];
        slot[u] = prefix + s_chunk[ch] + __popc(m & ((2u << in) - 1u)) - 1;
        orig[u] = perm_final[p];
        hh[u] = s_head[off];
        if ((unsigned)orig[u] >= (unsigned)a.n) {
          // a position left unwritten by an earlier failure: never follow it
          internal = true;
          orig[u] = -1;
          hh[u] = 0;
        }
      }
    }
    T xs[kB][kMaxD];
    T ws[kB];
    int cs[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      cs[u] = 0;
      ws[u] = T(1);
#pragma unroll
      for (int l = 0; l < kMaxD; ++l) xs[u][l] = T(0);
      if (hh[u]) cs[u] = cells[orig[u]];
      if (hh[u] == kHeadSingle) {
#pragma unroll
        for (int l = 0; l < kMaxD; ++l)
          if (l < a.dx + a.dp) xs[u][l] = static_cast<const T *>(a.q[l])[orig[u]];
        ws[u] = win[orig[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      if (orig[u] < 0) continue;
      if (a.out_index) a.out_index[orig[u]] = (int32_t)slot[u];
      if (!hh[u]) continue;
      a.out_cell[slot[u]] = cs[u];
      if (hh[u] == kHeadSingle) {
        // one-particle set: the particle itself (Step 7)
        for (int l = 0; l < a.dx; ++l) {
          bad |= !isfinite(xs[u][l]);
          static_cast<T *>(a.out_pos[l])[slot[u]] = xs[u][l];
        }
        for (int l = 0; l < a.dp; ++l) {
          bad |= !isfinite(xs[u][a.dx + l]);
          a.out_mom[l][slot[u]] = to_f64<T>(xs[u][a.dx + l]);
        }
        bad |= !(ws[u] > T(0)) || !isfinite(ws[u]);
        a.out_w[slot[u]] = to_f64<T>(ws[u]);
      } else {
        // merged set: summed below, densely, by the whole CTA
        const int k = atomicAdd(&s_nmerged, 1);
        s_merged[k] = make_int2((jb + u) * kEmitThreads + tid, (int)slot[u]);
      }
    }
  }
  __syncthreads();
  // merged sets of this tile: members are the positions up to the next head;
  // W, W X and W P are FP64 sums (a product of two floats is exact in FP64)
  const int D = a.dx + a.dp;
  for (int k = tid; k < s_nmerged; k += kEmitThreads) {
    const int64_t p = t0 + s_merged[k].x;
    const long long slot = s_merged[k].y;
    double W = 0.0, S1[kMaxD];
#pragma unroll
    for (int l = 0; l < kMaxD; ++l) S1[l] = 0.0;
    for (int64_t r = p; r < a.n; ++r) {
      if (r > p && a.head[r]) break;
      const int o = perm_final[r];
      if ((unsigned)o >= (unsigned)a.n) {
        internal = true;
        break;
      }
      const double w = to_f64<T>(win[o]);
      W += w;
#pragma unroll
      for (int l = 0; l < kMaxD; ++l)
        if (l < D) S1[l] = fma(w, to_f64<T>(static_cast<const T *>(a.q[l])[o]), S1[l]);
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
