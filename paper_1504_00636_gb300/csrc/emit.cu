// Step 7: replace every final set by its centroid, compacted in canonical
// order.  The final sets of all cells are contiguous position ranges marked by
// a head byte at their first position (1 for a single particle, the set's size
// for a merged set); cells are laid out in ascending order and the sets of a
// cell in V1-first depth-first order, so the output slot of a set is the
// number of heads before it.  The partition kernels staged every particle's
// coordinates and weight at its final position, so this step streams:
//   count_kernel   heads per tile of 1024 positions
//   tiles_kernel   exclusive prefix over tiles (one CTA) and the count M
//   emit_kernel    per tile: slots, merged particles, input -> output index;
//                  a merged set's centroid (W, X, P) is an FP64 sum over its
//                  staged members (a product of two floats is exact in FP64)
#include "lookback.cuh"
#include "pma_launch.h"

namespace pma {

constexpr int kEmitThreads = 256;
constexpr int kEmitChunk = 4;  // consecutive positions per thread
constexpr int kEmitTile = kEmitThreads * kEmitChunk;
constexpr int kScanCta = 1024;

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

// head bytes of my 4 consecutive positions
__device__ __forceinline__ unsigned load_heads(const uint8_t *head, int64_t c0, int64_t n) {
  unsigned hw = 0;
  if (c0 + kEmitChunk <= n) {
    hw = *reinterpret_cast<const unsigned *>(head + c0);
  } else {
    for (int j = 0; j < kEmitChunk; ++j)
      if (c0 + j < n) hw |= (unsigned)head[c0 + j] << (8 * j);
  }
  return hw;
}

__device__ __forceinline__ unsigned head_mask(unsigned hw) {
  unsigned mask = 0;
#pragma unroll
  for (int j = 0; j < kEmitChunk; ++j)
    if ((hw >> (8 * j)) & 0xffu) mask |= 1u << j;
  return mask;
}

__global__ void __launch_bounds__(kEmitThreads) count_kernel(EmitArgs a) {
  __shared__ int s_warp[32];
  const int64_t c0 = (int64_t)blockIdx.x * kEmitTile + (int64_t)threadIdx.x * kEmitChunk;
  int v = __popc(head_mask(load_heads(a.head, c0, a.n)));
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < kEmitThreads / 32; ++k) t += s_warp[k];
    a.tile_count[blockIdx.x] = t;
  }
}

// one CTA: exclusive prefix of the tile counts, and the total M
__global__ void __launch_bounds__(kScanCta) tiles_kernel(EmitArgs a) {
  __shared__ int s_warp[32];
  __shared__ long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < a.tiles; base += kScanCta) {
    const int i = base + threadIdx.x;
    const int v = i < a.tiles ? a.tile_count[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, s_warp, &total);
    if (i < a.tiles) a.tile_prefix[i] = s_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (a.out_count) *a.out_count = s_carry;
    if (a.out_count2) *a.out_count2 = s_carry;
  }
}

template <typename T>
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(EmitArgs a) {
  __shared__ int s_warp[32];
  __shared__ unsigned short s_mask[kEmitThreads];
  __shared__ int s_chunk[kEmitThreads];
  __shared__ __align__(16) uint8_t s_head[kEmitTile];
  __shared__ int s_nmerged;
  __shared__ int2 s_merged[kEmitTile / 2 + 1];  // (offset in tile, output slot)
  const int tid = threadIdx.x;
  if (tid == 0) s_nmerged = 0;
  const int64_t t0 = (int64_t)blockIdx.x * kEmitTile;
  const unsigned hw = load_heads(a.head, t0 + (int64_t)tid * kEmitChunk, a.n);
  const unsigned mask = head_mask(hw);
  reinterpret_cast<unsigned *>(s_head)[tid] = hw;
  int total;
  const int ex = block_exclusive_scan(__popc(mask), s_warp, &total);
  s_mask[tid] = (unsigned short)mask;
  s_chunk[tid] = ex;
  __syncthreads();
  const long long prefix = a.tile_prefix[blockIdx.x];
  const int32_t *__restrict__ perm_final = a.perm_final;
  const int32_t *__restrict__ cells = a.cells;
  const bool sorted = *a.unsorted == 0;
  const int D = a.dx + a.dp;
  bool bad = false, internal = false;
  // positions in strided order (consecutive threads, consecutive positions);
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
  for (int k = tid; k < s_nmerged; k += kEmitThreads) {
    const int64_t p = t0 + s_merged[k].x;
    const long long slot_m = s_merged[k].y;
    const int h = s_head[s_merged[k].x];
    // members: the head's count, or (255) every position up to the next head
    int64_t e = p + h;
    if (h == kHeadLong) {
      e = p + 1;
      while (e < a.n && a.head[e] == 0) ++e;
    }
    if (e > a.n) {
      internal = true;
      e = a.n;
    }
    double W = 0.0, S1[kMaxD];
#pragma unroll
    for (int l = 0; l < kMaxD; ++l) S1[l] = 0.0;
    for (int64_t r = p; r < e; ++r) {
      const double w = to_f64<T>(static_cast<const T *>(a.fin[D])[r]);
      W += w;
#pragma unroll
      for (int l = 0; l < kMaxD; ++l)
        if (l < D) S1[l] = fma(w, to_f64<T>(static_cast<const T *>(a.fin[l])[r]), S1[l]);
    }
    const double inv = 1.0 / W;
    a.out_w[slot_m] = W;
    for (int l = 0; l < a.dx; ++l) static_cast<T *>(a.out_pos[l])[slot_m] = (T)(S1[l] * inv);
    for (int l = 0; l < a.dp; ++l) a.out_mom[l][slot_m] = S1[a.dx + l] * inv;
  }
  if (bad) atomicOr(a.err, kErrInput);
  if (internal) atomicOr(a.err, kErrInternal);
}

cudaError_t launch_emit(const EmitArgs &a, cudaStream_t st) {
  if (a.tiles <= 0) return cudaSuccess;
  count_kernel<<<a.tiles, kEmitThreads, 0, st>>>(a);
  tiles_kernel<<<1, kScanCta, 0, st>>>(a);
  if (a.mixed)
    emit_kernel<float><<<a.tiles, kEmitThreads, 0, st>>>(a);
  else
    emit_kernel<double><<<a.tiles, kEmitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pma
