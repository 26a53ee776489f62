// Warp-per-cell partition (Sec. 3, Steps 2-7 for cells of at most cap_w
// particles, and the verbatim copy of cells with N <= N_min).
//
// Each warp owns one cell at a time; the warps of a CTA never wait for each
// other.  The cell's coordinates and weights are staged once in the warp's
// slice of shared memory (SoA columns) and stay in place; a subset is a
// contiguous range of a 16-bit index array, and a cut writes V1 = {q_k <= Q_k}
// to the front and V2 to the back of the same range in the other index array
// (double-buffered by tree depth).  Leaves therefore come out in V1-first
// depth-first order when listed by position.
//   subsets of more than kSmall particles: the whole warp, depth-first
//     (moments by lane-strided sums and a butterfly, cut by ballot scan);
//   subsets of at most kSmall particles: collected 32 at a time and finished
//     by one lane each, depth-first.
#include "pma_device.cuh"
#include "pma_launch.h"
#include "split_common.cuh"

namespace pma {

constexpr int kWarpChunk = 2;  // cells taken per work-counter increment

template <typename T, int D>
struct WarpTile {
  T *data;           // [D + 1][cap]: coordinates, then weight
  uint16_t *idx[2];  // index arrays, by depth parity
  Item *small;       // [64] pending small subsets
  Item *stack;       // [cap / kSmall + 2] pending large subsets
  int cap;
  __device__ __forceinline__ T *col(int l) const { return data + (size_t)l * cap; }
};

template <typename T, int D>
__host__ __device__ inline size_t warp_region_bytes(int cap) {
  size_t b = (size_t)(D + 1) * cap * sizeof(T) + (size_t)2 * cap * sizeof(uint16_t);
  b = (b + 15) & ~size_t(15);
  b += (size_t)(64 + cap / kSmall + 2) * sizeof(Item);
  return (b + 15) & ~size_t(15);
}

// ------------------------------------------------------------ leaf output

// final set [b, e) of index buffer `par`: permutation, head bytes and, for a
// merged set, its centroid record (one warp)
template <typename T, int D>
__device__ void warp_emit(const Problem &P, const WarpTile<T, D> &S, const int32_t *perm,
                          int64_t gb, int b, int e, int par, const Moments<T, D> &M, const T *s,
                          int lane) {
  const uint8_t h = (e - b == 1) ? kHeadSingle : kHeadMerged;
  for (int i = b + lane; i < e; i += 32) {
    P.perm_final[gb + i] = orig_index(perm, gb, S.idx[par][i]);
    P.head[gb + i] = (i == b) ? h : (uint8_t)0;
  }
  if (e - b == 1) return;
  const int64_t hp = gb + b;
  if constexpr (sizeof(T) == 8) {
    if (lane == 0) record_from_moments<D>(P, hp, M, s);
  } else {
    double W = 0.0, S1[D];
#pragma unroll
    for (int l = 0; l < D; ++l) S1[l] = 0.0;
    for (int i = b + lane; i < e; i += 32) {
      const int j = S.idx[par][i];
      const double w = f2d_exact(S.col(D)[j]);
      W += w;
#pragma unroll
      for (int l = 0; l < D; ++l) S1[l] = fma(w, f2d_exact(S.col(l)[j]), S1[l]);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      W += __shfl_xor_sync(0xffffffffu, W, m);
#pragma unroll
      for (int l = 0; l < D; ++l) S1[l] += __shfl_xor_sync(0xffffffffu, S1[l], m);
    }
    if (lane == 0) {
      P.rec_w[hp] = W;
#pragma unroll
      for (int l = 0; l < D; ++l) P.rec_c[l * P.stride + hp] = S1[l] / W;
    }
  }
}

// same, by one lane
template <typename T, int D>
__device__ void lane_emit(const Problem &P, const WarpTile<T, D> &S, const int32_t *perm,
                          int64_t gb, int b, int e, int par, const Moments<T, D> &M, const T *s) {
  const uint8_t h = (e - b == 1) ? kHeadSingle : kHeadMerged;
  for (int i = b; i < e; ++i) {
    P.perm_final[gb + i] = orig_index(perm, gb, S.idx[par][i]);
    P.head[gb + i] = (i == b) ? h : (uint8_t)0;
  }
  if (e - b == 1) return;
  const int64_t hp = gb + b;
  if constexpr (sizeof(T) == 8) {
    record_from_moments<D>(P, hp, M, s);
  } else {
    double W = 0.0, S1[D];
#pragma unroll
    for (int l = 0; l < D; ++l) S1[l] = 0.0;
    for (int i = b; i < e; ++i) {
      const int j = S.idx[par][i];
      const double w = f2d_exact(S.col(D)[j]);
      W += w;
#pragma unroll
      for (int l = 0; l < D; ++l) S1[l] = fma(w, f2d_exact(S.col(l)[j]), S1[l]);
    }
    P.rec_w[hp] = W;
#pragma unroll
    for (int l = 0; l < D; ++l) P.rec_c[l * P.stride + hp] = S1[l] / W;
  }
}

// ------------------------------------------------- large subsets (warp)

struct Counters {
  unsigned long long leaves, depth, splits, degenerate;
};

// Steps 2-6 on one subset by the whole warp.  Returns the number of children
// written to ch (0 when the subset is final).
template <typename T, int D>
__device__ int warp_cut(const Problem &P, const WarpTile<T, D> &S, const int32_t *perm,
                        int64_t gb, Item it, Item *ch, Counters &cnt, int lane) {
  const int b = it.b, e = it.e, par = it.par;
  T s[D];
  {
    const int j0 = S.idx[par][b];
#pragma unroll
    for (int l = 0; l < D; ++l) s[l] = S.col(l)[j0];
  }
  Moments<T, D> M;
  M.zero();
  for (int i = b + lane; i < e; i += 32) {
    const int j = S.idx[par][i];
    T q[D];
#pragma unroll
    for (int l = 0; l < D; ++l) q[l] = S.col(l)[j];
    M.add(S.col(D)[j], q, s);
  }
  M.warp_allreduce();
  const Cut c = Decider<T, D>::run(P, M, s);
  if (c.leaf) {
    warp_emit<T, D>(P, S, perm, gb, b, e, par, M, s, lane);
    if (lane == 0) {
      cnt.leaves += 1;
      cnt.depth += (unsigned long long)it.depth * (e - b);
    }
    return 0;
  }
  const int np = par ^ 1;
  const T *qk = S.col(c.k);
  const unsigned lt = lanemask_lt();
  int cntL = 0, cntR = 0;
  for (int base = b; base < e; base += 32) {
    const int i = base + lane;
    const bool valid = i < e;
    const int j = valid ? S.idx[par][i] : 0;
    const bool lft = valid && Decider<T, D>::left(qk[j], c);
    const unsigned bl = __ballot_sync(0xffffffffu, lft);
    const unsigned br = __ballot_sync(0xffffffffu, valid && !lft);
    if (valid) {
      const int dst = lft ? (b + cntL + __popc(bl & lt)) : (e - 1 - cntR - __popc(br & lt));
      S.idx[np][dst] = (uint16_t)j;
    }
    cntL += __popc(bl);
    cntR += __popc(br);
  }
  __syncwarp();
  if (cntL == 0 || cntR == 0) {
    // the rounded centroid lies beyond an extreme value: the set stays whole
    warp_emit<T, D>(P, S, perm, gb, b, e, np, M, s, lane);
    if (lane == 0) {
      cnt.leaves += 1;
      cnt.degenerate += 1;
      cnt.depth += (unsigned long long)it.depth * (e - b);
    }
    return 0;
  }
  if (lane == 0) cnt.splits += 1;
  const uint8_t d1 = (uint8_t)(it.depth + 1);
  ch[0] = Item{(uint16_t)b, (uint16_t)(b + cntL), (uint8_t)np, d1, 0};
  ch[1] = Item{(uint16_t)(b + cntL), (uint16_t)e, (uint8_t)np, d1, 0};
  return 2;
}

// ------------------------------------------------ small subsets (lane)

template <typename T, int D>
__device__ void lane_finish(const Problem &P, const WarpTile<T, D> &S, const int32_t *perm,
                            int64_t gb, Item root, Counters &cnt) {
  Item stk[kSmall + 2];
  int sp = 0;
  stk[sp++] = root;
  while (sp > 0) {
    const Item it = stk[--sp];
    const int b = it.b, e = it.e, par = it.par;
    if (e - b == 1) {
      P.perm_final[gb + b] = orig_index(perm, gb, S.idx[par][b]);
      P.head[gb + b] = kHeadSingle;
      cnt.leaves += 1;
      cnt.depth += it.depth;
      continue;
    }
    T s[D];
    {
      const int j0 = S.idx[par][b];
#pragma unroll
      for (int l = 0; l < D; ++l) s[l] = S.col(l)[j0];
    }
    Moments<T, D> M;
    M.zero();
    for (int i = b; i < e; ++i) {
      const int j = S.idx[par][i];
      T q[D];
#pragma unroll
      for (int l = 0; l < D; ++l) q[l] = S.col(l)[j];
      M.add(S.col(D)[j], q, s);
    }
    const Cut c = Decider<T, D>::run(P, M, s);
    if (c.leaf) {
      lane_emit<T, D>(P, S, perm, gb, b, e, par, M, s);
      cnt.leaves += 1;
      cnt.depth += (unsigned long long)it.depth * (e - b);
      continue;
    }
    const int np = par ^ 1;
    const T *qk = S.col(c.k);
    int cntL = 0, cntR = 0;
    for (int i = b; i < e; ++i) {
      const int j = S.idx[par][i];
      const bool lft = Decider<T, D>::left(qk[j], c);
      const int dst = lft ? (b + cntL++) : (e - 1 - cntR++);
      S.idx[np][dst] = (uint16_t)j;
    }
    if (cntL == 0 || cntR == 0) {
      lane_emit<T, D>(P, S, perm, gb, b, e, np, M, s);
      cnt.leaves += 1;
      cnt.degenerate += 1;
      cnt.depth += (unsigned long long)it.depth * (e - b);
      continue;
    }
    cnt.splits += 1;
    if (sp + 2 > kSmall + 2) {
      set_error(P.err, kErrInternal);
      return;
    }
    const uint8_t d1 = (uint8_t)(it.depth + 1);
    stk[sp++] = Item{(uint16_t)(b + cntL), (uint16_t)e, (uint8_t)np, d1, 0};
    stk[sp++] = Item{(uint16_t)b, (uint16_t)(b + cntL), (uint8_t)np, d1, 0};
  }
}

// --------------------------------------------------------------- kernel

template <typename T, int D>
__global__ void __launch_bounds__(128) warp_kernel(Problem P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cap = P.cap_w;
  WarpTile<T, D> S;
  {
    unsigned char *base = smem_raw + (size_t)warp * warp_region_bytes<T, D>(cap);
    S.data = reinterpret_cast<T *>(base);
    S.idx[0] = reinterpret_cast<uint16_t *>(S.data + (size_t)(D + 1) * cap);
    S.idx[1] = S.idx[0] + cap;
    size_t off = ((size_t)(D + 1) * cap * sizeof(T) + (size_t)2 * cap * sizeof(uint16_t) + 15) &
                 ~size_t(15);
    S.small = reinterpret_cast<Item *>(base + off);
    S.stack = S.small + 64;
    S.cap = cap;
  }
  const int max_stack = cap / kSmall + 2;
  const int32_t *perm = (*P.unsorted == 0) ? nullptr : P.perm;
  const int count = *P.warp_count;
  Counters cnt{0ull, 0ull, 0ull, 0ull};
  unsigned long long merged = 0, passed = 0;

  for (;;) {
    int c0 = 0;
    if (lane == 0) c0 = atomicAdd(P.warp_next, kWarpChunk);
    c0 = __shfl_sync(0xffffffffu, c0, 0);
    if (c0 >= count) break;
    const int c1 = min(c0 + kWarpChunk, count);
    for (int t = c0; t < c1; ++t) {
      const int cell = P.warp_list[t];
      const int64_t gb = P.cell_begin[cell];
      const int n = P.cell_begin[cell + 1] - (int)gb;
      if (n <= P.n_min || n == 1) {
        // Sec. 3 "Input": cells with at most N_min particles are not merged
        for (int i = lane; i < n; i += 32) {
          P.perm_final[gb + i] = orig_index(perm, gb, i);
          P.head[gb + i] = kHeadSingle;
        }
        passed += 1;
        continue;
      }
      merged += 1;
      bool bad = false;
      for (int i = lane; i < n; i += 32) {
        const int src = orig_index(perm, gb, i);
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const T x = StoreOf<T>::load(P.q[l], src);
          bad |= !finite_val(x);
          S.col(l)[i] = x;
        }
        const T w = StoreOf<T>::load(P.w, src);
        bad |= !(w > T(0)) || !finite_val(w);
        S.col(D)[i] = w;
        S.idx[0][i] = (uint16_t)i;
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(P.err, kErrInput);
      __syncwarp();
      const Item root{0, (uint16_t)n, 0, 0, 0};
      int sp = 0, ns = 0;
      if (n <= kSmall) {
        if (lane == 0) S.small[0] = root;
        ns = 1;
      } else {
        if (lane == 0) S.stack[0] = root;
        sp = 1;
      }
      __syncwarp();
      for (;;) {
        if (ns >= 32 || (sp == 0 && ns > 0)) {
          // one round of small subsets, one per lane
          const int take = min(ns, 32);
          if (lane < take) lane_finish<T, D>(P, S, perm, gb, S.small[lane], cnt);
          __syncwarp();
          if (lane == 0)
            for (int k = take; k < ns; ++k) S.small[k - take] = S.small[k];
          ns -= take;
          __syncwarp();
          continue;
        }
        if (sp == 0) break;
        const Item it = S.stack[--sp];
        Item ch[2];
        const int nch = warp_cut<T, D>(P, S, perm, gb, it, ch, cnt, lane);
        for (int h = 0; h < nch; ++h) {
          const int m = ch[h].e - ch[h].b;
          if (m == 1) {
            if (lane == 0) {
              P.perm_final[gb + ch[h].b] = orig_index(perm, gb, S.idx[ch[h].par][ch[h].b]);
              P.head[gb + ch[h].b] = kHeadSingle;
              cnt.leaves += 1;
              cnt.depth += ch[h].depth;
            }
          } else if (m <= kSmall) {
            if (lane == 0) S.small[ns] = ch[h];
            ++ns;
          } else if (sp < max_stack) {
            if (lane == 0) S.stack[sp] = ch[h];
            ++sp;
          } else {
            if (lane == 0) set_error(P.err, kErrInternal);
          }
        }
        __syncwarp();
      }
    }
  }
  // counters: lane-level work is spread over the lanes, warp-level work
  // was counted by lane 0 only
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    cnt.leaves += __shfl_xor_sync(0xffffffffu, cnt.leaves, m);
    cnt.depth += __shfl_xor_sync(0xffffffffu, cnt.depth, m);
    cnt.splits += __shfl_xor_sync(0xffffffffu, cnt.splits, m);
    cnt.degenerate += __shfl_xor_sync(0xffffffffu, cnt.degenerate, m);
  }
  if (lane == 0) {
    if (cnt.leaves) atomicAdd(&P.stats[kStLeaves], cnt.leaves);
    if (cnt.depth) atomicAdd(&P.stats[kStDepth], cnt.depth);
    if (cnt.splits) atomicAdd(&P.stats[kStSplits], cnt.splits);
    if (cnt.degenerate) atomicAdd(&P.stats[kStDegenerate], cnt.degenerate);
    if (merged) atomicAdd(&P.stats[kStCellsMerged], merged);
    if (passed) atomicAdd(&P.stats[kStCellsPass], passed);
  }
}

// ----------------------------------------------------------------- launch

template <typename T>
static size_t warp_smem_t(int D, int cap) {
  switch (D) {
    case 2: return warp_region_bytes<T, 2>(cap);
    case 3: return warp_region_bytes<T, 3>(cap);
    case 4: return warp_region_bytes<T, 4>(cap);
    case 5: return warp_region_bytes<T, 5>(cap);
    default: return warp_region_bytes<T, 6>(cap);
  }
}

size_t warp_smem(int mixed, int D, int cap_w) {
  return mixed ? warp_smem_t<float>(D, cap_w) : warp_smem_t<double>(D, cap_w);
}

template <typename T, int D>
static cudaError_t launch_warps_t(const Problem &P, int wpc, int grid, cudaStream_t st) {
  const size_t smem = (size_t)wpc * warp_region_bytes<T, D>(P.cap_w);
  cudaError_t e = cudaFuncSetAttribute(warp_kernel<T, D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  warp_kernel<T, D><<<grid, 32 * wpc, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_warps(const Problem &P, int mixed, int wpc, int grid, cudaStream_t st) {
  if (mixed) {
    switch (P.D) {
      case 2: return launch_warps_t<float, 2>(P, wpc, grid, st);
      case 3: return launch_warps_t<float, 3>(P, wpc, grid, st);
      case 4: return launch_warps_t<float, 4>(P, wpc, grid, st);
      case 5: return launch_warps_t<float, 5>(P, wpc, grid, st);
      default: return launch_warps_t<float, 6>(P, wpc, grid, st);
    }
  }
  switch (P.D) {
    case 2: return launch_warps_t<double, 2>(P, wpc, grid, st);
    case 3: return launch_warps_t<double, 3>(P, wpc, grid, st);
    case 4: return launch_warps_t<double, 4>(P, wpc, grid, st);
    case 5: return launch_warps_t<double, 5>(P, wpc, grid, st);
    default: return launch_warps_t<double, 6>(P, wpc, grid, st);
  }
}

}  // namespace pma
