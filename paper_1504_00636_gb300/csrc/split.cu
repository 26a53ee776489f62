// cluster_kernel: cells larger than any shared-memory tile are cut (Sec. 3,
// Steps 2-6) by a thread-block cluster in global memory, on the permutation
// array only, until every piece fits; the pieces then go through the team
// kernel (warp.cu).  Final sets met on the way are emitted here.
//
// The CTA-per-cell building blocks below (a double-buffered shared-memory
// tile, warp-level cuts of large subsets, thread-level depth-first finishing
// of small ones) serve the allocation-free entry point at the end of this
// file.
#include <cooperative_groups.h>

#include <cstddef>
#include <mutex>

#include "lookback.cuh"
#include "pma.h"
#include "pma_device.cuh"
#include "pma_launch.h"
#include "split_common.cuh"

namespace pma {

// ---------------------------------------------------------- shared layout

template <typename T, int D>
struct Tile {
  T *base;
  uint16_t *id[2];
  int cap;
  __device__ __forceinline__ T *col(int par, int l) const {
    return base + (size_t)(par * (D + 1) + l) * cap;
  }
};

// particle j of buffer `par`, staged at final position gp (when staging is on)
template <typename T, int D>
__device__ __forceinline__ void stage_tile(const Problem &P, const Tile<T, D> &S, int par,
                                           int64_t gp, int j) {
  if (!P.fin[0]) return;
#pragma unroll
  for (int l = 0; l <= D; ++l) static_cast<T *>(P.fin[l])[gp] = S.col(par, l)[j];
}

// input particle src, staged at final position gp (when staging is on)
template <typename T, int D>
__device__ __forceinline__ void stage_global(const Problem &P, int64_t gp, int src) {
  if (!P.fin[0]) return;
#pragma unroll
  for (int l = 0; l < D; ++l) static_cast<T *>(P.fin[l])[gp] = StoreOf<T>::load(P.q[l], src);
  static_cast<T *>(P.fin[D])[gp] = StoreOf<T>::load(P.w, src);
}

template <typename T, int D>
__host__ __device__ inline size_t unit_smem_bytes(int cap) {
  size_t v = (size_t)2 * (D + 1) * cap * sizeof(T);
  size_t ids = (size_t)2 * cap * sizeof(uint16_t);
  size_t lists = (size_t)(2 * (cap / kSmall + 2) + (cap / 2 + 2)) * sizeof(Item);
  return v + ids + lists;
}

// ------------------------------------------------------- leaf emission

// final set [b, e) of buffer `par`, by one warp: permutation and head
// bytes (the emit kernel sums merged sets up)
template <typename T, int D>
__device__ void emit_leaf_warp(const Problem &P, const Tile<T, D> &S, const int32_t *perm,
                               int64_t gb, int b, int e, int par, const Moments<T, D> &M,
                               const T *s, int lane) {
  const uint8_t h = head_code(e - b);
  for (int j = b + lane; j < e; j += 32) {
    P.perm_final[gb + j] = orig_index(perm, gb, S.id[par][j]);
    P.head[gb + j] = (j == b) ? h : (uint8_t)0;
    stage_tile<T, D>(P, S, par, gb + j, j);
  }
}

// same, by one thread
template <typename T, int D>
__device__ void emit_leaf_thread(const Problem &P, const Tile<T, D> &S, const int32_t *perm,
                                 int64_t gb, int b, int e, int par, const Moments<T, D> &M,
                                 const T *s) {
  const uint8_t h = head_code(e - b);
  for (int j = b; j < e; ++j) {
    P.perm_final[gb + j] = orig_index(perm, gb, S.id[par][j]);
    P.head[gb + j] = (j == b) ? h : (uint8_t)0;
    stage_tile<T, D>(P, S, par, gb + j, j);
  }
}

// --------------------------------------------------------------- phase A

template <typename T, int D>
__device__ void warp_split(const Problem &P, const Tile<T, D> &S, const int32_t *perm,
                           int64_t gb, Item it, Item *nxt, int *n_nxt, int max_nxt,
                           Item *small, int *n_small, unsigned long long *st, int lane) {
  const int b = it.b, e = it.e, par = it.par;
  T s[D];
#pragma unroll
  for (int l = 0; l < D; ++l) s[l] = S.col(par, l)[b];
  Moments<T, D> M;
  M.zero();
  for (int i = b + lane; i < e; i += 32) {
    T q[D];
#pragma unroll
    for (int l = 0; l < D; ++l) q[l] = S.col(par, l)[i];
    M.add(S.col(par, D)[i], q, s);
  }
  M.warp_allreduce();
  Cut c = Decider<T, D>::run(P, M, s, e - b, (e - b + 31) / 32);
  // FP32 storage: a decision or a cut too close to call is taken again with
  // FP64 sums of the set (warp-uniform: every lane holds the same sums)
  bool exact = sizeof(T) == 8;
  const int np = par ^ 1;
  int cntL = 0, cntR = 0;
  for (;;) {
    if (c.unsure) {
      Moments<double, D> X;
      X.zero();
      for (int i = b + lane; i < e; i += 32) {
        T q[D];
#pragma unroll
        for (int l = 0; l < D; ++l) q[l] = S.col(par, l)[i];
        add_exact<T, D>(X, S.col(par, D)[i], q, s);
      }
      X.warp_allreduce();
      c = decide_exact<T, D, true>(P, X, s, e - b);
      exact = true;
    }
    if (c.leaf) break;
    const T *qk = S.col(par, c.k);
    cntL = cntR = 0;
    bool nr = false;
    const unsigned lt = lanemask_lt();
    for (int base = b; base < e; base += 32) {
      int i = base + lane;
      bool valid = i < e;
      const T q = qk[valid ? i : b];
      bool lft = valid && Decider<T, D>::left(q, c);
      nr |= valid && Decider<T, D>::near(q, c);
      unsigned bl = __ballot_sync(0xffffffffu, lft);
      unsigned br = __ballot_sync(0xffffffffu, valid && !lft);
      if (valid) {
        int dst = lft ? (b + cntL + __popc(bl & lt)) : (e - 1 - cntR - __popc(br & lt));
#pragma unroll
        for (int l = 0; l <= D; ++l) S.col(np, l)[dst] = S.col(par, l)[i];
        S.id[np][dst] = S.id[par][i];
      }
      cntL += __popc(bl);
      cntR += __popc(br);
    }
    if (__any_sync(0xffffffffu, nr) && !exact) {
      c.unsure = 1;
      continue;
    }
    break;
  }
  if (c.leaf) {
    emit_leaf_warp<T, D>(P, S, perm, gb, b, e, par, M, s, lane);
    if (lane == 0) {
      atomicAdd(&st[kStLeaves], 1ull);
      atomicAdd(&st[kStDepth], (unsigned long long)it.depth * (e - b));
    }
    return;
  }
  __syncwarp();
  if (cntL == 0 || cntR == 0) {
    // rounded centroid beyond an extreme value: the set stays whole
    emit_leaf_warp<T, D>(P, S, perm, gb, b, e, np, M, s, lane);
    if (lane == 0) {
      atomicAdd(&st[kStLeaves], 1ull);
      atomicAdd(&st[kStDegenerate], 1ull);
      atomicAdd(&st[kStDepth], (unsigned long long)it.depth * (e - b));
    }
    return;
  }
  if (lane == 0) {
    atomicAdd(&st[kStSplits], 1ull);
    Item ch[2] = {{(uint16_t)b, (uint16_t)(b + cntL), (uint8_t)np, (uint8_t)(it.depth + 1), 0},
                  {(uint16_t)(b + cntL), (uint16_t)e, (uint8_t)np, (uint8_t)(it.depth + 1), 0}};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int n = ch[h].e - ch[h].b;
      if (n == 1) {
        P.perm_final[gb + ch[h].b] = orig_index(perm, gb, S.id[np][ch[h].b]);
        P.head[gb + ch[h].b] = kHeadSingle;
        stage_tile<T, D>(P, S, np, gb + ch[h].b, ch[h].b);
        atomicAdd(&st[kStLeaves], 1ull);
        atomicAdd(&st[kStDepth], (unsigned long long)ch[h].depth);
      } else if (n <= kSmall) {
        small[atomicAdd(n_small, 1)] = ch[h];
      } else {
        int slot = atomicAdd(n_nxt, 1);
        if (slot < max_nxt)
          nxt[slot] = ch[h];
        else
          set_error(P.err, kErrInternal);
      }
    }
  }
}

// --------------------------------------------------------------- phase B

template <typename T, int D>
__device__ void thread_finish(const Problem &P, const Tile<T, D> &S, const int32_t *perm,
                              int64_t gb, Item root, unsigned long long *cnt) {
  Item stk[kSmall + 2];
  int sp = 0;
  stk[sp++] = root;
  while (sp > 0) {
    Item it = stk[--sp];
    const int b = it.b, e = it.e, par = it.par;
    if (e - b == 1) {
      P.perm_final[gb + b] = orig_index(perm, gb, S.id[par][b]);
      P.head[gb + b] = kHeadSingle;
      stage_tile<T, D>(P, S, par, gb + b, b);
      cnt[0] += 1;
      cnt[1] += it.depth;
      continue;
    }
    T s[D];
#pragma unroll
    for (int l = 0; l < D; ++l) s[l] = S.col(par, l)[b];
    Moments<T, D> M;
    M.zero();
    for (int i = b; i < e; ++i) {
      T q[D];
#pragma unroll
      for (int l = 0; l < D; ++l) q[l] = S.col(par, l)[i];
      M.add(S.col(par, D)[i], q, s);
    }
    Cut c = Decider<T, D>::run(P, M, s, e - b, e - b);
    // FP32 storage: a decision or a cut too close to call is taken again
    // with FP64 sums of the set
    bool exact = sizeof(T) == 8;
    const int np = par ^ 1;
    int cntL = 0, cntR = 0;
    for (;;) {
      if (c.unsure) {
        Moments<double, D> X;
        X.zero();
        for (int i = b; i < e; ++i) {
          T q[D];
#pragma unroll
          for (int l = 0; l < D; ++l) q[l] = S.col(par, l)[i];
          add_exact<T, D>(X, S.col(par, D)[i], q, s);
        }
        c = decide_exact<T, D, true>(P, X, s, e - b);
        exact = true;
      }
      if (c.leaf) break;
      const T *qk = S.col(par, c.k);
      cntL = cntR = 0;
      bool nr = false;
      for (int i = b; i < e; ++i) {
        const T q = qk[i];
        bool lft = Decider<T, D>::left(q, c);
        nr |= Decider<T, D>::near(q, c);
        int dst = lft ? (b + cntL++) : (e - 1 - cntR++);
#pragma unroll
        for (int l = 0; l <= D; ++l) S.col(np, l)[dst] = S.col(par, l)[i];
        S.id[np][dst] = S.id[par][i];
      }
      if (nr && !exact) {
        c.unsure = 1;
        continue;
      }
      break;
    }
    if (c.leaf) {
      emit_leaf_thread<T, D>(P, S, perm, gb, b, e, par, M, s);
      cnt[0] += 1;
      cnt[1] += (unsigned long long)it.depth * (e - b);
      continue;
    }
    if (cntL == 0 || cntR == 0) {
      emit_leaf_thread<T, D>(P, S, perm, gb, b, e, np, M, s);
      cnt[0] += 1;
      cnt[1] += (unsigned long long)it.depth * (e - b);
      cnt[3] += 1;
      continue;
    }
    cnt[2] += 1;
    if (sp + 2 > kSmall + 2) {
      set_error(P.err, kErrInternal);
      return;
    }
    stk[sp++] = Item{(uint16_t)(b + cntL), (uint16_t)e, (uint8_t)np, (uint8_t)(it.depth + 1), 0};
    stk[sp++] = Item{(uint16_t)b, (uint16_t)(b + cntL), (uint8_t)np, (uint8_t)(it.depth + 1), 0};
  }
}

// ------------------------------------------------------------- big kernel

template <typename T, int D>
struct BlockMoments {
  Moments<T, D> part[32];
};

// block-wide moments of perm[b, e) about s, accumulated in A (T, or double
// for the FP64 recheck of an FP32 decision); result valid in all threads
template <typename A, typename T, int D>
__device__ Moments<A, D> block_moments(const Problem &P, const int32_t *perm, int64_t b,
                                       int64_t e, const T *s, BlockMoments<A, D> &sh,
                                       bool &bad) {
  Moments<A, D> M;
  M.zero();
  A sa[D];
#pragma unroll
  for (int l = 0; l < D; ++l) sa[l] = (A)s[l];
  // runs of at most kBigRun terms per thread, folded exactly into M (the
  // error bound of FP32 sums grows with the run length)
  constexpr int kBigRun = 32;
  const int64_t step = blockDim.x;
  for (int64_t blk = b + threadIdx.x; blk < e; blk += step * kBigRun) {
    Moments<A, D> R;
    R.zero();
    const int64_t end = min(e, blk + step * kBigRun);
    for (int64_t i = blk; i < end; i += step) {
      int src = perm[i];
      A q[D];
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const T x = StoreOf<T>::load(P.q[l], src);
        bad |= !finite_val(x);
        q[l] = (A)x;
      }
      T w = StoreOf<T>::load(P.w, src);
      bad |= !(w > T(0)) || !finite_val(w);
      R.add((A)w, q, sa);
    }
    M.merge(R);
  }
  M.warp_allreduce();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh.part[warp] = M;
  __syncthreads();
  Moments<A, D> R = sh.part[0];
  for (int k = 1; k < nw; ++k) R.merge(sh.part[k]);
  return R;
}

// The cluster-per-cell path.  A thread-block cluster of kClusterCtas CTAs
// (512 threads each) takes one big cell at a time and cuts it (Steps 2-6)
// in global memory, on the permutation only, until every piece fits one
// CTA's tile; the pieces go to the team kernel.  For each set, CTA r of the
// cluster handles the r-th contiguous chunk of the set's range: it sums the
// chunk's moments and counts the chunk's V1 and V2 members, and the partial
// sums and counts go to every CTA of the cluster through distributed shared
// memory.  Every CTA merges the partials in rank order, so all take the same
// decision; the chunks' V1 members are written to the front in chunk order
// and their V2 members from the back, which is the order one CTA walking the
// whole range would write.  Rank 0 keeps the cluster's stack of sets.
constexpr int kClusterCtas = 4;
constexpr int kClusterThreads = 256;

template <typename T, int D>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
    cluster_kernel(Problem P) {
  namespace cg = cooperative_groups;
  constexpr int K = kClusterCtas;
  constexpr int kStack = 1024;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  __shared__ int4 stk[kStack];  // rank 0: the cluster's pending sets
  __shared__ int s_sp;
  __shared__ int s_ticket;
  __shared__ int4 s_item;       // the current set (written by rank 0)
  __shared__ __align__(16) BlockMoments<T, D> sh;
  __shared__ __align__(16) Moments<double, D> s_part[K];  // partial sums by rank
  __shared__ int s_cnt[K][3];   // V1 count, V2 count, near flag, by rank
  __shared__ int s_wcnt[2][16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const unsigned lt = lanemask_lt();
  static_assert(sizeof(Moments<T, D>) == sizeof(Moments<double, D>), "partial slots");
  if (timed_out(P.err)) return;  // the same in every CTA: set before the launch
  for (;;) {
    if (rank == 0 && tid == 0) {
      const int t = atomicAdd(P.big_next, 1);
      for (int r = 0; r < K; ++r) *cl.map_shared_rank(&s_ticket, r) = t;
    }
    cl.sync();
    const int t = s_ticket;
    if (t >= *P.big_count) break;
    const int c = P.big_list[t];
    const int64_t gb = P.cell_begin[c], ge = P.cell_begin[c + 1];
    if (*P.unsorted == 0)
      for (int64_t i = gb + (int64_t)rank * blockDim.x + tid; i < ge; i += (int64_t)K * blockDim.x)
        P.perm[i] = (int32_t)i;
    if (rank == 0 && tid == 0) {
      stk[0] = make_int4((int)gb, (int)ge, 0, c);
      s_sp = 1;
      atomicAdd(&P.stats[kStBig], 1ull);
      atomicAdd(&P.stats[kStCellsMerged], 1ull);
    }
    for (;;) {
      cl.sync();  // perm up to date; the stack settled
      if (rank == 0 && tid == 0) {
        const int4 it = s_sp > 0 ? stk[--s_sp] : make_int4(-1, -1, 0, 0);
        for (int r = 0; r < K; ++r) *cl.map_shared_rank(&s_item, r) = it;
      }
      cl.sync();
      const int4 it = s_item;
      if (it.x < 0) break;
      const int64_t b = it.x, e = it.y;
      const int64_t m = e - b;
      const int64_t c0 = b + m * rank / K, c1 = b + m * (rank + 1) / K;  // my chunk
      T s[D];
      const int first = P.perm[b];
#pragma unroll
      for (int l = 0; l < D; ++l) s[l] = StoreOf<T>::load(P.q[l], first);
      // Steps 2-6 on perm[b, e).  FP32 storage: a decision or a cut too
      // close to call in FP32 is taken again with FP64 sums (exact = true);
      // the control flow is the same in every CTA (identical merged sums).
      bool exact = sizeof(T) == 8;
      Cut cut;
      int64_t nL = 0;
      for (;;) {
        bool bad = false;
        // my chunk's moments, to every CTA's slot `rank`
        if (sizeof(T) == 4 && exact) {
          Moments<double, D> M = block_moments<double, T, D>(
              P, P.perm, c0, c1, s, reinterpret_cast<BlockMoments<double, D> &>(sh), bad);
          if (tid == 0)
            for (int r = 0; r < K; ++r) *cl.map_shared_rank(&s_part[rank], r) = M;
        } else {
          Moments<T, D> M = block_moments<T, T, D>(P, P.perm, c0, c1, s, sh, bad);
          if (tid == 0)
            for (int r = 0; r < K; ++r)
              *reinterpret_cast<Moments<T, D> *>(cl.map_shared_rank(&s_part[rank], r)) = M;
        }
        if (bad) set_error(P.err, kErrInput);
        cl.sync();
        if (sizeof(T) == 4 && exact) {
          Moments<double, D> M = s_part[0];
          for (int r = 1; r < K; ++r) M.merge(s_part[r]);
          cut = decide_exact<T, D, true>(P, M, s, (int)m);
        } else {
          Moments<T, D> M = *reinterpret_cast<const Moments<T, D> *>(&s_part[0]);
          for (int r = 1; r < K; ++r) M.merge(*reinterpret_cast<const Moments<T, D> *>(&s_part[r]));
          cut = Decider<T, D>::run(P, M, s, (int)m, 32);
        }
        if (cut.unsure) {
          exact = true;
          if (rank == 0 && tid == 0) atomicAdd(&P.stats[kStRecheck], 1ull);
          cl.sync();  // every CTA has read the partial slots
          continue;
        }
        unsigned ev = cut.near;
        nL = 0;
        if (!cut.leaf) {
          // pass 1: my chunk's V1 and V2 counts and near band, to every CTA
          int cl1 = 0, cr1 = 0;
          bool nr = false;
          for (int64_t i = c0 + tid; i < c1; i += blockDim.x) {
            const T q = StoreOf<T>::load(P.q[cut.k], P.perm[i]);
            if (Decider<T, D>::left(q, cut))
              ++cl1;
            else
              ++cr1;
            nr |= Decider<T, D>::near(q, cut);
          }
          cl1 = __reduce_add_sync(0xffffffffu, (unsigned)cl1);
          cr1 = __reduce_add_sync(0xffffffffu, (unsigned)cr1);
          __syncthreads();
          if (lane == 0) {
            s_wcnt[0][warp] = cl1;
            s_wcnt[1][warp] = cr1;
          }
          const int anyn = __syncthreads_or(nr);
          if (tid == 0) {
            int L = 0, R = 0;
            for (int k = 0; k < nw; ++k) {
              L += s_wcnt[0][k];
              R += s_wcnt[1][k];
            }
            for (int r = 0; r < K; ++r) {
              int *dst = cl.map_shared_rank(&s_cnt[rank][0], r);
              dst[0] = L;
              dst[1] = R;
              dst[2] = anyn;
            }
          }
          cl.sync();
          int64_t offL = 0, offR = 0, totL = 0;
          bool gnear = false;
          for (int r = 0; r < K; ++r) {
            if (r < rank) {
              offL += s_cnt[r][0];
              offR += s_cnt[r][1];
            }
            totL += s_cnt[r][0];
            gnear |= s_cnt[r][2] != 0;
          }
          if (gnear && !exact) {
            exact = true;  // nothing written yet
            if (rank == 0 && tid == 0) atomicAdd(&P.stats[kStRecheck], 1ull);
            continue;
          }
          if (gnear) ev |= kNearCut;
          // pass 2: stable-left / reversed-right writes of my chunk into
          // perm_tmp at the offsets of the earlier chunks
          int64_t cntL = offL, cntR = offR;
          for (int64_t base = c0; base < c1; base += blockDim.x) {
            const int64_t i = base + tid;
            const bool valid = i < c1;
            const int src = valid ? P.perm[i] : 0;
            const bool lft = valid && Decider<T, D>::left(StoreOf<T>::load(P.q[cut.k], src), cut);
            const unsigned bl = __ballot_sync(0xffffffffu, lft);
            const unsigned br = __ballot_sync(0xffffffffu, valid && !lft);
            __syncthreads();
            if (lane == 0) {
              s_wcnt[0][warp] = __popc(bl);
              s_wcnt[1][warp] = __popc(br);
            }
            __syncthreads();
            int wL = 0, wR = 0, tL = 0, tR = 0;
            for (int k = 0; k < nw; ++k) {
              if (k < warp) {
                wL += s_wcnt[0][k];
                wR += s_wcnt[1][k];
              }
              tL += s_wcnt[0][k];
              tR += s_wcnt[1][k];
            }
            if (valid) {
              const int64_t dst = lft ? (b + cntL + wL + __popc(bl & lt))
                                      : (e - 1 - cntR - wR - __popc(br & lt));
              if (check_index(P.check, P.err, dst >= b && dst < e && (unsigned)src < (unsigned)P.n,
                              kChkCluster, dst))
                P.perm_tmp[dst] = src;
            }
            cntL += tL;
            cntR += tR;
          }
          cl.sync();  // every chunk written
          for (int64_t i = c0 + tid; i < c1; i += blockDim.x) P.perm[i] = P.perm_tmp[i];
          nL = totL;
          if (totL == 0 || totL == m) {
            cut.leaf = 1;
            if (rank == 0 && tid == 0) atomicAdd(&P.stats[kStDegenerate], 1ull);
          }
        }
        if (ev && rank == 0 && tid == 0) {
          if (ev & kNearStop) atomicAdd(&P.stats[kStNearStop], 1ull);
          if (ev & kNearArgmax) atomicAdd(&P.stats[kStNearArgmax], 1ull);
          if (ev & kNearCut) atomicAdd(&P.stats[kStNearCut], 1ull);
          if (atomicOr(&P.cell_flags[c], ev) == 0u) atomicAdd(&P.stats[kStCellsFlagged], 1ull);
        }
        break;
      }
      if (cut.leaf) {
        cl.sync();  // perm of the whole set copied back
        for (int64_t i = c0 + tid; i < c1; i += blockDim.x) {
          P.perm_final[i] = P.perm[i];
          P.head[i] = (i == b) ? head_code((int)m) : (uint8_t)0;
          stage_global<T, D>(P, i, P.perm[i]);
        }
        if (rank == 0 && tid == 0) {
          atomicAdd(&P.stats[kStLeaves], 1ull);
          atomicAdd(&P.stats[kStDepth], (unsigned long long)it.z * m);
        }
        continue;
      }
      if (rank == 0 && tid == 0) {
        atomicAdd(&P.stats[kStSplits], 1ull);
        const int4 ch[2] = {make_int4((int)b, (int)(b + nL), it.z + 1, c),
                            make_int4((int)(b + nL), (int)e, it.z + 1, c)};
        for (int h = 1; h >= 0; --h) {
          const int n = ch[h].y - ch[h].x;
          if (n > P.cap) {
            if (s_sp < kStack)
              stk[s_sp++] = ch[h];
            else
              set_error(P.err, kErrInternal);
          } else {
            const int slot = atomicAdd(P.piece_count, 1);
            if (slot < P.max_pieces)
              P.pieces[slot] = ch[h];
            else
              set_error(P.err, kErrInternal);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- launch

template <typename T, int D>
static cudaError_t launch_big_t(const Problem &P, int grid, cudaStream_t st) {
  // whole clusters only
  grid = (grid + kClusterCtas - 1) / kClusterCtas * kClusterCtas;
  cluster_kernel<T, D><<<grid, kClusterThreads, 0, st>>>(P);
  return cudaGetLastError();
}

template <typename T>
static size_t smem_t(int D, int cap) {
  switch (D) {
    case 2: return unit_smem_bytes<T, 2>(cap);
    case 3: return unit_smem_bytes<T, 3>(cap);
    case 4: return unit_smem_bytes<T, 4>(cap);
    case 5: return unit_smem_bytes<T, 5>(cap);
    default: return unit_smem_bytes<T, 6>(cap);
  }
}

size_t unit_smem(int mixed, int D, int cap) {
  return mixed ? smem_t<float>(D, cap) : smem_t<double>(D, cap);
}

#define PMA_DISPATCH_D(FN, T, ...)                        \
  switch (P.D) {                                          \
    case 2: return FN<T, 2>(__VA_ARGS__);                 \
    case 3: return FN<T, 3>(__VA_ARGS__);                 \
    case 4: return FN<T, 4>(__VA_ARGS__);                 \
    case 5: return FN<T, 5>(__VA_ARGS__);                 \
    case 6: return FN<T, 6>(__VA_ARGS__);                 \
    default: return cudaErrorInvalidValue;                \
  }

cudaError_t launch_big(const Problem &P, int mixed, int grid, cudaStream_t st) {
  if (mixed) {
    PMA_DISPATCH_D(launch_big_t, float, P, grid, st)
  } else {
    PMA_DISPATCH_D(launch_big_t, double, P, grid, st)
  }
}

}  // namespace pma

// ============================================================================
// Allocation-free variant (pma_merge_noalloc in include/pma.h).
//
// For callers that must not allocate device memory, the per-cell kernel
// above is repeated here with its scratch (look-back words, final
// permutation, head bytes, centroid records) in one file-scope device array
// of fixed size, and the Step 7 emission fused into the same kernel: each
// CTA takes cells in ascending order, partitions one in shared memory,
// counts its final sets, gets the number of sets before it by decoupled
// look-back over cells, and writes its merged particles.  Input must be
// grouped by cell (non-decreasing ids); cell ranges are found by binary
// search, so no binning workspace is needed.
// ============================================================================

namespace pma {

struct NoAllocScratch {
  // must be zero when a call starts: the header, and the look-back words of
  // the call's n_cells cells
  int32_t ticket;
  unsigned err;
  int64_t count;
  unsigned long long stats[kStCount];
  unsigned long long status[PMA_NOALLOC_MAX_CELLS];
  // written before being read within a call
  int32_t perm_final[PMA_NOALLOC_MAX_N];
  uint8_t head[PMA_NOALLOC_MAX_N];
};
constexpr size_t kNoAllocHeaderBytes = offsetof(NoAllocScratch, status);
constexpr unsigned kErrCellTooBig = 8u;

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

struct NoAllocOut {
  int32_t *cell;
  void *pos[3];
  double *mom[3];
  double *w;
  int32_t *index;
  int64_t *count_dev;
};

__device__ __forceinline__ int lower_bound_cell(const int32_t *cells, int n, int c) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cells[mid] < c)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <typename T, int D>
__global__ void __launch_bounds__(256) noalloc_kernel(Problem P, NoAllocScratch *Sc, int n,
                                                      NoAllocOut o) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ctr[4];
  __shared__ int s_cell, s_b, s_e;
  __shared__ int s_warp[32];
  __shared__ long long s_base;
  __shared__ unsigned long long s_st[kStCount];

  const int cap = P.cap;
  Tile<T, D> S;
  S.base = reinterpret_cast<T *>(smem_raw);
  S.cap = cap;
  S.id[0] = reinterpret_cast<uint16_t *>(S.base + (size_t)2 * (D + 1) * cap);
  S.id[1] = S.id[0] + cap;
  const int max_big = cap / kSmall + 2;
  Item *lists = reinterpret_cast<Item *>(S.id[1] + cap);
  Item *cur = lists, *nxt = lists + max_big;
  Item *small = lists + 2 * max_big;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid < kStCount) s_st[tid] = 0ull;
  unsigned long long cnt[4] = {0ull, 0ull, 0ull, 0ull};

  // ids in range and non-decreasing (the binary search relies on it)
  for (int i = blockIdx.x * blockDim.x + tid; i < n; i += gridDim.x * blockDim.x) {
    int c = P.cells[i];
    if (c < 0 || c >= P.n_cells || (i > 0 && P.cells[i - 1] > c)) atomicOr(&Sc->err, kErrInput);
  }

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      int c = atomicAdd(&Sc->ticket, 1);
      s_cell = c;
      if (c < P.n_cells) {
        s_b = lower_bound_cell(P.cells, n, c);
        s_e = lower_bound_cell(P.cells, n, c + 1);
        if (s_e < s_b) s_e = s_b;
      }
    }
    __syncthreads();
    const int c = s_cell;
    if (c >= P.n_cells) break;
    const int64_t gb = s_b;
    const int m = s_e - s_b;
    const bool pass = m > 0 && (m <= P.n_min || m == 1 || m > cap);
    if (m > cap && m > P.n_min && m > 1 && tid == 0) atomicOr(&Sc->err, kErrCellTooBig);
    if (pass) {
      for (int i = tid; i < m; i += blockDim.x) {
        P.perm_final[gb + i] = (int)(gb + i);
        P.head[gb + i] = kHeadSingle;
      }
    } else if (m > 0) {
      bool bad = false;
      for (int i = tid; i < m; i += blockDim.x) {
        const int src = (int)(gb + i);
#pragma unroll
        for (int l = 0; l < D; ++l) {
          T x = StoreOf<T>::load(P.q[l], src);
          bad |= !finite_val(x);
          S.col(0, l)[i] = x;
        }
        T w = StoreOf<T>::load(P.w, src);
        bad |= !(w > T(0)) || !finite_val(w);
        S.col(0, D)[i] = w;
        S.id[0][i] = (uint16_t)i;
      }
      if (bad) atomicOr(&Sc->err, kErrInput);
      if (tid == 0) {
        Item root{0, (uint16_t)m, 0, 0, 0};
        s_ctr[0] = s_ctr[1] = s_ctr[2] = s_ctr[3] = 0;
        if (m <= kSmall) {
          small[0] = root;
          s_ctr[2] = 1;
        } else {
          cur[0] = root;
          s_ctr[0] = 1;
        }
      }
      __syncthreads();
      for (;;) {
        const int ncur = s_ctr[0];
        if (ncur == 0) break;
        for (int k = warp; k < ncur; k += nwarps)
          warp_split<T, D>(P, S, nullptr, gb, cur[k], nxt, &s_ctr[1], max_big, small, &s_ctr[2],
                           s_st, lane);
        __syncthreads();
        if (tid == 0) {
          s_ctr[0] = min(s_ctr[1], max_big);
          s_ctr[1] = 0;
        }
        Item *t = cur;
        cur = nxt;
        nxt = t;
        __syncthreads();
      }
      const int n_small = s_ctr[2];
      for (;;) {
        int k = atomicAdd(&s_ctr[3], 1);
        if (k >= n_small) break;
        thread_finish<T, D>(P, S, nullptr, gb, small[k], cnt);
      }
    }
    __syncthreads();
    // Step 7 for this cell: count its sets, prefix over cells, write outputs
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int p0 = min(m, tid * per), p1 = min(m, p0 + per);
    int heads = 0;
    for (int p = p0; p < p1; ++p) heads += P.head[gb + p] != 0;
    int total;
    const int ex = block_exclusive_scan(heads, s_warp, &total);
    if (tid == 0) {
      s_base = tile_exclusive_prefix(Sc->status, c, total, &Sc->err);
      if (c == P.n_cells - 1) {
        Sc->count = s_base + total;
        if (o.count_dev) *o.count_dev = s_base + total;
      }
    }
    __syncthreads();
    long long run = s_base + ex;
    for (int p = p0; p < p1; ++p) {
      const int64_t gp = gb + p;
      const uint8_t h = P.head[gp];
      if (h) ++run;
      const long long slot = run - 1;
      const int orig = P.perm_final[gp];
      if (slot < 0 || (unsigned)orig >= (unsigned)n) {
        atomicOr(&Sc->err, kErrInternal);
        continue;
      }
      if (o.index) o.index[orig] = (int32_t)slot;
      if (!h) continue;
      o.cell[slot] = c;
      if (h == kHeadSingle) {
        // a particle copied as it is (a one-particle set or a cell passed
        // through): every loaded value is checked, as in pma_merge
        bool bad = false;
        for (int l = 0; l < P.dx; ++l) {
          const T x = StoreOf<T>::load(P.q[l], orig);
          bad |= !finite_val(x);
          static_cast<T *>(o.pos[l])[slot] = x;
        }
        for (int l = 0; l < P.D - P.dx; ++l) {
          T x = StoreOf<T>::load(P.q[P.dx + l], orig);
          bad |= !finite_val(x);
          o.mom[l][slot] = sizeof(T) == 4 ? f2d_exact((float)x) : (double)x;
        }
        T w = StoreOf<T>::load(P.w, orig);
        if (bad || !(w > T(0)) || !finite_val(w)) atomicOr(&Sc->err, kErrInput);
        o.w[slot] = sizeof(T) == 4 ? f2d_exact((float)w) : (double)w;
      } else {
        // merged set: FP64 sums over its members (positions up to the next
        // head of the cell)
        double W = 0.0, S1[D];
#pragma unroll
        for (int l = 0; l < D; ++l) S1[l] = 0.0;
        for (int r = p; r < m; ++r) {
          if (r > p && P.head[gb + r]) break;
          const int om = P.perm_final[gb + r];
          if ((unsigned)om >= (unsigned)n) break;
          const T wm = StoreOf<T>::load(P.w, om);
          const double wd = sizeof(T) == 4 ? f2d_exact((float)wm) : (double)wm;
          W += wd;
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const T x = StoreOf<T>::load(P.q[l], om);
            S1[l] = fma(wd, sizeof(T) == 4 ? f2d_exact((float)x) : (double)x, S1[l]);
          }
        }
        o.w[slot] = W;
        for (int l = 0; l < P.dx; ++l) static_cast<T *>(o.pos[l])[slot] = (T)(S1[l] / W);
        for (int l = 0; l < P.D - P.dx; ++l) o.mom[l][slot] = S1[P.dx + l] / W;
      }
    }
  }
  atomicAdd(&s_st[kStLeaves], cnt[0]);
  atomicAdd(&s_st[kStSplits], cnt[2]);
  __syncthreads();
  if (tid < kStCount && s_st[tid]) atomicAdd(&Sc->stats[tid], s_st[tid]);
}

template <typename T, int D>
static cudaError_t launch_noalloc_t(const Problem &P, NoAllocScratch *Sc, int n,
                                    const NoAllocOut &o, int grid, cudaStream_t st) {
  size_t smem = unit_smem_bytes<T, D>(P.cap);
  cudaError_t e = cudaFuncSetAttribute(noalloc_kernel<T, D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  noalloc_kernel<T, D><<<grid, 256, smem, st>>>(P, Sc, n, o);
  return cudaGetLastError();
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices];  // device address of the scratch, per device
int g_noalloc_sms[kMaxDevices];
int g_noalloc_smem[kMaxDevices];
}  // namespace

}  // namespace pma

extern "C" int pma_merge_noalloc(const pma_config *cfg, int64_t n, const int32_t *cells,
                                 const void *const *pos, const void *const *mom,
                                 const void *weights, double tol_x, double tol_p,
                                 const pma_output *out, int64_t *count_host, void *stream) {
  using namespace pma;
  if (!cfg || !out) return PMA_ERR_INVALID_ARG;
  // only the paper's rule and plain Step 7: a variant or energy flag would be
  // silently ignored here, so it is refused (PMA_FLAG_NO_INDEX is accepted)
  if (cfg->flags & ~PMA_FLAG_NO_INDEX) return PMA_ERR_INVALID_ARG;
  if (cfg->dx < 1 || cfg->dx > 3 || cfg->dp < 1 || cfg->dp > 3 || cfg->n_min < 0 ||
      cfg->n_cells < 1 || (cfg->precision != PMA_FP64 && cfg->precision != PMA_MIXED))
    return PMA_ERR_INVALID_ARG;
  for (int a = 0; a < cfg->dx; ++a)
    if (!(cfg->cell_size[a] > 0.0) || !isfinite(cfg->cell_size[a])) return PMA_ERR_INVALID_ARG;
  if (!(tol_x >= 0.0) || !(tol_p >= 0.0) || !isfinite(tol_x) || !isfinite(tol_p))
    return PMA_ERR_INVALID_ARG;
  if (n < 0) return PMA_ERR_INVALID_ARG;
  if (n > PMA_NOALLOC_MAX_N || cfg->n_cells > PMA_NOALLOC_MAX_CELLS) return PMA_ERR_CAPACITY;
  if (n > 0) {
    if (!cells || !pos || !mom || !weights || !out->cell || !out->w) return PMA_ERR_INVALID_ARG;
    for (int a = 0; a < cfg->dx; ++a)
      if (!pos[a] || !out->pos[a]) return PMA_ERR_INVALID_ARG;
    for (int a = 0; a < cfg->dp; ++a)
      if (!mom[a] || !out->mom[a]) return PMA_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PMA_ERR_CUDA;
  // once per device, with that device current: the scratch array's device
  // address (the symbol itself is a host-side stand-in)
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PMA_ERR_CUDA;
      }
      int sms = 0, smem = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
              cudaSuccess)
        return PMA_ERR_CUDA;
      g_noalloc_sms[dev] = sms;
      g_noalloc_smem[dev] = smem;
      g_noalloc_addr[dev] = p;
    }
    addr = g_noalloc_addr[dev];
  }
  NoAllocScratch *Sc = static_cast<NoAllocScratch *>(addr);
  if (cudaMemsetAsync(Sc, 0, kNoAllocHeaderBytes + (size_t)cfg->n_cells * sizeof(unsigned long long),
                      st) != cudaSuccess)
    return PMA_ERR_CUDA;
  if (n == 0) {
    if (out->count_dev && cudaMemsetAsync(out->count_dev, 0, sizeof(int64_t), st) != cudaSuccess)
      return PMA_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PMA_ERR_CUDA;
    if (count_host) *count_host = 0;
    return PMA_OK;
  }
  const int mixed = cfg->precision == PMA_MIXED;
  const int D = cfg->dx + cfg->dp;
  int cap = 8192;
  while (cap > 64 && unit_smem(mixed, D, cap) + 4096 > (size_t)g_noalloc_smem[dev]) cap -= 64;

  Problem P{};
  P.n_cells = (int32_t)cfg->n_cells;
  P.dx = cfg->dx;
  P.D = D;
  P.n_min = cfg->n_min;
  P.cap = cap;
  P.tol2_x = tol_x * tol_x;
  P.tol2_p = tol_p * tol_p;
  P.tol2_xf = (float)P.tol2_x;
  P.tol2_pf = (float)P.tol2_p;
  for (int a = 0; a < 3; ++a) {
    double L = a < cfg->dx ? cfg->cell_size[a] : 1.0;
    P.L2[a] = L * L;
    P.L2f[a] = (float)P.L2[a];
  }
  for (int a = 0; a < cfg->dx; ++a) P.q[a] = pos[a];
  for (int a = 0; a < cfg->dp; ++a) P.q[cfg->dx + a] = mom[a];
  P.w = weights;
  P.cells = cells;
  P.head = Sc->head;
  P.perm_final = Sc->perm_final;
  P.err = &Sc->err;
  P.stats = Sc->stats;
  NoAllocOut o{};
  o.cell = out->cell;
  for (int a = 0; a < 3; ++a) {
    o.pos[a] = out->pos[a];
    o.mom[a] = out->mom[a];
  }
  o.w = out->w;
  o.index = (cfg->flags & PMA_FLAG_NO_INDEX) ? nullptr : out->index;
  o.count_dev = out->count_dev;
  const int grid = (int)std::min<int64_t>(cfg->n_cells, g_noalloc_sms[dev]);
  cudaError_t e;
#define PMA_NOALLOC_CASE(TT, DD) e = launch_noalloc_t<TT, DD>(P, Sc, (int)n, o, grid, st)
  if (mixed) {
    switch (D) {
      case 2: PMA_NOALLOC_CASE(float, 2); break;
      case 3: PMA_NOALLOC_CASE(float, 3); break;
      case 4: PMA_NOALLOC_CASE(float, 4); break;
      case 5: PMA_NOALLOC_CASE(float, 5); break;
      default: PMA_NOALLOC_CASE(float, 6); break;
    }
  } else {
    switch (D) {
      case 2: PMA_NOALLOC_CASE(double, 2); break;
      case 3: PMA_NOALLOC_CASE(double, 3); break;
      case 4: PMA_NOALLOC_CASE(double, 4); break;
      case 5: PMA_NOALLOC_CASE(double, 5); break;
      default: PMA_NOALLOC_CASE(double, 6); break;
    }
  }
#undef PMA_NOALLOC_CASE
  if (e != cudaSuccess) return PMA_ERR_CUDA;
  struct {
    int32_t ticket;
    unsigned err;
    int64_t count;
  } st_host{};
  if (cudaMemcpyAsync(&st_host, &Sc->ticket, sizeof(st_host), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PMA_ERR_CUDA;
  if (count_host) *count_host = st_host.count;
  if (st_host.err & kErrInput) return PMA_ERR_INPUT;
  if (st_host.err & kErrCellTooBig) return PMA_ERR_CAPACITY;
  if (st_host.err & kErrTimeout) return PMA_ERR_TIMEOUT;
  if (st_host.err & kErrInternal) return PMA_ERR_INTERNAL;
  return PMA_OK;
}
