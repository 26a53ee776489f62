// Team kernel: Sec. 3, Steps 2-6 for every unit that fits one CTA's shared
// memory (a cell, or a piece of a cell first cut in global memory), and the
// verbatim copy of cells with N <= N_min.
//
// A team of 1, 4, 8 or 12 warps owns one batch of units at a time: the
// consecutive units of its ticket chunk that fit its tile together, side by
// side.  Their coordinates and weights are staged once in shared memory (SoA
// columns) and stay in place.
// A subset is a contiguous range of a 16-bit index array; a cut writes
// V1 = {q_k <= Q_k} to the front and V2 to the back of the same range in the
// other index array (double-buffered by tree depth), so the final sets come
// out in V1-first depth-first order when listed by position, whatever order
// the subsets are processed in.
//
// Pending subsets wait on one stack per size class.  A round takes up to
// 32/G subsets of one class per warp and gives each a group of G lanes
// (G = 32 for the largest sets down to G = 1, so that a lane reads at most
// about B particles, B the class base of the handle: 12 by default): moments by lane-strided sums and a butterfly inside the
// group, Steps 3-5, and the cut by group-masked ballots.  Two-particle sets
// have their own round, the same arithmetic without loops.  CTA barriers
// separate rounds.
//
// The template flag VAR selects the decision: false compiles the paper's rule
// only; true reads the optional variants (normalised split axis, momentum
// norm) from the problem at run time.  The two builds live in separate
// translation units (warp.cu, warp_var.cu).
#pragma once

#include "lookback.cuh"
#include "pma_device.cuh"
#include "pma_launch.h"
#include "split_common.cuh"

namespace pma {

constexpr int kWarpChunk = 4;  // cells taken per work-counter increment
constexpr int kClasses = 7;    // pairs, then G = 1, 2, 4, 8, 16, 32
constexpr int kMaxCapW = 8191;
constexpr int kMaxTeam = 12;   // warps of the largest team

// size class of a subset of m >= 2 particles for class base B: pairs, then
// up to B, 2B, 4B, 8B, 16B particles, and more
__device__ __forceinline__ int size_class(int m, int B) {
  if (m == 2) return 0;
  if (m <= B) return 1;
  if (m <= 2 * B) return 2;
  if (m <= 4 * B) return 3;
  if (m <= 8 * B) return 4;
  if (m <= 16 * B) return 5;
  return 6;
}

// most subsets of a class that can be pending at once: they are disjoint
// subsets of at least lo particles of one tile of at most cap
__host__ __device__ inline int class_capacity(int c, int cap, int B = kClassBaseMin) {
  // smallest size of class c: 2, 3, B + 1, 2B + 1, 4B + 1, 8B + 1, 16B + 1
  const int lo = c == 0 ? 2 : (c == 1 ? 3 : (B << (c - 2)) + 1);
  return cap / lo;
}

// Pending pairs (n0) and subsets of 3 to B particles (n1) are disjoint subsets
// of the tile, so 2 n0 + 3 n1 <= cap and n0 + n1 <= cap / 2: the two classes
// share one region of cap / 2 records, pairs from the front and the 3-B class
// from the back.  Every other class has a region of its own (sized here for
// the smallest B, which needs the most records).
__host__ __device__ inline int stacks_entries(int cap) {
  int t = cap / 2;
  for (int c = 2; c < kClasses; ++c) t += class_capacity(c, cap);
  return t;
}

// subset record: begin (13 bits) | length (13 bits) << 13 | parity << 26
__device__ __forceinline__ uint32_t pack_rec(int b, int m, int par) {
  return (uint32_t)b | ((uint32_t)m << 13) | ((uint32_t)par << 26);
}
__device__ __forceinline__ int rec_begin(uint32_t r) { return (int)(r & 8191u); }
__device__ __forceinline__ int rec_len(uint32_t r) { return (int)((r >> 13) & 8191u); }
__device__ __forceinline__ int rec_par(uint32_t r) { return (int)((r >> 26) & 1u); }

// Views into the tile's shared memory.  Every member is a plain pointer or
// integer (no arrays), so the struct lives in registers.
template <typename T, int D>
struct WarpTile {
  T *data;         // [D + 1][cap]: coordinates, then weight
  uint16_t *idx0;  // [2][cap] index arrays, by depth parity
  uint32_t *stk0;  // the class stacks, back to back
  int *top;        // [kClasses] stack heights
  uint16_t *soff;  // [kClasses] first entry of each stack (class 1: the end
                   // of the region shared with class 0), [kClasses] capacities
  int *ev;         // [kEvWords]: the batch's unit table, the CTA's counts of
                   // near-ties by kind and of FP64 rechecks
  const DecideConsts *dk;  // the FP64 decision's constants (for rechecks)
  void *wide;      // wide rounds: [kMaxTeam] partial moments, [kMaxTeam] counts
  int cap;
  int base;        // class base B
  __device__ __forceinline__ T *col(int l) const { return data + (size_t)l * cap; }
  __device__ __forceinline__ uint16_t *idx(int par) const { return idx0 + par * cap; }
  // entry i of class c's stack (class 1 runs backwards from its region's end)
  __device__ __forceinline__ uint32_t *rec(int c, int i) const {
    return c == 1 ? stk0 + (soff[1] - 1 - i) : stk0 + soff[c] + i;
  }
  __device__ __forceinline__ int stk_cap(int c) const { return soff[kClasses + c]; }
};

// A tile holds a batch of up to kMaxBatch units (consecutive units of the
// team's ticket chunk that fit together), cut in the same rounds, so that the
// sets of several small cells fill one round's lanes.  Their sets stay
// disjoint ranges of the tile, and each unit's final positions stay its own.
constexpr int kMaxBatch = 8;

// control words after the class stack heights: the unit ticket, then kEvWords
// words: the batch's unit count, the CTA's near-stop, near-argmax, near-cut
// and recheck counts, then per unit of the batch its near-tie bits, first
// tile position, size, first sorted position and cell
constexpr int kEvBatchN = 0;
constexpr int kEvBits = 5;
constexpr int kEvOff = kEvBits + kMaxBatch;
constexpr int kEvN = kEvOff + kMaxBatch;
constexpr int kEvGb = kEvN + kMaxBatch;
constexpr int kEvCell = kEvGb + kMaxBatch;
constexpr int kEvWords = kEvCell + kMaxBatch;

template <typename T, int D>
__host__ __device__ inline size_t warp_region_bytes(int cap) {
  size_t b = (size_t)(D + 1) * cap * sizeof(T) + (size_t)2 * cap * sizeof(uint16_t);
  b = (b + 15) & ~size_t(15);
  b += (size_t)stacks_entries(cap) * sizeof(uint32_t) +
       (kClasses + 1 + kEvWords) * sizeof(int) + 2 * kClasses * sizeof(uint16_t);
  b = (b + 15) & ~size_t(15);
  b += kMaxTeam * (sizeof(Moments<T, D>) + sizeof(int));
  b = (b + 15) & ~size_t(15);
  b += sizeof(DecideConsts);
  return (b + 15) & ~size_t(15);
}

// per-lane counters of one launch (32 bits suffice for the per-lane counts of
// sets; the depth sum is a 64-bit particle-level count)
struct Counters {
  unsigned leaves, splits, degenerate;
  unsigned long long depth;
};

// particle j of the tile, staged at final position gp
template <typename T, int D>
__device__ __forceinline__ void stage(const Problem &P, const WarpTile<T, D> &S, int64_t gp,
                                      int j) {
#pragma unroll
  for (int l = 0; l <= D; ++l) static_cast<T *>(P.fin[l])[gp] = S.col(l)[j];
}

// A final set's positions [b, b + m) belong to no other subset, so both
// index buffers are free there: buffer 0 takes the tile index of the particle
// at each final position and buffer 1 its head code (Step 7 input); the unit
// is written out to global memory in one coalesced pass at its end.
template <typename T, int D>
__device__ __forceinline__ void mark_final(const WarpTile<T, D> &S, int pos, int j, int h) {
  S.idx(0)[pos] = (uint16_t)j;
  S.idx(1)[pos] = (uint16_t)h;
}

template <typename T, int D>
__device__ __forceinline__ void emit_single(const Problem &, const WarpTile<T, D> &S,
                                            const int32_t *, int64_t, int pos, int j) {
  mark_final<T, D>(S, pos, j, kHeadSingle);
}

template <typename T, int D>
__device__ __forceinline__ void push_rec(unsigned *err, const WarpTile<T, D> &S, int c,
                                         uint32_t r) {
  const int slot = atomicAdd(&S.top[c], 1);
  if (slot < S.stk_cap(c))
    *S.rec(c, slot) = r;
  else
    set_error(err, kErrInternal);
}

// a child set of m particles at [b, b + m) of index buffer par: a single
// particle is final at once (returns 1, a final set), else it is pushed
template <typename T, int D>
__device__ __forceinline__ unsigned push_set(unsigned *err, const WarpTile<T, D> &S, int b,
                                             int m, int par) {
  if (m == 1) {
    mark_final<T, D>(S, b, S.idx(par)[b], kHeadSingle);
    return 1u;
  }
  push_rec<T, D>(err, S, size_class(m, S.base), pack_rec(b, m, par));
  return 0u;
}

template <typename T, int D>
__device__ __forceinline__ void push_child(const Problem &P, const WarpTile<T, D> &S,
                                           const int32_t *, int64_t, int b, int m, int par,
                                           Counters &cnt) {
  cnt.leaves += push_set<T, D>(P.err, S, b, m, par);
}

// A rare event of one decision on the set that starts at tile position b:
// near-tie bits (kNear*) and rechecks (kRechecked), into the bits of the
// batch unit that holds b and into the CTA's counts.
static __device__ __noinline__ void note_event_words(int *ev, int b, unsigned bits) {
  const int nb = ev[kEvBatchN];
  int u = 0;
  while (u + 1 < nb && b >= ev[kEvOff + u + 1]) ++u;
  atomicOr(reinterpret_cast<unsigned *>(&ev[kEvBits + u]), bits);
  if (bits & kNearStop) atomicAdd(&ev[1], 1);
  if (bits & kNearArgmax) atomicAdd(&ev[2], 1);
  if (bits & kNearCut) atomicAdd(&ev[3], 1);
  if (bits & kRechecked) atomicAdd(&ev[4], 1);
}

template <typename T, int D>
__device__ __forceinline__ void note_event(const WarpTile<T, D> &S, int b, unsigned bits) {
  note_event_words(S.ev, b, bits);
}

// Longest run of terms one lane adds in plain FP32 before the run is folded
// into the compensated sums (bounds the error of long sums).
constexpr int kRunBlock = 32;

// moments of the set's particles i = i0, i0 + step, ... < m about s, with
// every kRunBlock consecutive terms of a lane summed in plain FP32 and then
// folded exactly (two-sum) into M
template <typename T, int D>
__device__ __forceinline__ void accumulate_blocked(Moments<T, D> &M, const WarpTile<T, D> &S,
                                                   const uint16_t *ix, int b, int m, int i0,
                                                   int step, const T *s) {
  for (int blk = i0; blk < m; blk += step * kRunBlock) {
    Moments<T, D> R;
    R.zero();
    const int end = min(m, blk + step * kRunBlock);
#pragma unroll 4
    for (int i = blk; i < end; i += step) {
      const int j = ix[b + i];
      T q[D];
#pragma unroll
      for (int l = 0; l < D; ++l) q[l] = S.col(l)[j];
      R.add(S.col(D)[j], q, s);
    }
    M.merge(R);
  }
}

// FP32 storage: Steps 2-6 for one set in FP64 from its particles, by the
// whole warp (warp-uniform call), when an FP32 decision or cut value on it
// was closer than its error bound.  The cut value is the FP64 centroid
// rounded down to float; particles in the FP64 near band are cut near-ties.
// Called from the kernel's round loop after a round (not from inside the
// round bodies), where little else is live.  Returns the set's counts:
// leaves (bits 0-1), splits (bit 2), degenerate cuts (bit 3), and the set's
// size when it was split (bits 8-20, for the depth sum).
template <typename T, int D, bool VAR>
__device__ __forceinline__ unsigned exact_set(WarpTile<T, D> S, unsigned *err, int b, int m,
                                           int par, int lane) {
  const unsigned full = 0xffffffffu;
  const uint16_t *ix = S.idx(par);
  // the FP64 sums go through this warp's slot of the wide-round scratch
  // (W, m1[D], m2[D]), one axis at a time, so that few registers are live
  double *xs = reinterpret_cast<double *>(static_cast<Moments<T, D> *>(S.wide) +
                                          (threadIdx.x >> 5));
  const int j0 = ix[b];
  T s[D];
#pragma unroll
  for (int l = 0; l < D; ++l) {
    s[l] = S.col(l)[j0];
    const double sl = (double)s[l];
    double a1 = 0.0, a2 = 0.0, aw = 0.0;
    for (int i = lane; i < m; i += 32) {
      const int j = ix[b + i];
      const double w = (double)S.col(D)[j];
      const double d = (double)S.col(l)[j] - sl;
      const double t = w * d;
      a1 += t;
      a2 = fma(t, d, a2);
      if (l == 0) aw += w;
    }
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
      a1 += __shfl_xor_sync(full, a1, k);
      a2 += __shfl_xor_sync(full, a2, k);
      if (l == 0) aw += __shfl_xor_sync(full, aw, k);
    }
    if (lane == 0) {
      xs[1 + l] = a1;
      xs[1 + D + l] = a2;
      if (l == 0) xs[0] = aw;
    }
  }
  __syncwarp();
  double sd[D];
#pragma unroll
  for (int l = 0; l < D; ++l) sd[l] = (double)s[l];
  const Cut cut = decide_fp64<D, VAR, DecideConsts>(*S.dk, xs[0], xs + 1, xs + 1 + D, sd, m);
  const int np = par ^ 1;
  int cntL = 0;
  bool nr = false;
  if (!cut.leaf) {
    const T *qk = S.col(cut.k);
    const unsigned lt = lanemask_lt();
    int cntR = 0;
    for (int base = 0; base < m; base += 32) {
      const int i = base + lane;
      const bool valid = i < m;
      const int j = valid ? ix[b + i] : 0;
      const T q = qk[j];
      const bool lft = valid && Decider<T, D, VAR>::left(q, cut);
      nr |= valid && Decider<T, D, VAR>::near(q, cut);
      const unsigned bl = __ballot_sync(full, lft);
      const unsigned br = __ballot_sync(full, valid && !lft);
      if (valid) {
        const int dst = lft ? (b + cntL + __popc(bl & lt)) : (b + m - 1 - cntR - __popc(br & lt));
        S.idx(np)[dst] = (uint16_t)j;
      }
      cntL += __popc(bl);
      cntR += __popc(br);
    }
    nr = __any_sync(full, nr);
  }
  __syncwarp();
  if (lane == 0) note_event<T, D>(S, b, kRechecked | cut.near | (nr ? kNearCut : 0u));
  const bool degenerate = !cut.leaf && (cntL == 0 || cntL == m);
  unsigned counts = 0u;
  if (cut.leaf || degenerate) {
    const uint16_t *fx = S.idx(cut.leaf ? par : np);
    const int h = head_code(m);
    for (int i = lane; i < m; i += 32) mark_final<T, D>(S, b + i, fx[b + i], i == 0 ? h : 0);
    counts = 1u | (degenerate ? 8u : 0u);
  } else if (lane == 0) {
    const unsigned lv = push_set<T, D>(err, S, b, cntL, np) + push_set<T, D>(err, S, b + cntL,
                                                                          m - cntL, np);
    counts = lv | 4u | ((unsigned)m << 8);
  }
  __syncwarp();
  return counts;
}

template <typename T, int D, bool VAR>
__device__ __forceinline__ void exact_one(const Problem &P, const WarpTile<T, D> &S, int b,
                                          int m, int par, int lane, Counters &cnt) {
  const unsigned r = exact_set<T, D, VAR>(S, P.err, b, m, par, lane);
  if (lane == 0) {
    cnt.leaves += r & 3u;
    cnt.splits += (r >> 2) & 1u;
    cnt.degenerate += (r >> 3) & 1u;
    cnt.depth += r >> 8;
  }
}

// the sets of this warp marked in `pend` (a bit at a lane holding the set's
// record `rec`), one at a time in FP64 (exact_set)
template <typename T, int D, bool VAR>
__device__ __forceinline__ void exact_sets(const Problem &P, const WarpTile<T, D> &S,
                                           unsigned pend, uint32_t rec, int lane,
                                           Counters &cnt) {
  while (pend) {
    const int src = __ffs(pend) - 1;
    pend &= pend - 1u;
    const uint32_t r = __shfl_sync(0xffffffffu, rec, src);
    exact_one<T, D, VAR>(P, S, rec_begin(r), rec_len(r), rec_par(r), lane, cnt);
  }
}

// one round of a class c >= 1 for this warp: kw <= 32/G subsets, G = 2^lg
// lanes each (G >= 2^(c-1)); rec is the record of the lane's group (read
// before the round).
// Returns the lanes whose set needs the FP64 recheck (exact_sets).
template <typename T, int D, bool VAR, int TEAM>
__device__ unsigned group_round(const Problem &P, const WarpTile<T, D> &S, const int32_t *perm,
                                int64_t gb, int lg, int lane, Counters &cnt, int kw,
                                uint32_t rec) {
  constexpr bool kF = sizeof(T) == 4;
  const unsigned full = 0xffffffffu;
  const int G = 1 << lg;
  const int gid = lane >> lg, gl = lane & (G - 1);
  const bool act = gid < kw && check_index(P.check, P.err,
                                           rec_len(rec) >= 2 && rec_begin(rec) + rec_len(rec) <= S.cap,
                                           kChkRecord, rec_begin(rec));
  const int b = rec_begin(rec), m = act ? rec_len(rec) : 0, par = rec_par(rec);
  const uint16_t *ix = S.idx(par);

  // Steps 1-2: moments about the set's first particle
  T s[D];
  {
    const int j0 = act ? ix[b] : 0;
#pragma unroll
    for (int l = 0; l < D; ++l) s[l] = S.col(l)[j0];
  }
  Moments<T, D> M;
  M.zero();
  int run = (m + G - 1) >> lg;
  if (TEAM >= 8 && kF && G == 32 && m > kRunBlock * 32) {
    // sets above 1024 particles (large tiles only): FP32 runs of at most
    // kRunBlock terms, each folded exactly into the compensated sums
    accumulate_blocked<T, D>(M, S, ix, b, m, gl, G, s);
    run = kRunBlock;
  } else {
#pragma unroll 4
    for (int i = gl; i < m; i += G) {
      const int j = ix[b + i];
      if (!check_index(P.check, P.err, j < S.cap, kChkTileIndex, j)) continue;
      T q[D];
#pragma unroll
      for (int l = 0; l < D; ++l) q[l] = S.col(l)[j];
      M.add(S.col(D)[j], q, s);
    }
  }
  __syncwarp();
  M.group_allreduce(G);
  // Steps 3-5
  Cut cut = cut_none();
  if (act) cut = Decider<T, D, VAR>::run(P, M, s, m, run);
  // FP32 storage: a decision too close to call is taken again in FP64
  bool redo = kF && cut.unsure;
  if (cut.near && gl == 0) note_event<T, D>(S, b, cut.near);
  const bool split = act && !cut.leaf && !redo;
  // Step 6: cut by group-masked ballot scan into the other index buffer;
  // nr: some particle in the cut's near band
  const int np = par ^ 1;
  const T *qk = S.col(cut.k);
  int cntL = 0, cntR = 0;
  bool nr = false;
  if (G == 1) {
    // one lane per set: a serial stable-front / reversed-back partition
    if (split)
#pragma unroll 4
      for (int i = 0; i < m; ++i) {
        const int j = ix[b + i];
        if (!check_index(P.check, P.err, j < S.cap, kChkTileIndex, j)) continue;
        const T q = qk[j];
        nr |= Decider<T, D, VAR>::near(q, cut);
        const int dst = Decider<T, D, VAR>::left(q, cut) ? (b + cntL++) : (b + m - 1 - cntR++);
        if (check_index(P.check, P.err, dst >= b && dst < b + m, kChkCutDest, dst))
          S.idx(np)[dst] = (uint16_t)j;
      }
  } else {
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (gid * G));
    const unsigned lt = lanemask_lt();
    const int mmax = __reduce_max_sync(full, split ? (unsigned)m : 0u);
    for (int base = 0; base < mmax; base += G) {
      const int i = base + gl;
      int j = (split && i < m) ? ix[b + i] : 0;
      const bool valid =
          split && i < m && check_index(P.check, P.err, j < S.cap, kChkTileIndex, j);
      if (!valid) j = 0;
      const T q = qk[j];
      const bool lft = valid && Decider<T, D, VAR>::left(q, cut);
      nr |= valid && Decider<T, D, VAR>::near(q, cut);
      const unsigned bl = __ballot_sync(full, lft) & gmask;
      const unsigned br = __ballot_sync(full, valid && !lft) & gmask;
      if (valid) {
        const int dst =
            lft ? (b + cntL + __popc(bl & lt)) : (b + m - 1 - cntR - __popc(br & lt));
        if (check_index(P.check, P.err, dst >= b && dst < b + m, kChkCutDest, dst))
          S.idx(np)[dst] = (uint16_t)j;
      }
      cntL += __popc(bl);
      cntR += __popc(br);
    }
    nr = (__ballot_sync(full, nr) & gmask) != 0u;
  }
  __syncwarp();
  if (nr) {
    if (kF)
      redo = true;  // an FP32 cut value too close to a particle: retake in FP64
    else if (gl == 0)
      note_event<T, D>(S, b, kNearCut);
  }
  const bool degenerate = split && !redo && (cntL == 0 || cntR == 0);
  const bool final_set = act && !redo && (cut.leaf || degenerate);
  const int epar = cut.leaf ? par : np;
  // final sets: final order and head codes (Step 7 sums them up later)
  if (final_set) {
    const int h = head_code(m);
    for (int i = gl; i < m; i += G)
      mark_final<T, D>(S, b + i, S.idx(epar)[b + i], i == 0 ? h : 0);
  }
  if (gl == 0 && act && !redo) {
    if (final_set) {
      cnt.leaves += 1;
      if (degenerate) cnt.degenerate += 1;
    } else {
      cnt.splits += 1;
      cnt.depth += (unsigned long long)m;
      push_child<T, D>(P, S, perm, gb, b, cntL, np, cnt);
      push_child<T, D>(P, S, perm, gb, b + cntL, m - cntL, np, cnt);
    }
  }
  __syncwarp();
  return kF ? __ballot_sync(full, redo && act && gl == 0) : 0u;
}

// A wide round: the (up to TEAM/2) pending sets of the largest class,
// when they would leave warps idle, each get W warps: TEAM halved (rounded
// down) until the sets fit the team (12, 6, 3, 1 for a 12-warp team).
// Moments: each warp sums a strided share, the W partial sums are merged in
// warp order through shared memory.  Cut: warp u of the group takes the
// u-th contiguous segment of the set (32 lanes at a time, conflict-free), a
// first pass counts its V1 members, and a second writes V1 to the front and
// V2 to the back of the range at the offsets of the earlier segments, which
// is the order one warp would write.  An FP32 decision or cut too close to
// call is taken again in FP64 by the group's first warp.  Every warp of the
// team calls this (the idle ones too): it contains CTA barriers.
// Returns true when this warp must take its set's FP64 recheck (exact_set).
template <typename T, int D, bool VAR, int TEAM>
__device__ bool wide_round(const Problem &P, const WarpTile<T, D> &S, const int32_t *perm,
                          int64_t gb, int lane, int wt, int sub, int W, bool act, uint32_t rec,
                          Counters &cnt) {
  constexpr bool kF = sizeof(T) == 4;
  Moments<T, D> *xm = static_cast<Moments<T, D> *>(S.wide);
  int *xc = reinterpret_cast<int *>(xm + kMaxTeam);
  const unsigned full = 0xffffffffu;
  const int wl = wt - sub * W;  // warp within the group
  const int b = rec_begin(rec), m = act ? rec_len(rec) : 0, par = rec_par(rec);
  const uint16_t *ix = S.idx(par);
  // Steps 1-2: moments about the set's first particle
  T s[D];
  {
    const int j0 = act ? ix[b] : 0;
#pragma unroll
    for (int l = 0; l < D; ++l) s[l] = S.col(l)[j0];
  }
  Moments<T, D> M;
  M.zero();
  int run = (m + 32 * W - 1) / (32 * W);
  if (kF && run > kRunBlock) {
    accumulate_blocked<T, D>(M, S, ix, b, m, wl * 32 + lane, 32 * W, s);
    run = kRunBlock;
  } else {
#pragma unroll 4
    for (int i = wl * 32 + lane; i < m; i += 32 * W) {
      const int j = ix[b + i];
      T q[D];
#pragma unroll
      for (int l = 0; l < D; ++l) q[l] = S.col(l)[j];
      M.add(S.col(D)[j], q, s);
    }
  }
  M.warp_allreduce();
  if (lane == 0) xm[wt] = M;
  __syncthreads();
  Cut cut = cut_none();
  if (act) {
    Moments<T, D> Mt = xm[sub * W];
    for (int u = 1; u < W; ++u) Mt.merge(xm[sub * W + u]);
    cut = Decider<T, D, VAR>::run(P, Mt, s, m, run);
  }
  bool redo = kF && cut.unsure;
  if (cut.near && wl == 0 && lane == 0) note_event<T, D>(S, b, cut.near);
  const bool split = act && !cut.leaf && !redo;
  // Step 6: two passes over this warp's segment
  const int np = par ^ 1;
  const T *qk = S.col(cut.k);
  const int seg = ((m + 32 * W - 1) / (32 * W)) * 32;
  const int s0 = min(m, wl * seg), s1 = min(m, s0 + seg);
  const unsigned lt = lanemask_lt();
  int cl = 0;
  bool nr = false;
  if (split)
    for (int i0 = s0; i0 < s1; i0 += 32) {
      const int i = i0 + lane;
      const bool valid = i < s1;
      const T q = qk[ix[b + (valid ? i : 0)]];
      const bool lft = valid && Decider<T, D, VAR>::left(q, cut);
      nr |= valid && Decider<T, D, VAR>::near(q, cut);
      cl += __popc(__ballot_sync(full, lft));
    }
  nr = __any_sync(full, nr);
  if (lane == 0) xc[wt] = cl | (nr ? (1 << 30) : 0);
  __syncthreads();
  int rl = 0, rr = 0, totL = 0;
  bool gnear = false;
  for (int u = 0; u < W; ++u) {
    const int xv = act ? xc[sub * W + u] : 0;
    const int cu = xv & ((1 << 30) - 1);
    gnear |= (xv >> 30) != 0;
    const int nu = min(m, (u + 1) * seg) - min(m, u * seg);
    if (u < wl) {
      rl += cu;
      rr += nu - cu;
    }
    totL += cu;
  }
  if (gnear) {
    if (kF)
      redo = true;
    else if (wl == 0 && lane == 0)
      note_event<T, D>(S, b, kNearCut);
  }
  if (split && !redo) {
    uint16_t *ox = S.idx(np);
    for (int i0 = s0; i0 < s1; i0 += 32) {
      const int i = i0 + lane;
      const bool valid = i < s1;
      const int j = valid ? ix[b + i] : 0;
      const bool lft = valid && Decider<T, D, VAR>::left(qk[j], cut);
      const unsigned bl = __ballot_sync(full, lft);
      const unsigned br = __ballot_sync(full, valid && !lft);
      if (valid) {
        const int dst = lft ? (b + rl + __popc(bl & lt)) : (b + m - 1 - rr - __popc(br & lt));
        ox[dst] = (uint16_t)j;
      }
      rl += __popc(bl);
      rr += __popc(br);
    }
  }
  __syncthreads();
  const bool degenerate = split && !redo && (totL == 0 || totL == m);
  const bool final_set = act && !redo && (cut.leaf || degenerate);
  if (final_set) {
    const uint16_t *fx = S.idx(cut.leaf ? par : np);
    const int h = head_code(m);
    for (int i = wl * 32 + lane; i < m; i += 32 * W)
      mark_final<T, D>(S, b + i, fx[b + i], i == 0 ? h : 0);
  }
  if (act && !redo && wl == 0 && lane == 0) {
    if (final_set) {
      cnt.leaves += 1;
      if (degenerate) cnt.degenerate += 1;
    } else {
      cnt.splits += 1;
      cnt.depth += (unsigned long long)m;
      push_child<T, D>(P, S, perm, gb, b, totL, np, cnt);
      push_child<T, D>(P, S, perm, gb, b + totL, m - totL, np, cnt);
    }
  }
  // redo is the same in every lane of the group's warps
  return kF && act && redo && wl == 0;
}

// one round of two-particle sets for this warp: kw <= 32 of them, one per
// lane; rec is the lane's record (read before the round).  An FP32 decision
// or cut too close to call is taken again in FP64 (exact_set).
template <typename T, int D, bool VAR>
__device__ unsigned pair_round(const Problem &P, const WarpTile<T, D> &S, const int32_t *perm,
                               int64_t gb, int lane, Counters &cnt, int kw, uint32_t rec) {
  constexpr bool kF = sizeof(T) == 4;
  const bool act = lane < kw && check_index(P.check, P.err, rec_begin(rec) + 1 < S.cap,
                                            kChkPair, rec_begin(rec));
  const int b = rec_begin(rec), par = rec_par(rec);
  bool redo = false;
  if (act) {
    const int ja = S.idx(par)[b], jb = S.idx(par)[b + 1];
    T qa[D], qb[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      qa[l] = S.col(l)[ja];
      qb[l] = S.col(l)[jb];
    }
    const T wa = S.col(D)[ja], wb = S.col(D)[jb];
    Cut cut;
    if constexpr (kF) {
      // FP32 storage: the certified two-particle decision (cut by order)
      cut = decide_pair<D, VAR>(P, wa, wb, qa, qb);
    } else {
      // the same sums as the general path takes for two particles
      Moments<T, D> M;
      M.zero();
      M.add(wa, qa, qa);
      M.add(wb, qb, qa);
      cut = Decider<T, D, VAR>::run(P, M, qa, 2, 2);
    }
    T ka = qa[0], kb = qb[0];
#pragma unroll
    for (int l = 0; l < D; ++l)
      if (l == cut.k) {
        ka = qa[l];
        kb = qb[l];
      }
    const bool nr = !kF && !cut.leaf &&
                    (Decider<T, D, VAR>::near(ka, cut) || Decider<T, D, VAR>::near(kb, cut));
    redo = kF && cut.unsure;
    if (!redo) {
      const unsigned ev = cut.near | (nr ? kNearCut : 0u);
      if (ev) note_event<T, D>(S, b, ev);
      bool merged = cut.leaf != 0;
      int first = ja, second = jb;
      if (!merged) {
        // FP32: the smaller value is in V1 (the exact centroid lies between)
        const bool la = kF ? ka < kb : Decider<T, D, VAR>::left(ka, cut);
        const bool lb = kF ? kb < ka : Decider<T, D, VAR>::left(kb, cut);
        if (la == lb) {
          merged = true;  // degenerate cut: the set stays whole
          cnt.degenerate += 1;
        } else if (!la) {
          first = jb;
          second = ja;
        }
      }
      if (merged) {
        mark_final<T, D>(S, b, first, kHeadMerged);
        mark_final<T, D>(S, b + 1, second, 0);
        cnt.leaves += 1;
      } else {
        mark_final<T, D>(S, b, first, kHeadSingle);
        mark_final<T, D>(S, b + 1, second, kHeadSingle);
        cnt.leaves += 2;
        cnt.splits += 1;
        cnt.depth += 2;
      }
    }
  }
  return kF ? __ballot_sync(0xffffffffu, redo) : 0u;
}

// --------------------------------------------------------------- kernel

// Work sources: mode 3 the cells of the tiny class (one-warp teams), mode 0
// the cells of the small class (and larger pass-through cells), mode 1 the
// cells of the large class, mode 2 the pieces of cells that were first cut
// in global memory.
struct UnitSource {
  const int32_t *list;
  const int32_t *count;
  int32_t *next;
  int mode;
};

// one unit: first sorted position, size, depth of its root, cell id
__device__ __forceinline__ void unit_at(const Problem &P, const UnitSource &U, int t, int64_t &gb,
                                        int &n, int &depth0, int &cell) {
  if (U.mode == 2) {
    const int4 pc = P.pieces[t];
    gb = pc.x;
    n = pc.y - pc.x;
    depth0 = pc.z;
    cell = pc.w;
  } else {
    const int c = U.list[t];
    gb = P.cell_begin[c];
    n = P.cell_begin[c + 1] - (int)gb;
    depth0 = 0;
    cell = c;
  }
}

// The float small-cell teams are register-limited: keep 7 CTAs per SM for
// D <= 5 and 6 for D = 6 (what shared memory allows for D = 5 and 6; for
// D <= 4 an eighth CTA would fit but its 64-register limit measured slower);
// the other instances are limited by shared memory.
template <typename T, int D, int TEAM>
constexpr int team_min_blocks() {
  return (sizeof(T) == 4 && TEAM == 4) ? (D <= 5 ? 7 : 6) : 1;
}

template <typename T, int D, int TEAM, bool VAR>
__global__ void __launch_bounds__(32 * TEAM, (team_min_blocks<T, D, TEAM>()))
    team_kernel(Problem P, UnitSource U, int cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int count = *U.count;
  if (count == 0) return;  // an empty class: leave before any other work
  if (timed_out(P.err)) return;
  const int lane = threadIdx.x & 31, wt = threadIdx.x >> 5, tt = threadIdx.x;
  constexpr int kThreads = 32 * TEAM;
  WarpTile<T, D> S;
  int *ctl;
  {
    unsigned char *base = smem_raw;
    S.data = reinterpret_cast<T *>(base);
    S.idx0 = reinterpret_cast<uint16_t *>(S.data + (size_t)(D + 1) * cap);
    const size_t off =
        ((size_t)(D + 1) * cap * sizeof(T) + (size_t)2 * cap * sizeof(uint16_t) + 15) &
        ~size_t(15);
    S.stk0 = reinterpret_cast<uint32_t *>(base + off);
    S.top = reinterpret_cast<int *>(S.stk0 + stacks_entries(cap));
    ctl = S.top + kClasses;
    S.ev = ctl + 1;
    S.soff = reinterpret_cast<uint16_t *>(ctl + 1 + kEvWords);
    {
      const size_t woff =
          ((size_t)(reinterpret_cast<unsigned char *>(S.soff + 2 * kClasses) - base) + 15) &
          ~size_t(15);
      S.wide = base + woff;
    }
    S.cap = cap;
    S.base = P.class_base;
    {
      const size_t doff = ((size_t)(static_cast<unsigned char *>(S.wide) - base) +
                           kMaxTeam * (sizeof(Moments<T, D>) + sizeof(int)) + 15) &
                          ~size_t(15);
      DecideConsts *dk = reinterpret_cast<DecideConsts *>(base + doff);
      if (tt == 0) {
        dk->tol2_x = P.tol2_x;
        dk->tol2_p = P.tol2_p;
        for (int a = 0; a < 3; ++a) dk->L2[a] = P.L2[a];
        dk->dx = P.dx;
        dk->variant = P.variant;
      }
      S.dk = dk;
    }
    if (tt < kClasses) {
      int o = cap / 2;  // classes 0 and 1 share [0, cap / 2)
      for (int c = 2; c < tt; ++c) o += class_capacity(c, cap, S.base);
      S.soff[tt] = (uint16_t)(tt == 0 ? 0 : o);
      S.soff[kClasses + tt] = (uint16_t)class_capacity(tt, cap, S.base);
    }
    for (int i = tt; i < kEvWords; i += kThreads) S.ev[i] = 0;
  }
  const int32_t *perm = (U.mode == 2 || *P.unsorted != 0) ? P.perm : nullptr;
  // ungrouped input: the cells' particles were copied in sorted order into
  // the staging columns (gather_kernel), so a cell reads them contiguously;
  // pieces of big cells still read the inputs through the permutation
  // (recomputed where needed rather than held in a register)
#define PMA_SORTED_COPY (perm != nullptr && U.mode != 2)
  // cells per ticket: kWarpChunk, or kMaxBatch when the class has many cells
  // for the grid (more cells to pack into one tile); one piece or large cell
  const int chunk = (U.mode == 0 || U.mode == 3)
                        ? (count >= (int)gridDim.x * 32 ? kMaxBatch : kWarpChunk)
                        : 1;
  Counters cnt{0u, 0u, 0u, 0ull};
  unsigned long long merged = 0, passed = 0;

  for (;;) {
    if (tt == 0) {
      // once the counter has passed the end, stop without another atomic
      const int seen = *reinterpret_cast<volatile int *>(U.next);
      ctl[0] = seen >= count ? seen : atomicAdd(U.next, chunk);
    }
    __syncthreads();
    const int c0 = ctl[0];
    __syncthreads();
    if (c0 >= count) break;
    const int c1 = min(c0 + chunk, count);
    int t = c0;
    while (t < c1) {
      // the batch: the next units of the chunk that fit the tile together
      // (pass-through cells on the way are copied at once)
      int nb = 0, used = 0;
      while (t < c1 && nb < kMaxBatch) {
        int64_t gb;
        int n, depth0, cell;
        unit_at(P, U, t, gb, n, depth0, cell);
        if (U.mode != 2 && (n <= P.n_min || n == 1)) {
          // Sec. 3 "Input": cells with at most N_min particles are not merged
          for (int i = tt; i < n; i += kThreads) {
            const int src = orig_index(perm, gb, i);
            P.perm_final[gb + i] = src;
            P.head[gb + i] = kHeadSingle;
            if (!PMA_SORTED_COPY) {  // (the sorted copy already sits there)
#pragma unroll
              for (int l = 0; l < D; ++l)
                static_cast<T *>(P.fin[l])[gb + i] = StoreOf<T>::load(P.q[l], src);
              static_cast<T *>(P.fin[D])[gb + i] = StoreOf<T>::load(P.w, src);
            }
          }
          passed += 1;
          ++t;
          continue;
        }
        if (n > cap) {
          if (tt == 0) set_error(P.err, kErrInternal);
          ++t;
          continue;
        }
        if (used + n > cap) break;  // the next batch starts here
        if (tt == 0) {
          S.ev[kEvOff + nb] = used;
          S.ev[kEvN + nb] = n;
          S.ev[kEvGb + nb] = (int)gb;
          S.ev[kEvCell + nb] = cell;
          cnt.depth += (unsigned long long)depth0 * n;
        }
        if (U.mode != 2) merged += 1;
        used += n;
        ++nb;
        ++t;
      }
      if (nb == 0) continue;  // only pass-through cells were left
      if (tt == 0) S.ev[kEvBatchN] = nb;
      if (t < c1 && (!perm || PMA_SORTED_COPY) && tt < D + 1) {
        // the next unit of this chunk: pull its columns into L2 meanwhile
        int64_t nbg;
        int nn, nd, nc;
        unit_at(P, U, t, nbg, nn, nd, nc);
        const int64_t ne = nbg + nn;
        const size_t es = sizeof(T);
        const char *col = static_cast<const char *>(
            PMA_SORTED_COPY ? P.fin[tt] : (tt < D ? P.q[tt] : P.w));
        // the 16-byte-aligned part of the range only: never outside the array
        const uintptr_t a0 = (reinterpret_cast<uintptr_t>(col + nbg * es) + 15) & ~uintptr_t(15);
        const uintptr_t a1 = (reinterpret_cast<uintptr_t>(col + ne * es)) & ~uintptr_t(15);
        if (a1 > a0)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0),
                       "r"((unsigned)(a1 - a0))
                       : "memory");
      }
      __syncthreads();  // the batch table
      bool bad = false;
      for (int u = 0; u < nb; ++u) {
        const int64_t gb = S.ev[kEvGb + u];
        const int n = S.ev[kEvN + u], off = S.ev[kEvOff + u];
        if (PMA_SORTED_COPY) {
#pragma unroll 4
          for (int i = tt; i < n; i += kThreads) {
#pragma unroll
            for (int l = 0; l <= D; ++l) {
              const T x = static_cast<const T *>(P.fin[l])[gb + i];
              bad |= l < D ? !finite_val(x) : (!(x > T(0)) || !finite_val(x));
              S.col(l)[off + i] = x;
            }
            S.idx(0)[off + i] = (uint16_t)(off + i);
          }
        } else {
#pragma unroll 4
          for (int i = tt; i < n; i += kThreads) {
            const int src = orig_index(perm, gb, i);
#pragma unroll
            for (int l = 0; l < D; ++l) {
              const T x = StoreOf<T>::load(P.q[l], src);
              bad |= !finite_val(x);
              S.col(l)[off + i] = x;
            }
            const T w = StoreOf<T>::load(P.w, src);
            bad |= !(w > T(0)) || !finite_val(w);
            S.col(D)[off + i] = w;
            S.idx(0)[off + i] = (uint16_t)(off + i);
          }
        }
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(P.err, kErrInput);
      if (tt < kClasses) S.top[tt] = 0;
      __syncthreads();
      if (tt == 0) {
        for (int u = 0; u < nb; ++u) {
          const int n = S.ev[kEvN + u], off = S.ev[kEvOff + u];
          if (n == 1) {
            // a one-particle piece is final at once
            emit_single<T, D>(P, S, perm, 0, off, off);
            cnt.leaves += 1;
          } else {
            // the units are disjoint subsets of the tile: within every
            // class's capacity together
            const int c = size_class(n, S.base);
            *S.rec(c, S.top[c]) = pack_rec(off, n, 0);
            S.top[c] += 1;
          }
        }
      }
      // rounds: the team pops up to TEAM * 32/G subsets of the largest
      // non-empty class; warp wt takes the wt-th share.  Each lane reads its
      // record before the stack height drops: children pushed in this round
      // may reuse the popped slots.
      for (;;) {
        __syncthreads();
        int c = -1;
#pragma unroll
        for (int k = kClasses - 1; k >= 0; --k)
          if (c < 0 && S.top[k] > 0) c = k;
        if (c < 0) break;
        const int avail = S.top[c];
        if (TEAM >= 8 && c == kClasses - 1 && avail * 2 <= TEAM) {
          // few large sets: several warps per set (wide round).  Only the
          // 8- and 12-warp teams (one or two CTAs per SM) use it: in the 4-warp teams
          // other CTAs fill the idle warps' issue slots, and the extra
          // barriers measured slower.
          int W = TEAM;
          while (W * avail > TEAM) W >>= 1;
          const int sub = wt / W;
          const bool act = sub < avail;
          const uint32_t rec = act ? *S.rec(c, avail - 1 - sub) : 0u;
          __syncthreads();
          if (tt == 0) S.top[c] = 0;
          __syncthreads();
          if (wide_round<T, D, VAR, TEAM>(P, S, perm, 0, lane, wt, sub, W, act, rec, cnt))
            exact_sets<T, D, VAR>(P, S, 1u, rec, lane, cnt);
          continue;
        }
        // G = 2^lg lanes per set: the class's own, or (when the handle asks
        // for it) more while the team still takes every pending set of the
        // class in this round
        int lg = c == 0 ? 0 : c - 1;
        if (c >= 1 && P.widen_groups)
          while (lg < 5 && TEAM * (32 >> (lg + 1)) >= avail) ++lg;
        const int per = 32 >> lg;
        const int k = min(avail, TEAM * per);
        const int kw = max(0, min(per, k - wt * per));
        const int base = avail - 1 - wt * per;
        uint32_t rec = 0u;
        if (kw > 0) {
          const int gid = lane >> lg;
          if (gid < kw) rec = *S.rec(c, base - gid);
        }
        __syncthreads();
        if (tt == 0) S.top[c] = avail - k;
        __syncthreads();
        if (kw > 0) {
          unsigned pend;
          if (c == 0)
            pend = pair_round<T, D, VAR>(P, S, perm, 0, lane, cnt, kw, rec);
          else
            pend = group_round<T, D, VAR, TEAM>(P, S, perm, 0, lg, lane, cnt, kw, rec);
          // FP32 storage: the rare FP64 rechecks, by the whole warp, after
          // its share of the round
          if (sizeof(T) == 4 && pend) exact_sets<T, D, VAR>(P, S, pend, rec, lane, cnt);
        }
        __syncwarp();
      }
      // each unit in final order: permutation, head bytes, staged particles
      for (int u = 0; u < nb; ++u) {
        const int64_t gb = S.ev[kEvGb + u];
        const int n = S.ev[kEvN + u], off = S.ev[kEvOff + u];
        for (int i = tt; i < n; i += kThreads) {
          const int j = S.idx(0)[off + i];
          if (j < off || j >= off + n) {
            // only after an internal failure left a position unmarked
            set_error(P.err, kErrInternal);
            P.perm_final[gb + i] = -1;
            P.head[gb + i] = 0;
            continue;
          }
          if (!check_index(P.check, P.err, gb + i < P.n, kChkStage, gb + i)) continue;
          P.perm_final[gb + i] = orig_index(perm, gb, j - off);
          P.head[gb + i] = (uint8_t)S.idx(1)[off + i];
          stage<T, D>(P, S, gb + i, j);
        }
      }
      __syncthreads();
      if (tt == 0) {
        // each unit's near-tie bits, into its cell's word
        for (int u = 0; u < nb; ++u) {
          const unsigned f = (unsigned)S.ev[kEvBits + u];
          if (f == 0u) continue;
          S.ev[kEvBits + u] = 0;
          if (atomicOr(&P.cell_flags[S.ev[kEvCell + u]], f) == 0u)
            atomicAdd(&P.stats[kStCellsFlagged], 1ull);
        }
      }
    }
  }
  if (tt == 0) {
    const int kinds[4] = {kStNearStop, kStNearArgmax, kStNearCut, kStRecheck};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (S.ev[1 + k]) atomicAdd(&P.stats[kinds[k]], (unsigned long long)S.ev[1 + k]);
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    cnt.leaves += __shfl_xor_sync(0xffffffffu, cnt.leaves, m);
    cnt.depth += __shfl_xor_sync(0xffffffffu, cnt.depth, m);
    cnt.splits += __shfl_xor_sync(0xffffffffu, cnt.splits, m);
    cnt.degenerate += __shfl_xor_sync(0xffffffffu, cnt.degenerate, m);
  }
  if (lane == 0) {
    if (cnt.leaves) atomicAdd(&P.stats[kStLeaves], (unsigned long long)cnt.leaves);
    if (cnt.depth) atomicAdd(&P.stats[kStDepth], cnt.depth);
    if (cnt.splits) atomicAdd(&P.stats[kStSplits], (unsigned long long)cnt.splits);
    if (cnt.degenerate) atomicAdd(&P.stats[kStDegenerate], (unsigned long long)cnt.degenerate);
    if (wt == 0 && merged) atomicAdd(&P.stats[kStCellsMerged], merged);
    if (wt == 0 && passed) atomicAdd(&P.stats[kStCellsPass], passed);
  }
}
#undef PMA_SORTED_COPY

// ----------------------------------------------------------------- launch

template <typename T>
static size_t team_smem_t(int D, int cap) {
  switch (D) {
    case 2: return warp_region_bytes<T, 2>(cap);
    case 3: return warp_region_bytes<T, 3>(cap);
    case 4: return warp_region_bytes<T, 4>(cap);
    case 5: return warp_region_bytes<T, 5>(cap);
    default: return warp_region_bytes<T, 6>(cap);
  }
}

template <typename T, int D, int TEAM, bool VAR>
static cudaError_t launch_team_t(const Problem &P, const UnitSource &U, int cap, int grid,
                                 cudaStream_t st) {
  if (cap > kMaxCapW) return cudaErrorInvalidValue;
  const size_t smem = warp_region_bytes<T, D>(cap);
  // raise the dynamic shared-memory limit once per device (so that calls
  // captured into a graph after a first eager call make no attribute change)
  static int limit_set[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || (int)smem > limit_set[dev]) {
    e = cudaFuncSetAttribute(team_kernel<T, D, TEAM, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) limit_set[dev] = (int)smem;
  }
  team_kernel<T, D, TEAM, VAR><<<grid, 32 * TEAM, smem, st>>>(P, U, cap);
  return cudaGetLastError();
}

// CTAs of one team kernel instance resident per SM at tile size cap (its
// registers and shared memory), from the CUDA occupancy calculator; 1 when
// it cannot tell.  The shared-memory limit is first raised to the opt-in
// maximum (the launches only ever raise it further for their own tiles).
template <typename T, int D, int TEAM>
static int team_blocks_t(int cap, int smem_optin) {
  const size_t smem = warp_region_bytes<T, D>(cap);
  if (cudaFuncSetAttribute(team_kernel<T, D, TEAM, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin) != cudaSuccess)
    return 1;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, team_kernel<T, D, TEAM, false>, 32 * TEAM,
                                                    smem) != cudaSuccess)
    return 1;
  return b < 1 ? 1 : b;
}

template <typename T, int TEAM>
static int team_blocks_d(int D, int cap, int smem_optin) {
  switch (D) {
    case 2: return team_blocks_t<T, 2, TEAM>(cap, smem_optin);
    case 3: return team_blocks_t<T, 3, TEAM>(cap, smem_optin);
    case 4: return team_blocks_t<T, 4, TEAM>(cap, smem_optin);
    case 5: return team_blocks_t<T, 5, TEAM>(cap, smem_optin);
    default: return team_blocks_t<T, 6, TEAM>(cap, smem_optin);
  }
}

template <typename T, int TEAM, bool VAR>
static cudaError_t launch_team_d(const Problem &P, const UnitSource &U, int cap, int grid,
                                 cudaStream_t st) {
  switch (P.D) {
    case 2: return launch_team_t<T, 2, TEAM, VAR>(P, U, cap, grid, st);
    case 3: return launch_team_t<T, 3, TEAM, VAR>(P, U, cap, grid, st);
    case 4: return launch_team_t<T, 4, TEAM, VAR>(P, U, cap, grid, st);
    case 5: return launch_team_t<T, 5, TEAM, VAR>(P, U, cap, grid, st);
    default: return launch_team_t<T, 6, TEAM, VAR>(P, U, cap, grid, st);
  }
}

// all team launches of one decision build (precision, team size, D)
template <bool VAR>
static cudaError_t launch_team_build(const Problem &P, const UnitSource &U, int mixed,
                                     int team, int cap, int grid, cudaStream_t st) {
  if (team == 1)
    return mixed ? launch_team_d<float, 1, VAR>(P, U, cap, grid, st)
                 : launch_team_d<double, 1, VAR>(P, U, cap, grid, st);
  if (team == 4)
    return mixed ? launch_team_d<float, 4, VAR>(P, U, cap, grid, st)
                 : launch_team_d<double, 4, VAR>(P, U, cap, grid, st);
  // 12-warp teams in the paper's-rule build only (the variant build keeps
  // 8-warp teams for large cells: fewer instances to compile)
  if constexpr (!VAR) {
    if (team == 12)
      return mixed ? launch_team_d<float, 12, VAR>(P, U, cap, grid, st)
                   : launch_team_d<double, 12, VAR>(P, U, cap, grid, st);
  }
  return mixed ? launch_team_d<float, 8, VAR>(P, U, cap, grid, st)
               : launch_team_d<double, 8, VAR>(P, U, cap, grid, st);
}

// the build with run-time decision variants (warp_var.cu)
cudaError_t launch_team_variants(const Problem &P, const UnitSource &U, int mixed, int team,
                                 int cap, int grid, cudaStream_t st);

}  // namespace pma
