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
//                  staged members (a product of two floats is exact in FP64).
//                  The tile's staged columns reach shared memory by bulk
//                  asynchronous copies while the CTA scans the head bytes.
// With the energy-conserving option (EC) a head of a set of m >= 2 particles
// takes two output slots: a set of two is copied as it is, and a larger set
// becomes two particles of weight W/2 at X with momenta P + d and P - d that
// also keep the total energy sum w sqrt(1 + |p|^2); see energy_set below.
#include "lookback.cuh"
#include "pma_launch.h"

namespace pma {

constexpr int kEmitThreads = 256;
constexpr int kEmitChunk = 4;  // consecutive positions per thread
constexpr int kEmitTile = kEmitThreads * kEmitChunk;
constexpr int kWarpSet = 32;  // merged sets of at least this many members: one warp each
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

// output slots of a head byte: 1 for a single particle, 1 (or 2 with EC) for
// a merged set, 0 inside a set
template <bool EC>
__device__ __forceinline__ int head_slots(unsigned h) {
  return h == 0u ? 0 : ((EC && h != (unsigned)kHeadSingle) ? 2 : 1);
}

// output slots of the first `upto` of a thread's 4 consecutive positions
template <bool EC>
__device__ __forceinline__ int chunk_slots(unsigned hw, int upto) {
  if (!EC) return __popc(head_mask(hw) & ((1u << upto) - 1u));
  int v = 0;
#pragma unroll
  for (int j = 0; j < kEmitChunk; ++j)
    if (j < upto) v += head_slots<true>((hw >> (8 * j)) & 0xffu);
  return v;
}

// The count kernel takes kCountTiles tiles per CTA and 16 consecutive head
// bytes per thread (one 16-byte load), so that each thread has a useful
// amount of memory in flight: a tile is the 64 threads of two warps.
constexpr int kCountTiles = 4;
constexpr int kCountPer = 16;
static_assert(kEmitTile / kCountPer == 64 && kEmitThreads == 64 * kCountTiles,
              "a tile is two warps of the count kernel");

// output slots of the 16 positions c0 .. c0 + 15 (c0 a multiple of 16; the
// head array is padded to a multiple of 16 bytes, and bytes at n and beyond
// are never counted)
template <bool EC>
__device__ __forceinline__ int slots16(const uint8_t *head, int64_t c0, int64_t n) {
  if (c0 + kCountPer <= n) {
    const uint4 q = *reinterpret_cast<const uint4 *>(head + c0);
    return chunk_slots<EC>(q.x, kEmitChunk) + chunk_slots<EC>(q.y, kEmitChunk) +
           chunk_slots<EC>(q.z, kEmitChunk) + chunk_slots<EC>(q.w, kEmitChunk);
  }
  int v = 0;
#pragma unroll
  for (int k = 0; k < kCountPer / kEmitChunk; ++k)
    v += chunk_slots<EC>(load_heads(head, c0 + k * kEmitChunk, n), kEmitChunk);
  return v;
}

template <bool EC>
__global__ void __launch_bounds__(kEmitThreads) count_kernel(EmitArgs a) {
  __shared__ int s_warp[kEmitThreads / 32];
  if (timed_out(a.err)) return;
  const int64_t c0 = (int64_t)blockIdx.x * (kEmitTile * kCountTiles) +
                     (int64_t)threadIdx.x * kCountPer;
  int v = slots16<EC>(a.head, c0, a.n);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < kCountTiles) {
    const int t = blockIdx.x * kCountTiles + threadIdx.x;
    if (t < a.tiles) a.tile_count[t] = s_warp[2 * threadIdx.x] + s_warp[2 * threadIdx.x + 1];
  }
}

// one CTA: exclusive prefix of the tile counts (four consecutive tiles per
// thread), and the total M
constexpr int kScanPer = 4;
__global__ void __launch_bounds__(kScanCta) tiles_kernel(EmitArgs a) {
  __shared__ int s_warp[32];
  __shared__ long long s_carry;
  if (timed_out(a.err)) return;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < a.tiles; base += kScanCta * kScanPer) {
    const int i0 = base + threadIdx.x * kScanPer;
    int v[kScanPer];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      v[k] = i0 + k < a.tiles ? a.tile_count[i0 + k] : 0;
      sum += v[k];
    }
    int total;
    const int ex = block_exclusive_scan(sum, s_warp, &total);
    long long run = s_carry + ex;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      if (i0 + k < a.tiles) a.tile_prefix[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (a.out_count) *a.out_count = s_carry;
    if (a.out_count2) *a.out_count2 = s_carry;
  }
}

// ---- bulk asynchronous copies global -> shared, completed on an mbarrier

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// dst and src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// waits at most limit_ns; true when the phase completed
__device__ inline bool mbar_wait(uint64_t *bar, unsigned phase, unsigned long long limit_ns) {
  unsigned long long t0 = 0;
  while (!mbar_try_wait(bar, phase)) {
    const unsigned long long now = global_ns();
    if (t0 == 0)
      t0 = now;
    else if (now - t0 > limit_ns)
      return false;
  }
  return true;
}

size_t emit_smem_bytes(int D, int mixed) {
  return (size_t)(D + 1) * kEmitTile * (mixed ? 4 : 8) + (size_t)kEmitTile * 4;
}

// kinetic energy w (sqrt(1 + p^2) - 1) of weight w and momentum squared p2
// (in m c units), in the form without cancellation for small p2
__device__ __forceinline__ double kinetic(double w, double p2) {
  return w * p2 / (sqrt(1.0 + p2) + 1.0);
}

// ---- sums over the members of a merged set
//
// W = sum w and S1_l = sum w q_l over the members r = first, first + stride,
// ... < end (in this tile's shared memory below t0 + cnt, else in global
// memory), in FP64, where a product of two floats is exact.  The FP64 pipe of
// this GPU is slow, so the plain float build forms each product exactly as
// two floats (Ogita, Rump & Oishi's TwoProduct, with an FMA) and adds them
// to a two-float accumulator whose leading part is updated by Knuth's
// error-free TwoSum; every kFold members the accumulator is added to the FP64
// sum.  The result differs from the exact sum by at most about
// kFold^2 2^-48 (below 2.5e-13) of sum |w q| per fold.  The other builds
// (FP64 storage, energy accounting) add in FP64 directly.
constexpr int kFold = 8;

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ void f2_add(F2 &a, float x) {
  const float s = __fadd_rn(a.hi, x);
  const float bp = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}

__device__ __forceinline__ void f2_add_prod(F2 &a, float w, float q) {
  const float p = __fmul_rn(w, q);
  const float e = __fmaf_rn(w, q, -p);  // w q = p + e exactly
  f2_add(a, p);
  a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ void f2_fold(double &d, F2 &a) {
  d += to_f64<float>(a.hi);
  d += to_f64<float>(a.lo);
  a.hi = 0.f;
  a.lo = 0.f;
}

template <typename T, bool EN, int DT>
__device__ __forceinline__ void set_sums(const EmitArgs &a, const T *s_col, int64_t t0, int cnt,
                                         int64_t first, int64_t end, int stride, double &W,
                                         double *S1, double &ein) {
  const int D = DT ? DT : a.dx + a.dp;
  auto val = [&](int l, int64_t r) -> T {
    return r < t0 + cnt ? s_col[l * kEmitTile + (int)(r - t0)]
                        : static_cast<const T *>(a.fin[l])[r];
  };
  W = 0.0;
#pragma unroll
  for (int l = 0; l < kMaxD; ++l) S1[l] = 0.0;
  if constexpr (sizeof(T) == 4 && !EN) {
    F2 fw{0.f, 0.f}, fs[kMaxD];
#pragma unroll
    for (int l = 0; l < kMaxD; ++l) fs[l] = F2{0.f, 0.f};
    int k = 0;
    for (int64_t r = first; r < end; r += stride) {
      const float w = val(D, r);
      f2_add(fw, w);
#pragma unroll
      for (int l = 0; l < kMaxD; ++l)
        if (l < D) f2_add_prod(fs[l], w, val(l, r));
      if (++k == kFold) {
        k = 0;
        f2_fold(W, fw);
#pragma unroll
        for (int l = 0; l < kMaxD; ++l)
          if (l < D) f2_fold(S1[l], fs[l]);
      }
    }
    f2_fold(W, fw);
#pragma unroll
    for (int l = 0; l < kMaxD; ++l)
      if (l < D) f2_fold(S1[l], fs[l]);
  } else {
    for (int64_t r = first; r < end; r += stride) {
      const double w = to_f64<T>(val(D, r));
      W += w;
      double p2 = 0.0;
#pragma unroll
      for (int l = 0; l < kMaxD; ++l)
        if (l < D) {
          const double q = to_f64<T>(val(l, r));
          S1[l] = fma(w, q, S1[l]);
          if (l >= a.dx) p2 = fma(q, q, p2);
        }
      if (EN) ein += kinetic(w, p2);
    }
  }
}

// EC: one final set of m >= 2 members at positions [p, e) of the staged
// arrays (in this tile's shared memory below t0 + cnt, else in global
// memory), first output slot `slot`.  m = 2: both members as they are.
// m >= 3: W/2 at X twice, momenta P + d and P - d with g = E / W,
// E = sum w sqrt(1 + |p|^2): d across P with |d|^2 = g^2 - 1 - |P|^2 along
// the momentum axis of largest sigma_k^2 (1 - Phat_k^2) made orthogonal to P
// (the axis of smallest |P_k| when all are 0); one momentum axis: d along P
// with d^2 = g^2 (g^2 - 1 - P^2) / (g^2 - P^2).  The members map to the first
// slot (a pair: each to its own, the lower input index first).
template <typename T>
__device__ void energy_set(const EmitArgs &a, const T *s_col, const int32_t *s_perm,
                           int64_t t0, int cnt, int64_t p, int64_t e, long long slot,
                           double &ein, double &eout) {
  const int D = a.dx + a.dp;
  auto raw = [&](int l, int64_t r) -> T {
    return r < t0 + cnt ? s_col[l * kEmitTile + (int)(r - t0)]
                        : static_cast<const T *>(a.fin[l])[r];
  };
  auto orig = [&](int64_t r) -> int { return r < t0 + cnt ? s_perm[r - t0] : a.perm_final[r]; };
  if (e - p == 2) {
    const bool swap = orig(p + 1) < orig(p);
    for (int t = 0; t < 2; ++t) {
      const int64_t r = p + (t ^ (int)swap);
      const int o = orig(r);
      if (a.out_index && (unsigned)o < (unsigned)a.n) a.out_index[o] = (int32_t)(slot + t);
      for (int l = 0; l < a.dx; ++l) static_cast<T *>(a.out_pos[l])[slot + t] = raw(l, r);
      double p2 = 0.0;
      for (int l = 0; l < a.dp; ++l) {
        const double q = to_f64<T>(raw(a.dx + l, r));
        a.out_mom[l][slot + t] = q;
        p2 = fma(q, q, p2);
      }
      const double w = to_f64<T>(raw(D, r));
      a.out_w[slot + t] = w;
      if (a.energy) {
        ein += kinetic(w, p2);
        eout += kinetic(w, p2);
      }
    }
    return;
  }
  // pass 1: W, sum w x, sum w p (the momentum axes as 0..2), total energy
  double W = 0.0, E = 0.0, SX[3] = {0.0, 0.0, 0.0}, SP[3] = {0.0, 0.0, 0.0};
  for (int64_t r = p; r < e; ++r) {
    const double w = to_f64<T>(raw(D, r));
    double p2 = 0.0;
    W += w;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (l < a.dx) SX[l] = fma(w, to_f64<T>(raw(l, r)), SX[l]);
      if (l < a.dp) {
        const double q = to_f64<T>(raw(a.dx + l, r));
        SP[l] = fma(w, q, SP[l]);
        p2 = fma(q, q, p2);
      }
    }
    E = fma(w, sqrt(1.0 + p2), E);
    if (a.energy) ein += kinetic(w, p2);
    const int o = orig(r);
    if (a.out_index && (unsigned)o < (unsigned)a.n) a.out_index[o] = (int32_t)slot;
  }
  const double inv = 1.0 / W;
  double Pm[3] = {0.0, 0.0, 0.0}, P2 = 0.0;
#pragma unroll
  for (int l = 0; l < 3; ++l)
    if (l < a.dp) {
      Pm[l] = SP[l] * inv;
      P2 = fma(Pm[l], Pm[l], P2);
    }
  const double g = E * inv;
  double da[3] = {0.0, 0.0, 0.0};
  if (a.dp == 1) {
    const double u2 = g * g * (g * g - 1.0 - P2) / (g * g - P2);
    da[0] = sqrt(fmax(u2, 0.0));
  } else {
    const double nP = sqrt(P2);
    double ph[3] = {0.0, 0.0, 0.0};
    if (nP > 0.0) {
#pragma unroll
      for (int l = 0; l < 3; ++l) ph[l] = Pm[l] / nP;
    }
    // pass 2: sigma_k^2 about the centroid, scored across P
    double var[3] = {0.0, 0.0, 0.0};
    for (int64_t r = p; r < e; ++r) {
      const double w = to_f64<T>(raw(D, r));
#pragma unroll
      for (int l = 0; l < 3; ++l)
        if (l < a.dp) {
          const double dq = to_f64<T>(raw(a.dx + l, r)) - Pm[l];
          var[l] = fma(w * dq, dq, var[l]);
        }
    }
    int k = -1;
    double best = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l)
      if (l < a.dp) {
        const double sc = (var[l] * inv) * (1.0 - ph[l] * ph[l]);
        if (sc > best) {
          best = sc;
          k = l;
        }
      }
    if (k < 0) {
      k = 0;
      double pk = fabs(Pm[0]);
#pragma unroll
      for (int l = 1; l < 3; ++l)
        if (l < a.dp && fabs(Pm[l]) < pk) {
          pk = fabs(Pm[l]);
          k = l;
        }
    }
    double phk = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l)
      if (l == k) phk = ph[l];
    double dir[3], n2 = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      dir[l] = (l == k ? 1.0 : 0.0) - phk * ph[l];
      if (l < a.dp) n2 = fma(dir[l], dir[l], n2);
    }
    const double sc = sqrt(fmax(g * g - 1.0 - P2, 0.0)) / sqrt(n2);
#pragma unroll
    for (int l = 0; l < 3; ++l) da[l] = sc * dir[l];
  }
  const double Wh = 0.5 * W;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const long long s = slot + t;
    a.out_w[s] = Wh;
    double p2 = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (l < a.dx) static_cast<T *>(a.out_pos[l])[s] = (T)(SX[l] * inv);
      if (l < a.dp) {
        const double q = t == 0 ? Pm[l] + da[l] : Pm[l] - da[l];
        a.out_mom[l][s] = q;
        p2 = fma(q, q, p2);
      }
    }
    if (a.energy) eout += kinetic(Wh, p2);
  }
}

// One CTA per tile of 1024 final positions.  One thread starts bulk copies of
// the tile's staged columns and final permutation into shared memory; the
// CTA meanwhile reads the head bytes and scans them into output slots.  The
// positions are then handled in consecutive order across the threads, so the
// output stores of runs of one-particle sets are coalesced.
// CTAs per SM the plain builds are held to (float: 5 for D <= 4, 4 for
// D = 5, 3 for D = 6, what their two-float sums need without spills; FP64: 4,
// what its shared memory allows); the energy-conserving and energy-accounting
// builds take the registers they need
template <typename T, bool EC, bool EN, int DT>
constexpr int emit_min_blocks() {
  return (EC || EN) ? 1 : (sizeof(T) == 4 ? (DT <= 4 ? 5 : (DT == 5 ? 4 : 3)) : 4);
}

// DT: the coordinate count D = dx + dp fixed at compile time (the plain
// float builds, whose two-float sums need registers per axis), or 0 (read
// from the arguments)
template <typename T, bool EC, bool EN, int DT>
__global__ void __launch_bounds__(kEmitThreads, (emit_min_blocks<T, EC, EN, DT>()))
    emit_kernel(EmitArgs a) {
  extern __shared__ __align__(128) unsigned char s_dyn[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_warp[32];
  __shared__ unsigned short s_mask[kEmitThreads];
  __shared__ int s_chunk[kEmitThreads];
  __shared__ __align__(16) uint8_t s_head[kEmitTile];
  __shared__ int s_nmerged;
  __shared__ int2 s_merged[kEmitTile / 2 + 1];  // (offset in tile, output slot)
  if (timed_out(a.err)) return;
  const int tid = threadIdx.x;
  const int D = DT ? DT : a.dx + a.dp;
  const int64_t t0 = (int64_t)blockIdx.x * kEmitTile;
  const int cnt = (int)(a.n - t0 < (int64_t)kEmitTile ? a.n - t0 : (int64_t)kEmitTile);
  T *s_col = reinterpret_cast<T *>(s_dyn);  // column l at s_col[l * kEmitTile]
  int32_t *s_perm = reinterpret_cast<int32_t *>(s_dyn + (size_t)(D + 1) * kEmitTile * sizeof(T));
  if (tid == 0) {
    s_nmerged = 0;
    mbar_init(&s_bar, 1);
    // the staging columns and perm_final hold a multiple of 16 entries, so
    // the rounded-up tail stays inside their allocations
    const unsigned cb = ((unsigned)cnt * (unsigned)sizeof(T) + 15u) & ~15u;
    const unsigned pb = ((unsigned)cnt * 4u + 15u) & ~15u;
    mbar_expect_tx(&s_bar, cb * (unsigned)(D + 1) + pb);
    for (int l = 0; l <= D; ++l)
      bulk_copy_g2s(s_col + (size_t)l * kEmitTile, static_cast<const T *>(a.fin[l]) + t0, cb,
                    &s_bar);
    bulk_copy_g2s(s_perm, a.perm_final + t0, pb, &s_bar);
  }
  const unsigned hw = load_heads(a.head, t0 + (int64_t)tid * kEmitChunk, a.n);
  const unsigned mask = head_mask(hw);
  reinterpret_cast<unsigned *>(s_head)[tid] = hw;
  int total;
  // barriers inside: s_bar is set up
  const int ex = block_exclusive_scan(chunk_slots<EC>(hw, kEmitChunk), s_warp, &total);
  s_mask[tid] = (unsigned short)mask;
  s_chunk[tid] = ex;
  const long long prefix = a.tile_prefix[blockIdx.x];
  const bool sorted = *a.unsorted == 0;
  // grouped input: the cell ids of my positions, loaded while the bulk
  // copies are in flight (ungrouped input reads them through the permutation)
  int32_t cid[kEmitChunk];
#pragma unroll
  for (int j = 0; j < kEmitChunk; ++j) {
    const int off = j * kEmitThreads + tid;
    cid[j] = (sorted && off < cnt) ? a.cells[t0 + off] : 0;
  }
  const bool late = __syncthreads_or(!mbar_wait(&s_bar, 0, kWaitNs));
  if (late) {
    // never leave with copies in flight into this CTA's shared memory
    if (tid == 0) atomicOr(a.err, kErrTimeout);
    mbar_wait(&s_bar, 0, kWaitNs);
    return;
  }
  bool bad = false, internal = false;
  double ein = 0.0, eout = 0.0;  // kinetic energy in and out (EN only)
  int2 mg[kEmitChunk];           // this thread's merged heads: (offset, slot)
  unsigned mmask = 0u;
#pragma unroll
  for (int j = 0; j < kEmitChunk; ++j) {
    const int off = j * kEmitThreads + tid;
    if (off >= cnt) break;
    const int ch = off / kEmitChunk, in = off % kEmitChunk;
    const int h = s_head[off];
    if (EC && h == 0) continue;  // members of merged sets: handled with their set
    long long slot;
    if (EC) {
      slot = prefix + s_chunk[ch] +
             chunk_slots<true>(reinterpret_cast<const unsigned *>(s_head)[ch], in);
    } else {
      const unsigned m = s_mask[ch];
      slot = prefix + s_chunk[ch] + __popc(m & ((2u << in) - 1u)) - 1;
    }
    const int orig = s_perm[off];
    if ((unsigned)orig >= (unsigned)a.n) {
      // a position left unwritten by an earlier failure: never follow it
      internal = true;
      continue;
    }
    if (!check_index(a.check, a.err, slot >= 0 && slot + ((EC && h > 1) ? 1 : 0) < a.n,
                     kChkEmitSlot, slot))
      continue;
    if (a.out_index && (!EC || h == kHeadSingle)) a.out_index[orig] = (int32_t)slot;
    if (!h) continue;
    const int32_t cell_id = sorted ? cid[j] : a.cells[orig];
    a.out_cell[slot] = cell_id;
    if (EC && h != kHeadSingle) a.out_cell[slot + 1] = cell_id;
    if (h == kHeadSingle) {
      // one-particle set: the particle itself (Step 7)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        if (l < a.dx) {
          const T v = s_col[l * kEmitTile + off];
          bad |= !isfinite(v);
          static_cast<T *>(a.out_pos[l])[slot] = v;
        }
      }
      double p2 = 0.0;
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        if (l < a.dp) {
          const T v = s_col[(a.dx + l) * kEmitTile + off];
          bad |= !isfinite(v);
          const double q = to_f64<T>(v);
          a.out_mom[l][slot] = q;
          if (EN) p2 = fma(q, q, p2);
        }
      }
      const T w = s_col[D * kEmitTile + off];
      bad |= !(w > T(0)) || !isfinite(w);
      a.out_w[slot] = to_f64<T>(w);
      if (EN) {
        const double k = kinetic(to_f64<T>(w), p2);
        ein += k;
        eout += k;
      }
    } else {
      // merged set: summed below, densely, by the whole CTA
      mg[j] = make_int2(off, (int)slot);
      mmask |= 1u << j;
    }
  }
  {
    // the merged heads in position order (a scan, not an atomic), so that
    // each set is summed by the same thread on every run
    int total;
    int at = block_exclusive_scan(__popc(mmask), s_warp, &total);
#pragma unroll
    for (int j = 0; j < kEmitChunk; ++j)
      if (mmask & (1u << j)) s_merged[at++] = mg[j];
    if (tid == 0) s_nmerged = total;
  }
  __syncthreads();
  for (int k = tid; k < s_nmerged; k += kEmitThreads) {
    const int off = s_merged[k].x;
    const long long slot_m = s_merged[k].y;
    const int h = s_head[off];
    if (!EC && h >= kWarpSet) continue;  // summed by a warp below
    if (!check_index(a.check, a.err, slot_m + (EC ? 1 : 0) < a.n, kChkEmitSlot, slot_m)) continue;
    // members: the head's count, or (255) every position up to the next head
    int64_t e = t0 + off + h;
    if (h == kHeadLong) {
      e = t0 + off + 1;
      while (e < t0 + cnt && s_head[e - t0] == 0) ++e;
      if (e == t0 + cnt)
        while (e < a.n && a.head[e] == 0) ++e;
    }
    if (e > a.n) {
      internal = true;
      e = a.n;
    }
    if (EC) {
      energy_set<T>(a, s_col, s_perm, t0, cnt, t0 + off, e, slot_m, ein, eout);
      continue;
    }
    double W, S1[kMaxD];
    set_sums<T, EN, DT>(a, s_col, t0, cnt, t0 + off, e, 1, W, S1, ein);
    const double inv = 1.0 / W;
    a.out_w[slot_m] = W;
    double P2 = 0.0;
#pragma unroll
    for (int l = 0; l < kMaxD; ++l) {
      if (l < D) {
        const double v = S1[l] * inv;
        if (l < 3 && l < a.dx) {
          static_cast<T *>(a.out_pos[l])[slot_m] = (T)v;
        } else {
          a.out_mom[l - a.dx][slot_m] = v;
          P2 = fma(v, v, P2);
        }
      }
    }
    if (EN) eout += kinetic(W, P2);
  }
  if (!EC) {
    // sets of kWarpSet or more members: one warp each, lane-strided FP64
    // sums and a fixed butterfly (the same order on every run)
    const unsigned full = 0xffffffffu;
    const int lane = tid & 31;
    for (int k = tid >> 5; k < s_nmerged; k += kEmitThreads / 32) {
      const int off = s_merged[k].x;
      const int h = s_head[off];
      if (h < kWarpSet) continue;  // warp-uniform
      const long long slot_m = s_merged[k].y;
      if (!check_index(a.check, a.err, slot_m < a.n, kChkEmitSlot, slot_m)) continue;  // warp-uniform
      int64_t e = t0 + off + h;
      if (h == kHeadLong) {
        // the next head (or the end), 32 head bytes per step
        int64_t from = t0 + off + 1;
        for (;;) {
          const int64_t i = from + lane;
          const bool hd = i >= a.n || (i < t0 + cnt ? s_head[i - t0] : a.head[i]) != 0;
          const unsigned bh = __ballot_sync(full, hd);
          if (bh) {
            e = from + __ffs(bh) - 1;
            break;
          }
          from += 32;
        }
      }
      if (e > a.n) {
        internal = true;
        e = a.n;
      }
      double W, S1[kMaxD];
      set_sums<T, EN, DT>(a, s_col, t0, cnt, t0 + off + lane, e, 32, W, S1, ein);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        W += __shfl_xor_sync(full, W, o);
#pragma unroll
        for (int l = 0; l < kMaxD; ++l)
          if (l < D) S1[l] += __shfl_xor_sync(full, S1[l], o);
      }
      if (lane == 0) {
        const double inv = 1.0 / W;
        a.out_w[slot_m] = W;
        double P2 = 0.0;
#pragma unroll
        for (int l = 0; l < kMaxD; ++l) {
          if (l < D) {
            const double v = S1[l] * inv;
            if (l < 3 && l < a.dx) {
              static_cast<T *>(a.out_pos[l])[slot_m] = (T)v;
            } else {
              a.out_mom[l - a.dx][slot_m] = v;
              P2 = fma(v, v, P2);
            }
          }
        }
        if (EN) eout += kinetic(W, P2);
      }
    }
  }
  if (EN) {
    // kinetic energy in and out: block sums per tile, then the last CTA to
    // finish adds the tiles up in tile order (the same sum on every run)
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      ein += __shfl_xor_sync(0xffffffffu, ein, o);
      eout += __shfl_xor_sync(0xffffffffu, eout, o);
    }
    __shared__ double s_e[2][kEmitThreads / 32];
    __shared__ int s_last;
    if ((tid & 31) == 0) {
      s_e[0][tid >> 5] = ein;
      s_e[1][tid >> 5] = eout;
    }
    __syncthreads();
    if (tid == 0) {
      double x = 0.0, y = 0.0;
      for (int w = 0; w < kEmitThreads / 32; ++w) {
        x += s_e[0][w];
        y += s_e[1][w];
      }
      a.energy_tiles[blockIdx.x] = x;
      a.energy_tiles[a.tiles + blockIdx.x] = y;
      __threadfence();
      s_last = atomicAdd(a.energy_ticket, 1) == a.tiles - 1;
    }
    __syncthreads();
    if (s_last && tid < 2) {
      __threadfence();
      const volatile double *t = a.energy_tiles + (size_t)tid * a.tiles;
      double v = 0.0;
      for (int k = 0; k < a.tiles; ++k) v += t[k];
      a.energy[tid] = v;
    }
  }
  if (bad) atomicOr(a.err, kErrInput);
  if (internal) atomicOr(a.err, kErrInternal);
}

template <typename T, bool EC, bool EN, int DT = 0>
static cudaError_t launch_emit_t(const EmitArgs &a, cudaStream_t st) {
  const size_t smem = emit_smem_bytes(a.dx + a.dp, sizeof(T) == 4);
  // raise the dynamic shared-memory limit once per device
  static int limit_set[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || (int)smem > limit_set[dev]) {
    e = cudaFuncSetAttribute(emit_kernel<T, EC, EN, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) limit_set[dev] = (int)smem;
  }
  emit_kernel<T, EC, EN, DT><<<a.tiles, kEmitThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_emit(const EmitArgs &a, cudaStream_t st) {
  if (a.tiles <= 0) return cudaSuccess;
  const int count_grid = (a.tiles + kCountTiles - 1) / kCountTiles;
  if (a.ec)
    count_kernel<true><<<count_grid, kEmitThreads, 0, st>>>(a);
  else
    count_kernel<false><<<count_grid, kEmitThreads, 0, st>>>(a);
  tiles_kernel<<<1, kScanCta, 0, st>>>(a);
  // the energy sums are a separate build: they cost the plain path registers
  const bool en = a.energy != nullptr;
  if (a.ec) {
    if (en) return a.mixed ? launch_emit_t<float, true, true>(a, st)
                           : launch_emit_t<double, true, true>(a, st);
    return a.mixed ? launch_emit_t<float, true, false>(a, st)
                   : launch_emit_t<double, true, false>(a, st);
  }
  if (en) return a.mixed ? launch_emit_t<float, false, true>(a, st)
                         : launch_emit_t<double, false, true>(a, st);
  if (!a.mixed) return launch_emit_t<double, false, false>(a, st);
  switch (a.dx + a.dp) {
    case 2: return launch_emit_t<float, false, false, 2>(a, st);
    case 3: return launch_emit_t<float, false, false, 3>(a, st);
    case 4: return launch_emit_t<float, false, false, 4>(a, st);
    case 5: return launch_emit_t<float, false, false, 5>(a, st);
    default: return launch_emit_t<float, false, false, 6>(a, st);
  }
}

}  // namespace pma
