// Single-pass exclusive prefix over tiles with decoupled look-back: a tile
// publishes its own count, then walks back over its predecessors until it
// meets one whose inclusive prefix is known.  Tiles are numbered by an atomic
// ticket, so every predecessor belongs to a CTA that is already running.
// The walk gives up after a bounded time, sets kErrTimeout and returns.
#pragma once

#include <cstdint>

#include "pma_device.cuh"

namespace pma {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Called by one thread of the tile; returns the exclusive prefix of `tile`.
// The status word of tile t is status[t * stride] (several independent scans
// can interleave their words).
__device__ inline long long tile_exclusive_prefix(unsigned long long *status, int tile,
                                                  long long aggregate, unsigned *err,
                                                  int stride = 1,
                                                  unsigned long long wait_ns = kWaitNs) {
  if (tile == 0) {
    st_release_u64(&status[0], kFlagInc | (unsigned long long)aggregate);
    return 0;
  }
  st_release_u64(&status[(size_t)tile * stride], kFlagAgg | (unsigned long long)aggregate);
  long long prefix = 0;
  int t = tile - 1;
  unsigned long long t0 = 0;
  while (t >= 0) {
    unsigned long long s = ld_acquire_u64(&status[(size_t)t * stride]);
    unsigned long long f = s >> 62;
    if (f == 0) {
      unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > wait_ns) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(64);
      continue;
    }
    prefix += (long long)(s & kValMask);
    if (f == 2) break;
    --t;
  }
  st_release_u64(&status[(size_t)tile * stride],
                 kFlagInc | (unsigned long long)(prefix + aggregate));
  return prefix;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// As tile_exclusive_prefix, for a caller that reads nothing else its
// predecessors wrote (only their status words): the walk loads the words of
// kLookAhead predecessors at once (relaxed loads, so they are in flight
// together) and sums them in order up to the first inclusive prefix, so a
// long walk costs about 1/kLookAhead of the round trips.
constexpr int kLookAhead = 8;

__device__ inline long long tile_exclusive_prefix_batched(unsigned long long *status, int tile,
                                                          long long aggregate, unsigned *err,
                                                          int stride, unsigned long long wait_ns) {
  if (tile == 0) {
    st_release_u64(&status[0], kFlagInc | (unsigned long long)aggregate);
    return 0;
  }
  st_release_u64(&status[(size_t)tile * stride], kFlagAgg | (unsigned long long)aggregate);
  long long prefix = 0;
  int t = tile - 1;  // newest predecessor not yet summed
  unsigned long long t0 = 0;
  while (t >= 0) {
    unsigned long long sv[kLookAhead];
#pragma unroll
    for (int k = 0; k < kLookAhead; ++k)
      sv[k] = t - k >= 0 ? ld_relaxed_u64(&status[(size_t)(t - k) * stride]) : kFlagInc;
    int used = 0;
    bool done = false, stalled = false;
#pragma unroll
    for (int k = 0; k < kLookAhead; ++k) {
      if (done || stalled) continue;
      const unsigned long long f = sv[k] >> 62;
      if (f == 0) {
        stalled = true;
        continue;
      }
      prefix += (long long)(sv[k] & kValMask);
      ++used;
      if (f == 2) done = true;
    }
    if (done) break;
    t -= used;
    if (stalled) {
      const unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > wait_ns) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(64);
    }
  }
  st_release_u64(&status[(size_t)tile * stride],
                 kFlagInc | (unsigned long long)(prefix + aggregate));
  return prefix;
}

// Warp-wide version: called by all 32 lanes of one warp; examines 32
// predecessors per step.  Returns the exclusive prefix of `tile` in every lane.
// `publish` = false withholds this tile's status words (used only by the
// failure-detection test: the tiles after it wait until wait_ns and report
// kErrTimeout).
__device__ inline long long warp_exclusive_prefix(unsigned long long *status, int tile,
                                                  long long aggregate, unsigned *err,
                                                  unsigned long long wait_ns = kWaitNs,
                                                  bool publish = true) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0 && publish) st_release_u64(&status[0], kFlagInc | (unsigned long long)aggregate);
    return 0;
  }
  if (lane == 0 && publish) st_release_u64(&status[tile], kFlagAgg | (unsigned long long)aggregate);
  long long prefix = 0;
  int t = tile - 1;  // newest predecessor not yet summed
  unsigned long long t0 = 0;
  while (t >= 0) {
    const int q = t - lane;
    unsigned long long sv = q >= 0 ? ld_acquire_u64(&status[q]) : (kFlagInc | 0ull);
    const unsigned long long f = sv >> 62;
    // lanes up to the nearest inclusive prefix must all be ready
    const unsigned inc = __ballot_sync(0xffffffffu, f == 2);
    const int stop = inc ? (__ffs(inc) - 1) : 31;  // lane holding the inclusive (or last)
    const unsigned notready = __ballot_sync(0xffffffffu, f == 0) & ((2u << stop) - 1u);
    if (notready) {
      unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > wait_ns) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(32);
      continue;
    }
    long long v = (lane <= stop) ? (long long)(sv & kValMask) : 0;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    prefix += v;
    if (inc) break;
    t -= 32;
  }
  if (lane == 0 && publish)
    st_release_u64(&status[tile], kFlagInc | (unsigned long long)(prefix + aggregate));
  return prefix;
}

// true once a bounded wait of this call gave up: the kernels after it then
// return at once (their inputs are incomplete), and the call reports
// PMA_ERR_TIMEOUT
__device__ __forceinline__ bool timed_out(const unsigned *err) {
  return (*reinterpret_cast<const volatile unsigned *>(err) & kErrTimeout) != 0u;
}

// exclusive scan of one int per thread across the CTA (blockDim <= 1024);
// `warp_sums` holds 32 ints of shared memory; returns the block total in *total
__device__ inline int block_exclusive_scan(int v, int *warp_sums, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  int before = warp > 0 ? warp_sums[warp - 1] : 0;
  *total = warp_sums[nw - 1];
  __syncthreads();
  return before + x - v;
}

}  // namespace pma
