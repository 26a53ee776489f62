// Pieces shared by the partition kernels (split.cu, warp.cu): subset
// records, typed loads, the Step 3-5 decision wrappers and small helpers.
#pragma once

#include <cstdint>

#include "pma_device.cuh"

namespace pma {

constexpr int kSmall = 32;

struct Item {
  uint16_t b, e;
  uint8_t par, depth;
  uint16_t pad;
};

template <typename T>
struct StoreOf {
  __device__ static __forceinline__ T load(const void *p, int64_t i) {
    return static_cast<const T *>(p)[i];
  }
};

template <typename T>
__device__ __forceinline__ bool finite_val(T x) {
  return isfinite(x);
}

// ------------------------------------------------------------ cut helpers

// VAR = false compiles the paper's rule only; true reads Problem::variant
template <typename T, int D, bool VAR = true>
struct Decider;

template <int D, bool VAR>
struct Decider<double, D, VAR> {
  __device__ static __forceinline__ Cut run(const Problem &P, const Moments<double, D> &M,
                                            const double *s) {
    double m1[D], m2[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      m1[l] = M.m1[l].v;
      m2[l] = M.m2[l].v;
    }
    return decide_fp64<D, VAR>(P, M.W.v, m1, m2, s);
  }
  __device__ static __forceinline__ bool left(double q, const Cut &c) { return q <= c.Q; }
};

template <int D, bool VAR>
struct Decider<float, D, VAR> {
  __device__ static __forceinline__ Cut run(const Problem &P, const Moments<float, D> &M,
                                            const float *s) {
    return decide_mixed<D, VAR>(P, M, s);
  }
  __device__ static __forceinline__ bool left(float q, const Cut &c) { return q <= c.Qt; }
};

__device__ __forceinline__ int orig_index(const int32_t *perm, int64_t gb, int j) {
  return perm ? perm[gb + j] : (int)(gb + j);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace pma
