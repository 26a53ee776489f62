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

// VAR = false compiles the paper's rule only; true reads Problem::variant.
// run(P, M, s, m, run): Steps 3-5 for a subset of m particles whose sums were
// formed by lanes of at most `run` terms each.  left(q): Step 5 side V1.
// near(q): q lies in the cut's near band (an FP32 cut may be wrong there; an
// FP64 cut is a near-tie there).
template <typename T, int D, bool VAR = true>
struct Decider;

template <int D, bool VAR>
struct Decider<double, D, VAR> {
  __device__ static __forceinline__ Cut run(const Problem &P, const Moments<double, D> &M,
                                            const double *s, int m, int) {
    double m1[D], m2[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      m1[l] = M.m1[l].v;
      m2[l] = M.m2[l].v;
    }
    return decide_fp64<D, VAR>(P, M.W.v, m1, m2, s, m);
  }
  // order-preserving integer keys of doubles: the cut compares run on the
  // integer pipes, off the (slow) FP64 pipe.  The key order equals the
  // numeric order except that -0 < +0, so the cut value's -0 becomes +0.
  __device__ static __forceinline__ unsigned long long key(double x) {
    const long long b = __double_as_longlong(x);
    return (unsigned long long)(b ^ ((b >> 63) | (long long)0x8000000000000000ull));
  }
  __device__ static __forceinline__ unsigned long long key_cut(double Q) {
    const long long b = __double_as_longlong(Q);
    return b == (long long)0x8000000000000000ull ? 0x8000000000000000ull : key(Q);
  }
  __device__ static __forceinline__ bool left(double q, const Cut &c) {
    return key(q) <= key_cut(c.Q);
  }
  __device__ static __forceinline__ bool near(double q, const Cut &c) {
    const unsigned long long k = key(q);
    return k >= key(c.Qlo) && k <= key(c.Qhi);
  }
};

template <int D, bool VAR>
struct Decider<float, D, VAR> {
  __device__ static __forceinline__ Cut run(const Problem &P, const Moments<float, D> &M,
                                            const float *s, int, int run) {
    return decide_mixed<D, VAR>(P, M, s, run);
  }
  __device__ static __forceinline__ bool left(float q, const Cut &c) { return q <= c.Qt; }
  __device__ static __forceinline__ bool near(float q, const Cut &c) {
    return q >= c.Qlo_f && q <= c.Qhi_f;
  }
};

// FP64 moments of float (or double) particle data about the shift s: the
// recheck of an FP32 decision that was too close to call
template <typename T, int D>
__device__ __forceinline__ void add_exact(Moments<double, D> &M, T w, const T *q, const T *s) {
  double qd[D], sd[D];
#pragma unroll
  for (int l = 0; l < D; ++l) {
    qd[l] = (double)q[l];
    sd[l] = (double)s[l];
  }
  M.add((double)w, qd, sd);
}

// Steps 3-5 in FP64 for a subset of float (or double) data with FP64 moments
template <typename T, int D, bool VAR, class PP = Problem>
__device__ __forceinline__ Cut decide_exact(const PP &P, const Moments<double, D> &M,
                                            const T *s, int m) {
  double m1[D], m2[D], sd[D];
#pragma unroll
  for (int l = 0; l < D; ++l) {
    m1[l] = M.m1[l].v;
    m2[l] = M.m2[l].v;
    sd[l] = (double)s[l];
  }
  return decide_fp64<D, VAR, PP>(P, M.W.v, m1, m2, sd, m);
}

__device__ __forceinline__ int orig_index(const int32_t *perm, int64_t gb, int j) {
  return perm ? perm[gb + j] : (int)(gb + j);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace pma
