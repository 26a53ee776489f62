// Device-side building blocks of the Voronoi merge (Sec. 3, Steps 1-7 of
// Luu, Tueckmantel & Pukhov, arXiv:1504.00636).
//
// Notation follows the paper: a subset V has weight W = sum w, centroid
// (X, P) = sum w q / W, per-axis standard deviation sigma and coefficient of
// variation Delta (Eqs. cv_x, cv_p).  Moments are accumulated about a shift
// s (the subset's first particle): W, m1_l = sum w (q_l - s_l) and
// m2_l = sum w (q_l - s_l)^2, so that
//     W^2 var_l = m2_l W - m1_l^2,     W Q_l = s_l W + m1_l.
// Step 3 and Step 4 then need no square root or division:
//     Delta_l <= T    <=>  W^2 var_l <= T^2 den_l,
//     Delta_a > Delta_b  <=>  (W^2 var_a) den_b > (W^2 var_b) den_a,
// with den_l = (L_l W)^2 on a position axis and (W Q_l)^2 on a momentum axis
// (den = 0 and var > 0 is Delta = +infinity; var = 0 is Delta = 0).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pma {

constexpr int kMaxD = 6;

// error bits of the device status word
constexpr unsigned kErrInput = 1u;
constexpr unsigned kErrInternal = 2u;
constexpr unsigned kErrTimeout = 4u;

// counters kept on the device (indices into Problem::stats)
enum Stat {
  kStCellsMerged = 0,
  kStCellsPass,
  kStSplits,
  kStLeaves,
  kStDepth,
  kStDegenerate,
  kStBig,
  kStSorted,
  kStCount
};

// head byte of a final position: 0 inside a final set, 1 first (only)
// particle of a one-particle set, m (2..254) first particle of a merged set of
// m particles, 255 first particle of a merged set of 255 or more
constexpr uint8_t kHeadSingle = 1;
constexpr uint8_t kHeadMerged = 2;
constexpr uint8_t kHeadLong = 255;
__host__ __device__ __forceinline__ uint8_t head_code(int m) {
  return (uint8_t)(m < 255 ? m : 255);
}

// decision variants (Problem::variant bits)
constexpr int kVarNormalized = 2;  // Step 4 on Delta_l / T_l
constexpr int kVarPNorm = 4;       // Eq. cv_p with |P| of the mean momentum vector

struct Problem {
  int32_t n_cells;
  int32_t dx;
  int32_t D;
  int32_t n_min;
  int32_t variant;      // kVarNormalized | kVarPNorm, or 0 for the literal rule
  int32_t cap;          // particles per unit held in shared memory
  const int32_t *unsorted;  // device flag: 0 when cell ids are non-decreasing
  double tol2_x, tol2_p;  // T^2
  double L2[3];           // L^2 per position axis
  float tol2_xf, tol2_pf;
  float L2f[3];
  const void *q[kMaxD];   // input coordinates by axis: positions, then momenta
  const void *w;          // input weights
  const int32_t *cells;   // input cell ids
  const int32_t *cell_begin;  // [n_cells + 1] first sorted position of each cell
  int32_t *perm;          // sorted position -> input index (workspace)
  uint8_t *head;          // [N] head byte per final position
  int32_t *perm_final;    // [N] input index at each final position
  void *fin[kMaxD + 1];   // [D + 1][N] coordinates and weight in final order,
                          // or all null (then the emit step gathers)
  unsigned *err;          // device status word
  unsigned long long *stats;
  // big cells: cells above `cap` are cut in global memory first
  int32_t *big_list;
  int32_t *big_count;
  int32_t *big_next;
  int4 *pieces;           // {begin, end, depth, 0}
  int32_t *piece_count;
  int32_t *perm_tmp;
  int32_t max_pieces;
  int32_t *unit_next;     // ticket counters of the unit kernel, one per mode
  // population classes: cells of at most cap_w particles (and pass-through
  // cells) go one per warp; cells up to cap one per CTA
  int32_t cap_w;
  int32_t *warp_list;
  int32_t *warp_count;
  int32_t *warp_next;
  // tiny cells (at most cap_t particles) go to one-warp teams
  int32_t cap_t;
  int32_t *tiny_list;
  int32_t *tiny_count;
  int32_t *tiny_next;
  int32_t *block_list;
  int32_t *block_count;
};

// ------------------------------------------------------------ accumulators

template <typename T>
struct Acc;

// plain FP64 sum
template <>
struct Acc<double> {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void merge(const Acc &o) { v += o.v; }
  __device__ __forceinline__ void shfl_xor(int m) { v += __shfl_xor_sync(0xffffffffu, v, m); }
  __device__ __forceinline__ double hi() const { return v; }
  __device__ __forceinline__ double value() const { return v; }
};

// compensated FP32 sum in blocks: each lane adds its own short run of terms
// (at most a few dozen) in plain FP32; runs are combined with an error-free
// two-sum whose rounding errors are kept in c.  value = s - c.
template <>
struct Acc<float> {
  float s, c;
  __device__ __forceinline__ void zero() {
    s = 0.f;
    c = 0.f;
  }
  __device__ __forceinline__ void add(float x) { s = __fadd_rn(s, x); }
  __device__ __forceinline__ void add_prod(float a, float b) { s = __fmaf_rn(a, b, s); }
  // exact two-sum of the leading parts, errors folded into c
  __device__ __forceinline__ void merge2(float s2, float c2) {
    float t = __fadd_rn(s, s2);
    float bp = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    c = __fsub_rn(__fadd_rn(c, c2), e);
    s = t;
  }
  __device__ __forceinline__ void merge(const Acc &o) { merge2(o.s, o.c); }
  __device__ __forceinline__ void shfl_xor(int m) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, m);
    float c2 = __shfl_xor_sync(0xffffffffu, c, m);
    merge2(s2, c2);
  }
  __device__ __forceinline__ float hi() const { return s; }
  __device__ __forceinline__ float lo() const { return -c; }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename T, int D>
struct Moments {
  Acc<T> W;
  Acc<T> m1[D];
  Acc<T> m2[D];
  __device__ __forceinline__ void zero() {
    W.zero();
#pragma unroll
    for (int l = 0; l < D; ++l) {
      m1[l].zero();
      m2[l].zero();
    }
  }
  __device__ __forceinline__ void add(T w, const T *q, const T *s) {
    W.add(w);
#pragma unroll
    for (int l = 0; l < D; ++l) {
      T d = q[l] - s[l];
      T t = w * d;
      m1[l].add(t);
      m2[l].add_prod(t, d);
    }
  }
  __device__ __forceinline__ void merge(const Moments &o) {
    W.merge(o.W);
#pragma unroll
    for (int l = 0; l < D; ++l) {
      m1[l].merge(o.m1[l]);
      m2[l].merge(o.m2[l]);
    }
  }
  // sum over aligned groups of g lanes (g a power of two, <= 32)
  __device__ __forceinline__ void group_allreduce(int g) {
    for (int m = g >> 1; m >= 1; m >>= 1) {
      W.shfl_xor(m);
#pragma unroll
      for (int l = 0; l < D; ++l) {
        m1[l].shfl_xor(m);
        m2[l].shfl_xor(m);
      }
    }
  }
  __device__ __forceinline__ void warp_allreduce() {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      W.shfl_xor(m);
#pragma unroll
      for (int l = 0; l < D; ++l) {
        m1[l].shfl_xor(m);
        m2[l].shfl_xor(m);
      }
    }
  }
};

// ------------------------------------------------------------- decisions

struct Cut {
  int leaf;   // Step 3 stop test passed
  int k;      // Step 4 axis
  double Q;   // Step 5 centroid coordinate on axis k (FP64)
  float Qt;   // largest float <= Q (FP32 storage: q <= Q  <=>  q <= Qt)
};

// Steps 3-5 in FP64 from moment values (W, m1, m2 about the shift s).
// VAR = false: the paper's rule only; true: the variants in P.variant.
template <int D, bool VAR = true>
__device__ __forceinline__ Cut decide_fp64(const Problem &P, double W, const double *m1,
                                           const double *m2, const double *s) {
  Cut c;
  c.leaf = 1;
  c.k = 0;
  const bool normd = VAR && (P.variant & kVarNormalized) != 0;
  const bool pnorm = VAR && (P.variant & kVarPNorm) != 0;
  double bestV = -1.0, bestDen = 1.0;
  double W2 = W * W;
  double denN = 0.0;  // (W |P|)^2 for the momentum-norm variant
  if (pnorm) {
#pragma unroll
    for (int l = 0; l < D; ++l)
      if (l >= P.dx) {
        const double Pw = fma(s[l], W, m1[l]);
        denN = fma(Pw, Pw, denN);
      }
  }
#pragma unroll
  for (int l = 0; l < D; ++l) {
    double V = fmax(fma(m2[l], W, -m1[l] * m1[l]), 0.0);
    double den, tol2;
    if (l < P.dx) {
      den = P.L2[l] * W2;
      tol2 = P.tol2_x;
    } else {
      double Pw = fma(s[l], W, m1[l]);
      den = pnorm ? denN : Pw * Pw;
      tol2 = P.tol2_p;
    }
    // Delta_l <= T  <=>  V <= T^2 den  (den = 0: only V = 0 passes)
    if (!(V <= tol2 * den)) c.leaf = 0;
    // first maximum of V / kden = Delta_l^2, or (Delta_l / T_l)^2 for the
    // normalised variant; kden = 0 is +infinity, and V = 0 counts as 0
    double kden = normd ? den * tol2 : den;
    if (V == 0.0) kden = 1.0;
    if (bestV < 0.0 || V * bestDen > bestV * kden) {
      bestV = V;
      bestDen = kden;
      c.k = l;
    }
  }
  double Q = s[0];
#pragma unroll
  for (int l = 0; l < D; ++l)
    if (l == c.k) Q = s[l] + m1[l] / W;
  c.Q = Q;
  c.Qt = __double2float_rd(Q);
  return c;
}

// Step 3-5 for compensated FP32 moments.  The stop test and the axis choice
// are evaluated in FP32 with an error bound; when a comparison is closer
// than the bound the FP64 evaluation of the same sums decides.  The cut value
// is computed as a double-float (hi + lo) and rounded down to float.
template <int D, bool VAR = true>
__device__ __forceinline__ Cut decide_mixed(const Problem &P, const Moments<float, D> &M,
                                            const float *s) {
  const float g = 1.0f / (1 << 17);  // error budget relative to the terms
  float W = M.W.hi();
  float W2 = W * W;
  Cut c;
  c.leaf = 1;
  c.k = 0;
  bool sure = true;
  const bool normd = VAR && (P.variant & kVarNormalized) != 0;
  const bool pnorm = VAR && (P.variant & kVarPNorm) != 0;
  // momentum-norm variant: (W |P|)^2 and its error bound
  float denN = 0.f, eDN = 0.f;
  if (pnorm) {
#pragma unroll
    for (int l = 0; l < D; ++l)
      if (l >= P.dx) {
        const float m1 = M.m1[l].hi();
        const float Pw = fmaf(s[l], W, m1);
        const float eP = g * (fabsf(s[l] * W) + fabsf(m1));
        denN = fmaf(Pw, Pw, denN);
        eDN += 2.f * fabsf(Pw) * eP + eP * eP;
      }
    eDN += g * denN;
  }
  // first and second largest V / kden: Delta^2 (position: V / (L W)^2,
  // momentum: V / (W P)^2), or (Delta / T)^2 for the normalised variant;
  // kden = 0 is +infinity unless V = 0
  float r1 = -1.f, r2 = -1.f;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    float m1 = M.m1[l].hi(), m2 = M.m2[l].hi();
    float a = m2 * W, b = m1 * m1;
    float V = fmaxf(a - b, 0.f);
    float eV = g * (fabsf(a) + b);
    float den, eD, tol2;
    if (l < P.dx) {
      den = P.L2f[l] * W2;
      eD = g * den;
      tol2 = P.tol2_xf;
    } else if (pnorm) {
      den = denN;
      eD = eDN;
      tol2 = P.tol2_pf;
    } else {
      float Pw = fmaf(s[l], W, m1);
      float eP = g * (fabsf(s[l] * W) + fabsf(m1));
      den = Pw * Pw;
      eD = 2.f * fabsf(Pw) * eP + eP * eP + g * den;
      tol2 = P.tol2_pf;
    }
    float f = V - tol2 * den;
    if (fabsf(f) <= eV + tol2 * eD) sure = false;
    if (f > 0.f) c.leaf = 0;
    const float kden = normd ? den * tol2 : den, eK = normd ? eD * tol2 : eD;
    float r;
    if (V == 0.f)
      r = 0.f;
    else if (kden <= eK)
      r = __int_as_float(0x7f800000);
    else
      r = __fdividef(V, kden);
    if (V != 0.f && (V <= eV || kden <= eK)) sure = false;
    if (r > r1) {
      r2 = r1;
      r1 = r;
      c.k = l;
    } else if (r > r2) {
      r2 = r;
    }
  }
  // the runner-up axis within the error budget: FP64 decides
  if (!c.leaf && r2 >= r1 * (1.f - 16.f * g)) sure = false;
  if (!sure) {
    double W64 = M.W.value(), m1d[D], m2d[D], sd[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      m1d[l] = M.m1[l].value();
      m2d[l] = M.m2[l].value();
      sd[l] = (double)s[l];
    }
    Cut d = decide_fp64<D, VAR>(P, W64, m1d, m2d, sd);
    d.Q = 0.0;
    c.leaf = d.leaf;
    c.k = d.k;
  }
  if (c.leaf) return c;
  // cut value Q = s_k + m1_k / W as a double-float, then rounded down
  float sk = s[0], m1h = M.m1[0].hi(), m1l = M.m1[0].lo();
#pragma unroll
  for (int l = 0; l < D; ++l)
    if (l == c.k) {
      sk = s[l];
      m1h = M.m1[l].hi();
      m1l = M.m1[l].lo();
    }
  float Wh = M.W.hi(), Wl = M.W.lo();
  float q0 = __fdiv_rn(m1h, Wh);
  float p = q0 * Wh;
  float pe = fmaf(q0, Wh, -p);
  float rr = ((m1h - p) - pe) + m1l - q0 * Wl;
  float q1 = rr / Wh;
  // (h, e) = TwoSum(sk, q0)
  float h = __fadd_rn(sk, q0);
  float bp = __fsub_rn(h, sk);
  float e = __fadd_rn(__fsub_rn(sk, __fsub_rn(h, bp)), __fsub_rn(q0, bp));
  float lo = __fadd_rn(e, q1);
  float Qh = __fadd_rn(h, lo);
  float Ql = __fsub_rn(lo, __fsub_rn(Qh, h));
  c.Qt = (Ql < 0.f) ? __int_as_float(__float_as_int(Qh) - (Qh > 0.f ? 1 : (Qh < 0.f ? -1 : 0)))
                    : Qh;
  if (Qh == 0.f && Ql < 0.f) c.Qt = -__int_as_float(1);  // largest float below zero
  c.Q = 0.0;  // the float path compares against Qt only
  return c;
}

// FP32 -> FP64 exactly, with integer operations only (no FP64 pipe):
// normal numbers rebias the exponent, subnormals are normalised, zero, inf
// and nan keep their class.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  unsigned long long ee, mm;
  if (e != 0u && e != 0xffu) {
    ee = (unsigned long long)(e + 896u) << 52;
    mm = (unsigned long long)m << 29;
  } else if (e == 0xffu) {
    ee = 0x7ffull << 52;
    mm = (unsigned long long)m << 29;
  } else if (m == 0u) {
    ee = 0ull;
    mm = 0ull;
  } else {
    const int msb = 31 - __clz(m);  // value = m 2^-149 = 1.f 2^(msb - 149)
    ee = (unsigned long long)(msb + 874) << 52;
    mm = (unsigned long long)((m << (23 - msb)) & 0x7fffffu) << 29;
  }
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  return __longlong_as_double((long long)(sign | ee | mm));
}

__device__ __forceinline__ void set_error(unsigned *err, unsigned bit) { atomicOr(err, bit); }

}  // namespace pma
