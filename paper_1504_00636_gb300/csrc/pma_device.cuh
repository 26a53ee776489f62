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

// Bounds-checked build (compiled with -DPMA_CHECKED, in place of a memory
// sanitizer): an index that a check finds out of range records the site and
// the index of the first such failure of the call in *check, sets
// kErrInternal, and the access it guards is skipped.  In the normal build
// every check is the constant true and compiles to nothing.
enum CheckSite : unsigned {
  kChkRecord = 1,   // a subset record outside the tile
  kChkTileIndex,    // a tile index read from an index buffer
  kChkCutDest,      // a cut's destination outside its subset
  kChkPair,         // a two-particle record outside the tile
  kChkStage,        // a final position outside the workspace
  kChkEmitSlot,     // an output slot outside the output arrays
  kChkCluster       // a position outside the cell being cut in global memory
};

#ifdef PMA_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ bool check_index(unsigned long long *check, unsigned *err, bool ok,
                                            unsigned site, long long index) {
  if (kChecked && !ok) {
    if (check)
      atomicCAS(check, 0ull,
                ((unsigned long long)site << 48) | ((unsigned long long)index & 0xffffffffffffull));
    atomicOr(err, kErrInternal);
  }
  return kChecked ? ok : true;
}

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
  kStNearStop,     // decisions flagged near a tie, by kind
  kStNearArgmax,
  kStNearCut,
  kStRecheck,      // FP32 decisions taken again in FP64
  kStCellsFlagged, // cells with at least one near-tie flag
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
  int64_t n;              // particles of the call
  unsigned long long *check;  // first failed bounds check (checked build)
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
  uint32_t *cell_flags;   // [n_cells] near-tie bits of each cell (zeroed per call)
  // big cells: cells above `cap` are cut in global memory first
  int32_t *big_list;
  int32_t *big_count;
  int32_t *big_next;
  int4 *pieces;           // {begin, end, depth, cell}
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
  // size classes of pending subsets in the team kernels: pairs, then up to
  // class_base particles, up to 2, 4, 8, 16 times class_base, and larger
  int32_t class_base;
  // nonzero: a round of a size class with few pending subsets gives each
  // more lanes (up to a warp) instead of leaving warps of the team idle
  int32_t widen_groups;
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
  __device__ __forceinline__ float val() const { return __fsub_rn(s, c); }
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

// Near-tie bits, recorded per cell: a decision taken within rounding of the
// opposite outcome (Step 3 stop test, Step 4 runner-up axis, Step 5 particle
// at the cut value), and kRechecked when an FP32 decision was too close to
// call and was taken again in FP64 from the particles.
constexpr unsigned kNearStop = 1u;
constexpr unsigned kNearArgmax = 2u;
constexpr unsigned kNearCut = 4u;
constexpr unsigned kRechecked = 8u;
// FP64 near-tie threshold on squared CVs (|Delta^2 - T^2| <= 4e-9 T^2 covers
// |Delta - T| <= 1e-9 T with room for the rounding of either side); the stop
// test uses the exponent-field test near_rel28, at 2^-28 to 2^-27 relative
constexpr double kNearRel2 = 4e-9;

struct Cut {
  int leaf;        // Step 3 stop test passed
  int k;           // Step 4 axis
  int unsure;      // FP32 decision closer than its error bound: retake in FP64
  unsigned near;   // kNearStop | kNearArgmax (FP64 decisions)
  double Q;        // Step 5 centroid coordinate on axis k (FP64 decisions)
  double Qlo, Qhi; // FP64 decisions: particles in [Qlo, Qhi] are cut near-ties
  float Qt;        // largest float <= Q (FP32 storage: q <= Q  <=>  q <= Qt)
  float Qlo_f, Qhi_f;  // FP32 storage: particles in [Qlo_f, Qhi_f] make the cut
                       // uncertain (FP32 decisions) or are near-ties (FP64 ones)
};

__device__ __forceinline__ Cut cut_none() {
  Cut c;
  c.leaf = 1;
  c.k = 0;
  c.unsure = 0;
  c.near = 0u;
  c.Q = c.Qlo = c.Qhi = 0.0;
  c.Qt = c.Qlo_f = c.Qhi_f = 0.f;
  return c;
}

// Approximate MUFU square root and reciprocal (relative error below 2^-21);
// used only inside error bounds, which carry a safety factor for them.
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// |a - b| <= 2^-28 |b| (up to a factor 2), from the exponent fields alone
// (no FP64 arithmetic): the near-tie test of an FP64 comparison
__device__ __forceinline__ bool near_rel28(double diff, double b) {
  const int ed = (__double2hiint(diff) >> 20) & 0x7ff, eb = (__double2hiint(b) >> 20) & 0x7ff;
  return ed <= eb - 28;
}

// Steps 3-5 in FP64 from moment values (W, m1, m2 about the shift s) of a
// subset of m particles.  VAR = false: the paper's rule only; true: the
// variants in P.variant.  Near-tie bits: some |Delta_l^2 - T_l^2| within
// about 2^-28 T_l^2 (stop), the runner-up axis within kNearRel2 of the
// chosen one (argmax).  The cut band is 64 m eps (|s_k| + sqrt(m2_k / W)), which is
// at least 64 m eps (sum w |q_k|) / W by Cauchy-Schwarz.
// The constants of the FP64 decision in a small struct (same member names as
// in Problem) that an out-of-line path can read from shared memory.
struct DecideConsts {
  double tol2_x, tol2_p;
  double L2[3];
  int32_t dx, variant;
};

template <int D, bool VAR = true, class PP = Problem>
__device__ __forceinline__ Cut decide_fp64(const PP &P, double W, const double *m1,
                                           const double *m2, const double *s, int m) {
  Cut c = cut_none();
  const bool normd = VAR && (P.variant & kVarNormalized) != 0;
  const bool pnorm = VAR && (P.variant & kVarPNorm) != 0;
  double bestV = -1.0, bestDen = 1.0, secV = -1.0, secDen = 1.0;
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
    const double t = tol2 * den;
    if (!(V <= t)) c.leaf = 0;
    if (t > 0.0 && near_rel28(V - t, t)) c.near |= kNearStop;
    // first maximum of V / kden = Delta_l^2, or (Delta_l / T_l)^2 for the
    // normalised variant; kden = 0 is +infinity, and V = 0 counts as 0
    double kden = normd ? t : den;
    if (V == 0.0) kden = 1.0;
    if (bestV < 0.0 || V * bestDen > bestV * kden) {
      secV = bestV;
      secDen = bestDen;
      bestV = V;
      bestDen = kden;
      c.k = l;
    } else if (secV < 0.0 || V * secDen > secV * kden) {
      secV = V;
      secDen = kden;
    }
  }
  if (c.leaf) {
    c.near &= kNearStop;
    return c;
  }
  // the runner-up within kNearRel2 of the chosen axis (two infinite scores tie)
  if (secV >= 0.0 && secV * bestDen >= bestV * secDen * (1.0 - kNearRel2)) c.near |= kNearArgmax;
  double Q = s[0], sk = s[0], m2k = m2[0];
#pragma unroll
  for (int l = 0; l < D; ++l)
    if (l == c.k) {
      Q = s[l] + m1[l] / W;
      sk = s[l];
      m2k = m2[l];
    }
  const float tau = 64.0f * (float)m * 2.220446049250313e-16f *
                    (fabsf((float)sk) + sqrtf(fmaxf((float)m2k, 0.f) / (float)W)) * 1.0625f;
  c.Q = Q;
  c.Qlo = Q - (double)tau;
  c.Qhi = Q + (double)tau;
  c.Qt = __double2float_rd(Q);
  c.Qlo_f = __double2float_rd(c.Qlo);
  c.Qhi_f = __double2float_ru(c.Qhi);
  return c;
}

// Steps 3-5 for compensated FP32 moments of a subset of m particles, with a
// certificate.  Every comparison is made in FP32 together with a bound on its
// error: the sums W, m1_l, m2_l are off by at most kk times W, sqrt(W m2_l)
// (which bounds sum w |q - s| by Cauchy-Schwarz) and m2_l, where kk follows
// from the run length `run`, the most terms one lane added in plain FP32
// (the runs are combined exactly).  When a comparison lies within its bound
// the result has unsure = 1, and the caller takes the decision again in FP64
// from the particles themselves; otherwise it is the exact-arithmetic
// decision on the stored values.  The cut value Q = s_k + m1_k / W is formed
// as a double-float and rounded down to float; [Qlo_f, Qhi_f] contains the
// exact Q, so only a particle inside that band can fall on the wrong side.
template <int D, bool VAR = true>
__device__ __forceinline__ Cut decide_mixed(const Problem &P, const Moments<float, D> &M,
                                            const float *s, int run) {
  constexpr float u = 1.0f / (1 << 24);
  const float kk = (float)(run + 8) * (2.0f * u);
  // |V - V_exact| <= cV (a + b): W m2 and m1^2 are off by 2 kk a and by
  // 2 |m1| kk sqrt(a) + ... <= kk (a + b) (AM-GM), plus the roundings
  const float cV = (3.f * kk + 10.f * u) * 1.0625f;
  const float inf = __int_as_float(0x7f800000);
  const float W = M.W.val();
  const float eW = kk * W;
  Cut c = cut_none();
  const bool normd = VAR && (P.variant & kVarNormalized) != 0;
  const bool pnorm = VAR && (P.variant & kVarPNorm) != 0;
  // momentum-norm variant: (W |P|)^2 and its error bound
  float denN = 0.f, eDN = 0.f;
  if (pnorm) {
#pragma unroll
    for (int l = 0; l < D; ++l)
      if (l >= P.dx) {
        const float m1 = M.m1[l].val(), m2 = fmaxf(M.m2[l].val(), 0.f);
        const float sa = sqrt_approx(W * m2) * 1.0001f;
        const float Pw = fmaf(s[l], W, m1);
        const float eP = kk * (fabsf(s[l]) * W + sa) + 3.f * u * (fabsf(s[l] * W) + fabsf(m1));
        denN = fmaf(Pw, Pw, denN);
        eDN = fmaf(2.f * fabsf(Pw) + eP, eP, eDN);
      }
    eDN = (eDN + 8.f * u * denN) * 1.0625f;
  }
  bool sure = true;
  // the axis of the largest score (point estimate), a lower bound of its
  // score and an upper bound of every other axis' score
  float best = -1.f, bestLo = 0.f, bestHi = 0.f, otherHi = 0.f;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const float m1 = M.m1[l].val(), m2 = fmaxf(M.m2[l].val(), 0.f);
    const float a = m2 * W, b = m1 * m1;
    const float V = fmaxf(a - b, 0.f);
    const float eV = cV * (a + b);
    float den, eD, tol2;
    if (l < P.dx) {
      den = P.L2f[l] * (W * W);
      eD = (2.f * kk + 4.f * u) * 1.0625f * den;
      tol2 = P.tol2_xf;
    } else if (pnorm) {
      den = denN;
      eD = eDN;
      tol2 = P.tol2_pf;
    } else {
      const float Pw = fmaf(s[l], W, m1);
      const float sa = sqrt_approx(a) * 1.0001f;  // >= sum w |q - s|
      const float eP = kk * (fabsf(s[l]) * W + sa) + 3.f * u * (fabsf(s[l] * W) + fabsf(m1));
      den = Pw * Pw;
      eD = (fmaf(2.f * fabsf(Pw) + eP, eP, 2.f * u * den)) * 1.0625f;
      tol2 = P.tol2_pf;
    }
    // Step 3: Delta_l <= T  <=>  V <= T^2 den
    const float t = tol2 * den;
    const float f = V - t;
    if (f > 0.f) c.leaf = 0;
    if (!(fabsf(f) > fmaf(tol2, eD, eV) + 2.f * u * (V + t))) sure = false;
    // relative bounds need the sums away from the ends of the FP32 range
    // (a tiny a + b may be an underflowed spread): FP64 decides there
    if (!(a + b >= 1e-24f) || !(a + b <= 1e30f) || !(den <= 1e30f) || (den != 0.f && den < 1e-30f))
      sure = false;
    // Step 4: score V / kden (Delta^2, or (Delta / T)^2 normalised) with
    // bounds: 1 / (k + e) >= (1 - e / k) / k and 1 / (k - e) <= (1 + 2 e / k) / k
    // for e <= k / 2
    const float kden = normd ? t : den, eK = normd ? tol2 * eD : eD;
    const float rk = rcp_approx(kden);
    const float rho = eK * rk * 1.0001f + 4.f * u;
    float r, lo, hi;
    if (kden > 0.f && rho < 0.5f) {
      r = V * rk;
      lo = V > eV ? (V - eV) * rk * (1.f - rho - 8.f * u) : 0.f;
      hi = (V + eV) * rk * (1.f + 2.f * rho + 8.f * u);
    } else {
      r = V == 0.f ? 0.f : (kden > 0.f ? V * rk : inf);
      lo = (V > eV && eK == 0.f && kden == 0.f) ? inf : 0.f;
      hi = (V + eV == 0.f) ? 0.f : inf;
    }
    if (r > best) {
      otherHi = fmaxf(otherHi, bestHi);
      best = r;
      bestLo = lo;
      bestHi = hi;
      c.k = l;
    } else {
      otherHi = fmaxf(otherHi, hi);
    }
  }
  if (!c.leaf && !(bestLo > otherHi)) sure = false;
  if (!sure) {
    c.unsure = 1;
    c.leaf = 0;
    return c;
  }
  if (c.leaf) return c;
  // cut value Q = s_k + m1_k / W as a double-float Qh + Ql
  float sk = s[0], m1h = M.m1[0].hi(), m1l = M.m1[0].lo(), m2k = M.m2[0].val();
#pragma unroll
  for (int l = 0; l < D; ++l)
    if (l == c.k) {
      sk = s[l];
      m1h = M.m1[l].hi();
      m1l = M.m1[l].lo();
      m2k = M.m2[l].val();
    }
  // any approximation q0 of m1h / Wh serves: the exact remainder
  // m1h - q0 Wh gives the correction q1
  const float Wh = M.W.hi(), Wl = M.W.lo(), rW = rcp_approx(Wh);
  const float q0 = m1h * rW;
  const float p = q0 * Wh;
  const float pe = fmaf(q0, Wh, -p);
  const float rr = ((m1h - p) - pe) + m1l - q0 * Wl;
  const float q1 = rr * rW;
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
  // |Qh + Ql - Q_exact| <= eQ = (e_m1 + |m1 / W| e_W) / W plus the
  // double-float's own rounding.  A float q is on the same side of Qh + Ql as
  // of Q_exact unless it lies within eQ of Qh + Ql: the band [Qlo_f, Qhi_f]
  // holds those floats (it is empty when no float is that close).
  const float em1k = kk * sqrt_approx(fmaxf(m2k, 0.f) * W) * 1.0001f + u * fabsf(m1h);
  const float eQ = (em1k + fabsf(q0) * eW) * rW * 1.0625f + 4.f * u * fabsf(q1) +
                   16.f * u * u * (fabsf(sk) + fabsf(q0)) + 1e-37f;
  c.Qlo_f = __fadd_ru(Qh, __fsub_rd(Ql, eQ));
  c.Qhi_f = __fadd_rd(Qh, __fadd_ru(Ql, eQ));
  return c;
}

// Steps 3-4 for a set of two float particles a, b (weights wa, wb), with a
// certificate, as decide_mixed: W^2 var_l = wa wb d_l^2 (d = q_b - q_a) and
// W P_l = wa q_a + wb q_b carry relative errors of a few u, so the bounds are
// simple.  The cut needs no value: the exact centroid lies strictly between
// two distinct values, so the smaller goes to V1.  unsure = 1 hands the pair
// to the FP64 recheck.
template <int D, bool VAR = true>
__device__ __forceinline__ Cut decide_pair(const Problem &P, float wa, float wb, const float *qa,
                                           const float *qb) {
  constexpr float u = 1.0f / (1 << 24);
  const float inf = __int_as_float(0x7f800000);
  const bool normd = VAR && (P.variant & kVarNormalized) != 0;
  const bool pnorm = VAR && (P.variant & kVarPNorm) != 0;
  Cut c = cut_none();
  const float W = wa + wb, ww = wa * wb;
  float denN = 0.f, eDN = 0.f;
  if (pnorm) {
#pragma unroll
    for (int l = 0; l < D; ++l)
      if (l >= P.dx) {
        const float Pw = fmaf(wa, qa[l], wb * qb[l]);
        const float eP = 3.f * u * (fabsf(wa * qa[l]) + fabsf(wb * qb[l]));
        denN = fmaf(Pw, Pw, denN);
        eDN = fmaf(2.f * fabsf(Pw) + eP, eP, eDN);
      }
    eDN = (eDN + 8.f * u * denN) * 1.0625f;
  }
  bool sure = true;
  float best = -1.f, bestLo = 0.f, bestHi = 0.f, otherHi = 0.f;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const float d = qb[l] - qa[l];
    const float V = ww * (d * d);
    const float eV = 8.f * u * V;
    // an underflowed or overflowed V: FP64 decides
    if ((d != 0.f && !(V >= 1e-30f)) || !(V <= 1e30f)) sure = false;
    float den, eD, tol2;
    if (l < P.dx) {
      den = P.L2f[l] * (W * W);
      eD = 8.f * u * den;
      tol2 = P.tol2_xf;
    } else if (pnorm) {
      den = denN;
      eD = eDN;
      tol2 = P.tol2_pf;
    } else {
      const float Pw = fmaf(wa, qa[l], wb * qb[l]);
      const float eP = 3.f * u * (fabsf(wa * qa[l]) + fabsf(wb * qb[l]));
      den = Pw * Pw;
      eD = (fmaf(2.f * fabsf(Pw) + eP, eP, 2.f * u * den)) * 1.0625f;
      tol2 = P.tol2_pf;
    }
    if (!(den <= 1e30f) || (den != 0.f && den < 1e-30f)) sure = false;
    const float t = tol2 * den;
    const float f = V - t;
    if (f > 0.f) c.leaf = 0;
    if (!(fabsf(f) > fmaf(tol2, eD, eV) + 2.f * u * (V + t))) sure = false;
    const float kden = normd ? t : den, eK = normd ? tol2 * eD : eD;
    const float rk = rcp_approx(kden);
    const float rho = eK * rk * 1.0001f + 4.f * u;
    float r, lo, hi;
    if (kden > 0.f && rho < 0.5f) {
      r = V * rk;
      lo = V > eV ? (V - eV) * rk * (1.f - rho - 8.f * u) : 0.f;
      hi = (V + eV) * rk * (1.f + 2.f * rho + 8.f * u);
    } else {
      r = V == 0.f ? 0.f : (kden > 0.f ? V * rk : inf);
      lo = (V > eV && eK == 0.f && kden == 0.f) ? inf : 0.f;
      hi = (V + eV == 0.f) ? 0.f : inf;
    }
    if (r > best) {
      otherHi = fmaxf(otherHi, bestHi);
      best = r;
      bestLo = lo;
      bestHi = hi;
      c.k = l;
    } else {
      otherHi = fmaxf(otherHi, hi);
    }
  }
  if (!c.leaf && !(bestLo > otherHi)) sure = false;
  if (!sure) {
    c.unsure = 1;
    c.leaf = 0;
  }
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
