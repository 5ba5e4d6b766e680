// coal_kernel.cu -- the persistent collision-coalescence kernel (both precision forms).
//
// One CTA owns one grid point at a time (the unit coal_bott_new is called on, Sec. III,
// Listing 1) and takes the next point from the compacted, cost-ordered list through an
// atomic queue head until the list is exhausted. The point's spectra live in shared memory
// for all n_steps steps; only the first load and the final store touch the caller's buffer.
// The pair collection kernels are read straight from the L2-resident tables (one FP64 and
// one FP32 copy per layout), one entry per bin pair (the on-demand lookup of Listing 5).
//
// Per step (Bott's flux method, pairwise form):
//   1. budget B = sum M (FP64, fixed reduction tree), active bin range of every species;
//   2. N = M / x;  R^a_i = dt x_i N^a_i sum_{b,j} K N^b_j      (row mat-vec, lane per row);
//      lambda = min(1, M / R) in FP64;
//   3. loss^a_i = dt x_i N^a_i sum_{b,j} K N^b_j min(lambda^a_i, lambda^b_j)
//      (equal to R when no ratio fired anywhere in the point: the pass is skipped; else
//      a correction over the limited rows sorted by ratio);
//   4. gain pass: one lane per (target bin k, ordered species orientation) item walks the
//      bin distances d of the pairs (m - d, m) whose mass lands in k (m = k - kappa[d]),
//      computes dM and Bott's flux F, and keeps (sum of dM - F) for bin k and (sum of F)
//      for bin k + 1 in registers; the lanes of a warp hold one or two targets, walk the
//      same d and read contiguous kernel entries. Partial sums land in per-orientation
//      shared arrays and are added in a fixed order: the result does not depend on
//      scheduling;
//   5. M' = M - loss + gain (FP64), mass error, round-off negatives to 0, rescale to B.
// FP32_SPLIT runs 2-4 with float values and float sums; 1 and 5 stay FP64.
#include <algorithm>
#include <cfloat>
#include <cstdio>

#include "fsbm_internal.cuh"

namespace fsbm {
namespace {

struct Orient {
  int8_t s, l;      // slots of the small-index and the large-index partner
  int8_t dmin;      // 0, or 1 when the two species' roles are swapped (d = 0 belongs to the
                    // other orientation of the same species pair)
  int8_t c;         // slot of the product species
  int table;        // s_id * S + l_id: position of the orientation inside a Kd row
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_min_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// e / n for 0 <= e < 5 n, 2 <= n <= 512, from the grid's inv_n = floor(2^32 / n) + 1 (exact
// in that range; an integer division by a value known only at run time costs some twenty
// instructions)
__device__ __forceinline__ int div_n(int e, unsigned inv_n) { return (int)__umulhi((unsigned)e, inv_n); }
// x / d for 0 <= x, d < 2^16 through inv = floor(2^32 / d) + 1 (exact there: x (inv d - 2^32)
// < 2^32); d = 1, whose inverse would not fit, takes inv = 0 and returns x
__device__ __forceinline__ unsigned div_inv(int d) {
  return d == 1 ? 0u : (unsigned)(0x100000000ull / (unsigned long long)d + 1);
}
__device__ __forceinline__ int div_by(int x, int d, unsigned inv) {
  return d == 1 ? x : (int)__umulhi((unsigned)x, inv);
}
// eight consecutive shared-memory values from a 16-byte aligned address
__device__ __forceinline__ void lds8(const float* p, float (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void lds8(const double* p, double (&v)[8]) {
#pragma unroll
  for (int u = 0; u < 8; u += 2) {
    const double2 a = *reinterpret_cast<const double2*>(p + u);
    v[u] = a.x;
    v[u + 1] = a.y;
  }
}
__device__ __forceinline__ void lds8(const int* p, int (&v)[8]) {
  const int4 a = *reinterpret_cast<const int4*>(p), b = *reinterpret_cast<const int4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Bott's flux of mass dM deposited in bin k toward bin k + 1 (see fsbm_coal.h).
__device__ __forceinline__ double bott_flux(double dM, double Mk, double Mk1, double c) {
  const double g = Mk + dM;
  const double x1 = log(Mk1 / g + kBottEps);
  double F;
  if (x1 == 0.0)
    F = dM * c;
  else if (isinf(x1))  // the ratio overflowed: the flux's limit is all of dM (c > 0) or 0
    F = c > 0.0 ? dM : 0.0;
  else
    F = dM * exp(0.5 * x1) * (-expm1(-c * x1)) / x1;
  return fmin(fmax(F, 0.0), dM);
}

// FP32 form. 1e-60 is below FP32's range, so ln(rho + 1e-60) becomes ln(rho) clamped at
// ln(1e-60); the two differ only for rho within a few orders of 1e-60. ln(rho) is capped at
// 80, above which F >= dM for every c > 0 (and F = 0 for c = 0) in either form.
//
// One formula for every pair, with no branch, from the SFU's approximations (relative error
// near 2^-22 each):
//   rho = M_{k+1} / g through the SFU reciprocal; x1 = log2(rho) ln 2, clamped to
//   [ln 1e-60, 80] (an empty bin k+1 gives rho = 0 and x1 = ln 1e-60; a ratio that overflows
//   gives x1 = 80; a NaN from 0 / 0 takes the lower clamp);
//   F = dM e^{x1/2} (1 - e^{-z}) / x1 with z = c x1, where
//     (1 - e^{-z}) / x1 = c e^{-z/2} sinh(z/2) / (z/2)   for |z| <= 1 (no cancellation near
//       z = 0: sinh(y)/y = 1 + y^2/6 + y^4/120 + y^6/5040, next term below 1.1e-8), and
//     (1 - e^{-z}) / x1 = (1 - (e^{-z/2})^2) / x1        otherwise;
//   both are formed and one is selected, so the lanes of a warp never diverge here.
// The code works in base-2 units, which saves the multiply by ln 2: l = log2(rho) clamped to
// [log2 1e-60, 80 / ln 2] (x1 = l ln 2) and zl = c l (z = zl ln 2); with the factor ln 2 moved
// into the constants, F = dM A' r' where A' = e^{x1/2} / ln 2 = 2^{l/2 - log2 ln 2} and r' =
// ln 2 (1 - e^{-z}) / x1 is c w ln 2 sinh(z/2)/(z/2) (the series in zl^2, each coefficient
// times the matching power of ln 2) for |zl| <= 1 / ln 2, or (1 - w^2) / l, w = 2^{-zl/2}.
// Five SFU operations per pair: the two reciprocals, log2, e^{x1/2} and e^{-z/2}. They flush
// subnormal inputs and results to zero (one SFU instruction each, no subnormal fix-up): a ratio
// rho below FP32's normal range then reads as 0 (x1 = ln 1e-60) and a sum g below it as an
// overflowing ratio (x1 = 80), both in bins more than 30 orders below any normal content; the
// exponentials' results (e^{x1/2} >= 1e-30, e^{-z/2} in [e^-40, e^69]) stay normal.
__device__ __forceinline__ float sfu_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sfu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sfu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr double kLn2d = 0.69314718055994531;
constexpr float kLog2BottEps = (float)(-138.15510557964274 / kLn2d);  // log2(1e-60)
constexpr float kLog2Cap = (float)(80.0 / kLn2d);                     // 80 / ln 2
constexpr float kLog2InvLn2 = 0.52876637294f;                         // -log2(ln 2)
constexpr float kInvLn2f = (float)(1.0 / kLn2d);
constexpr float kS0 = (float)kLn2d;  // ln 2 (1 + u / 24 + u^2 / 1920 + u^3 / 322560), u = z^2
constexpr float kS1 = (float)(kLn2d * kLn2d * kLn2d / 24.0);
constexpr float kS2 = (float)(kLn2d * kLn2d * kLn2d * kLn2d * kLn2d / 1920.0);
constexpr float kS3 = (float)(kLn2d * kLn2d * kLn2d * kLn2d * kLn2d * kLn2d * kLn2d / 322560.0);
__device__ __forceinline__ float bott_flux_f32(float dM, float Mk, float Mk1, float c) {
  const float g = Mk + dM;
  const float rho = Mk1 * sfu_rcp(g);
  const float l = fminf(fmaxf(sfu_lg2(rho), kLog2BottEps), kLog2Cap);  // x1 / ln 2
  const float zl = c * l;                                               // z / ln 2
  const float A = sfu_ex2(fmaf(l, 0.5f, kLog2InvLn2));                  // e^{x1/2} / ln 2
  const float w = sfu_ex2(zl * -0.5f);                                  // e^{-z/2}
  const float u = zl * zl;                                              // z^2 / ln^2 2
  float P = fmaf(u, kS3, kS2);
  P = fmaf(u, P, kS1);
  P = fmaf(u, P, kS0);
  const float near0 = c * w * P;
  const float far = fmaf(-w, w, 1.f) * sfu_rcp(l);  // an overflowing e^{-z} gives +inf: F = dM
  const float ratio = fabsf(zl) <= kInvLn2f ? near0 : far;
  return fminf(dM * (A * ratio), dM);  // A * ratio first: dM * A alone can underflow; fminf
                                       // keeps dM where dM * inf gave inf or 0 * inf NaN
}

template <typename T> struct Sel;
template <> struct Sel<double> {
  static __device__ const double* x(const GridDev& g) { return g.x64; }
  static __device__ const double* invx(const GridDev& g) { return g.invx64; }
  static __device__ const double* cd(const GridDev& g) { return g.cd64; }
  static __device__ const double* Kd(const GridDev& g) { return g.Kd64; }
  static __device__ const double* Kr(const GridDev& g) { return g.Kr64; }
  static __device__ const double* Kd_d(const GridDev& g) { return g.Kd64_d; }
  static __device__ const double* Kr_d(const GridDev& g) { return g.Kr64_d; }
};
template <> struct Sel<float> {
  static __device__ const float* x(const GridDev& g) { return g.x32; }
  static __device__ const float* invx(const GridDev& g) { return g.invx32; }
  static __device__ const float* cd(const GridDev& g) { return g.cd32; }
  static __device__ const float* Kd(const GridDev& g) { return g.Kd32; }
  static __device__ const float* Kr(const GridDev& g) { return g.Kr32; }
  static __device__ const float* Kd_d(const GridDev& g) { return g.Kd32_d; }
  static __device__ const float* Kr_d(const GridDev& g) { return g.Kr32_d; }
};

// Running sums. The FP64 form adds each term in FP64. The FP32 form adds short runs of
// terms in FP32 and folds each run into a float-float total (hi + lo, Knuth's two-sum), so
// rounding grows with the run length (16 or 32 terms) rather than with a sum over a few
// hundred bins, and no FP64 instruction enters the pair loops.
struct FF {
  float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void ff_add(FF& a, float v) {
  const float s = a.hi + v;
  const float bp = s - a.hi;
  const float e = (a.hi - (s - bp)) + (v - bp);
  a.hi = s;
  a.lo += e;
}
__device__ __forceinline__ void ff_add(FF& a, const FF& b) {
  ff_add(a, b.hi);
  a.lo += b.lo;
}

template <typename T> struct Num;
template <> struct Num<double> {
  using Sum = double;
  static __device__ __forceinline__ void add(Sum& a, const Sum& b) { a += b; }
  static __device__ __forceinline__ void sub(Sum& a, const Sum& b) { a -= b; }
  static __device__ __forceinline__ double val(const Sum& a) { return a; }
  static __device__ __forceinline__ Sum zero() { return 0.0; }
};
template <> struct Num<float> {
  using Sum = FF;
  static __device__ __forceinline__ void add(Sum& a, const Sum& b) { ff_add(a, b); }
  static __device__ __forceinline__ void sub(Sum& a, const Sum& b) {
    ff_add(a, -b.hi);
    a.lo -= b.lo;
  }
  static __device__ __forceinline__ double val(const Sum& a) { return (double)a.hi + (double)a.lo; }
  static __device__ __forceinline__ Sum zero() { return FF{}; }
};

template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ double sum() const { return s; }
};
template <> struct Acc<float> {
  float r = 0.f;
  FF s;
  __device__ __forceinline__ void add(float v) { r += v; }
  __device__ __forceinline__ void flush() {
    ff_add(s, r);
    r = 0.f;
  }
  __device__ __forceinline__ FF sum() const {
    FF t = s;
    ff_add(t, r);
    return t;
  }
};
// pairs a gain lane adds in T before folding the run into its total: FP32 runs of 32 (one run
// per item on the 33-bin grid); FP64 adds every term in FP64, so one run per group
template <typename T> struct GainRun;
template <> struct GainRun<float> { static constexpr int value = 32; };
template <> struct GainRun<double> { static constexpr int value = 1 << 20; };
constexpr int kLossRun = 32;
constexpr int kSplitLanes = 128;  // a point's gain items share lanes until they fill 4 warps

// A loss pass cuts its padded column list (a multiple of 8 long) into runs of at most kLossRun
// columns, at most 2 ns of them (their partial sums fill the two gain arrays), of equal length
// in blocks of 8 but for the last.
__device__ __forceinline__ int loss_runs(int cols, int ns) {
  return max(1, min((cols + kLossRun - 1) / kLossRun, 2 * ns));
}
__device__ __forceinline__ int loss_span(int cols, int nch) { return (((cols >> 3) + nch - 1) / nch) << 3; }

// a += (a of lane ^ off), every lane of the warp taking part
template <typename T>
__device__ __forceinline__ void shfl_add(typename Num<T>::Sum& a, int off);
template <>
__device__ __forceinline__ void shfl_add<double>(double& a, int off) {
  a += __shfl_xor_sync(0xffffffffu, a, off);
}
template <>
__device__ __forceinline__ void shfl_add<float>(FF& a, int off) {
  const FF b{__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
  ff_add(a, b);
}

// N and lambda of one bin side by side: the gain pass reads both of a pair's smaller bin at once
template <typename T>
struct __align__(2 * sizeof(T)) NLPair {
  T n, l;
};

// Shared-memory carve-up for nmax bins and S species (T = pair-arithmetic type).
template <typename T>
struct Smem {
  using Sum = typename Num<T>::Sum;
  double* M;      // [S][nmax] FP64 state
  double* loss;   // [S][nmax] R, then loss
  Sum* stay;      // [S*S][nmax] per-orientation partial gains of bin k
  Sum* up;        // [S*S][nmax] per-orientation fluxes from bin k to k+1
  T* Mt;          // [S][nmax] state in T (aliases M when T = double)
  NLPair<T>* NL;  // [S][nmax] (N, lambda) of every bin: N from step 1, lambda from step 2
  T* nlam;        // FP64 form: [S][nmax] N lambda of every bin (else NULL)
  T* lNl;         // FP64 form: [S*nmax + 8] N lambda of the listed columns, padded to 8 (else NULL)
  T* xs;          // [nmax]
  T* cd;          // [nmax] Courant number per bin distance
  T* llam;        // [S*nmax + 8] ratios of the listed columns (limited rows), padded to 8
  T* lN;          // [S*nmax + 8] number concentrations of the listed columns, padded to 8
  int* lim;       // [S*nmax + 8] rows whose limiter ratio is below 1, ascending row index
  int* loff;      // [S*nmax + 8] Kr offset (species, bin) of the listed columns, padded to 8
  // every array starts on a 16-byte boundary (the column lists are read four entries at a time)
  static __host__ __device__ size_t up16(size_t b) { return (b + 15) & ~size_t(15); }
  static __host__ __device__ size_t bytes(int nmax, int S) {
    const size_t e = (size_t)S * nmax, l = e + 8;
    size_t b = 2 * up16(sizeof(double) * e) + 2 * up16(sizeof(Sum) * S * e);
    if (sizeof(T) != sizeof(double)) b += up16(sizeof(T) * e);
    b += up16(sizeof(NLPair<T>) * e) + 2 * up16(sizeof(T) * nmax) + 2 * up16(sizeof(T) * l) + 2 * up16(sizeof(int) * l);
    if (sizeof(T) == sizeof(double)) b += up16(sizeof(T) * e) + up16(sizeof(T) * l);
    return b;
  }
  __device__ void carve(unsigned char* base, int nmax, int S) {
    const size_t e = (size_t)S * nmax, l = e + 8;
    unsigned char* p = base;
    auto take = [&](size_t nbytes) {
      unsigned char* q = p;
      p += up16(nbytes);
      return q;
    };
    M = reinterpret_cast<double*>(take(sizeof(double) * e));
    loss = reinterpret_cast<double*>(take(sizeof(double) * e));
    stay = reinterpret_cast<Sum*>(take(sizeof(Sum) * S * e));
    up = reinterpret_cast<Sum*>(take(sizeof(Sum) * S * e));
    Mt = sizeof(T) != sizeof(double) ? reinterpret_cast<T*>(take(sizeof(T) * e)) : reinterpret_cast<T*>(M);
    NL = reinterpret_cast<NLPair<T>*>(take(sizeof(NLPair<T>) * e));
    xs = reinterpret_cast<T*>(take(sizeof(T) * nmax));
    cd = reinterpret_cast<T*>(take(sizeof(T) * nmax));
    llam = reinterpret_cast<T*>(take(sizeof(T) * l));
    lN = reinterpret_cast<T*>(take(sizeof(T) * l));
    lim = reinterpret_cast<int*>(take(sizeof(int) * l));
    loff = reinterpret_cast<int*>(take(sizeof(int) * l));
    nlam = sizeof(T) == sizeof(double) ? reinterpret_cast<T*>(take(sizeof(T) * e)) : nullptr;
    lNl = sizeof(T) == sizeof(double) ? reinterpret_cast<T*>(take(sizeof(T) * l)) : nullptr;
  }
};

// 1 / sqrt(x) for normal x > 0: the SFU's approximation y (relative error near 2^-20)
// corrected once to third order: with e = 1 - x y^2, 1/sqrt(x) = y (1 - e)^(-1/2)
// = y (1 + e/2 + 3e^2/8 + O(e^3)).
__device__ __forceinline__ double fsbm_rsqrt(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}
// 1 / x for normal x != 0: the SFU's approximation y corrected once to third order:
// with e = 1 - x y, 1/x = y / (1 - e) = y (1 + e + e^2 + O(e^3)).
__device__ __forceinline__ double fsbm_rcp(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
// Sign tests on the bit pattern run on the integer pipes instead of the (slow) FP64 pipe.
__device__ __forceinline__ bool is_zero(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool is_zero(float v) { return (__float_as_int(v) << 1) == 0; }
// min of two non-negative doubles through their bit patterns (they order like integers)
__device__ __forceinline__ double min_nonneg(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ float min_nonneg(float a, float b) { return fminf(a, b); }
// a < b for non-negative doubles, on the integer pipes
__device__ __forceinline__ bool lt_nonneg(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool lt_nonneg(float a, float b) { return a < b; }
// Bott's flux with target-bin constants hoisted out of the pair loop:
//  * bin k+1 holds at least 1e-43 of the largest content bin k can reach (Mk + 2B): then
//    1e-60 g is below half an ulp of M_{k+1}, M_{k+1} + 1e-60 g rounds to M_{k+1} exactly, and
//    ln(rho + 1e-60) = ln M_{k+1} - ln g, e^{x1/2} = sqrt(M_{k+1}) / sqrt(g);
//  * bin k+1 is empty: x1 = ln 1e-60 and e^{x1/2} = 1e-30 for every pair;
//  * otherwise (a deep tail): x1 = ln(M_{k+1} + 1e-60 g) - ln g and e^{x1/2} =
//    sqrt(M_{k+1} + 1e-60 g) / sqrt(g).
// Per pair that is one or two logarithms, one exponential (which also gives e^y - 1 without
// cancellation), a reciprocal square root and a reciprocal, all table-driven or refined from
// the SFU's approximations. A sum g below 1e-300 falls back to the direct form above.
struct TargetFP64 {
  double Mk, Mk1, lnMk1, sqMk1;
  int kind;  // 0: regular, 1: bin k+1 empty, 2: deep tail
};
__device__ __forceinline__ TargetFP64 target_fp64(double Mk, double Mk1, double B, const MathTabs& mt) {
  TargetFP64 tg;
  tg.Mk = Mk;
  tg.Mk1 = Mk1;
  tg.kind = (Mk1 >= 1e-43 * (Mk + 2.0 * B) && Mk1 >= 1e-300) ? 0 : (is_zero(Mk1) ? 1 : 2);
  tg.lnMk1 = tg.kind == 0 ? fsbm_log(Mk1, mt) : mt.ln_eps;
  tg.sqMk1 = tg.kind == 0 ? sqrt(Mk1) : 0.0;
  return tg;
}
// F for one pair (see TargetFP64). F >= 0 holds exactly (the factors' signs agree), so only
// the upper clip is needed.
__device__ __forceinline__ double bott_flux_fast(double dM, const TargetFP64& tg, double c, const MathTabs& mt) {
  const double g = tg.Mk + dM;
  if (__double_as_longlong(g) < 0x01a56e1fc2f8f359LL)  // g < 1e-300
    return bott_flux(dM, tg.Mk, tg.Mk1, c);
  const double rg = fsbm_rsqrt(g);
  double x1, A;
  if (tg.kind == 0) {
    x1 = tg.lnMk1 - fsbm_log(g, mt);
    A = tg.sqMk1 * rg;
  } else if (tg.kind == 1) {
    x1 = mt.ln_eps;
    A = mt.sqrt_eps;
  } else {
    const double u = fma(kBottEps, g, tg.Mk1);
    if (__double_as_longlong(u) < 0x01a56e1fc2f8f359LL) return bott_flux(dM, tg.Mk, tg.Mk1, c);
    x1 = fsbm_log(u, mt) - fsbm_log(g, mt);
    A = u * fsbm_rsqrt(u) * rg;
  }
  if (is_zero(x1)) return min_nonneg(dM * c, dM);
  double E, em1;
  fsbm_exp_em1(-c * x1, mt, &E, &em1);
  return min_nonneg((dM * A) * (-em1) * fsbm_rcp(x1), dM);
}

// Flux of one pair into a regular target bin (precision-specific target constants).
template <typename T> struct TargetOf;
template <> struct TargetOf<double> {
  TargetFP64 tg;
  __device__ __forceinline__ void init(double Mk, double Mk1, double B, const MathTabs& mt) {
    tg = target_fp64(Mk, Mk1, B, mt);
  }
  __device__ __forceinline__ double flux(double dM, double c, const MathTabs& mt) const {
    return bott_flux_fast(dM, tg, c, mt);
  }
};
template <> struct TargetOf<float> {
  float Mk, Mk1;
  __device__ __forceinline__ void init(float mk, float mk1, double, const MathTabs&) {
    Mk = mk;
    Mk1 = mk1;
  }
  __device__ __forceinline__ float flux(float dM, float c, const MathTabs&) const {
    return bott_flux_f32(dM, Mk, Mk1, c);
  }
};

// Gain pass for one (target bin k, orientation o) item per lane. The pairs (m - d, m) whose
// mass lands in k come in groups: for each distance class kappa (kappa(d) = kappa for d in
// [d_lo, d_hi]) the larger bin is m = k - kappa (every m in [n-1-kappa, n-1] for the top bin,
// which keeps what reaches or passes it, with no flux), and d runs over one contiguous range.
// The loops are nested (class, m, d): the class loop has the same trip count in every lane, so
// the lanes of a warp move from group to group together and only the d ranges differ (by range
// cut-offs and by one pair between adjacent targets). Within a group the loop reads the
// pre-scaled kernel entry (contiguous across the warp's orientations), N of the smaller bin,
// its limiter ratio and the Courant number c(d); everything else is in registers.
//   dM = C (x_i + x_m) = [K (1 + alpha^-d)] N_i [M_m dt]      (x_i = x_m alpha^-d)
// LEVELS: the point lies between two pressure levels; its kernel is K1 + wl (K2 - K1).
// SPLIT: the item's pairs are shared by P lanes; part p takes every P-th distance of each group
// (d = d0 + p, d0 + p + P, ...), and the caller adds the P partial sums in a fixed order.
template <typename T, bool LIMITED, bool LEVELS, bool TOP>
__device__ __forceinline__ void gain_task(const GridDev& G, int S2, const Smem<T>& sm, const Orient& o_ref,
                                          const int* lo, const int* hi, int k, bool on, int p, int P, T dt,
                                          double B, const MathTabs& mt, T wl, typename Num<T>::Sum* out_stay,
                                          typename Num<T>::Sum* out_up) {
  const int n = G.n;
  const Orient o = o_ref;  // register copy
  Acc<T> stay, up;
  const T* __restrict__ Kd = Sel<T>::Kd(G) + o.table;
  const T* __restrict__ Kdd = LEVELS ? Sel<T>::Kd_d(G) + o.table : nullptr;
  const NLPair<T>* __restrict__ NLs = sm.NL + o.s * n;
  const T* __restrict__ NLm = sizeof(T) == sizeof(double) ? sm.nlam + o.s * n : nullptr;
  const T* __restrict__ Ml = sm.Mt + o.l * n;
  const NLPair<T>* __restrict__ NLl = sm.NL + o.l * n;
  const T* __restrict__ cds = sm.cd;
  const int lo_s = lo[o.s], hi_s = hi[o.s], lo_l = lo[o.l], hi_l = hi[o.l];
  on = on && k >= 1 && k < n;
  if (FSBM_CHECKED_BUILD && on && !TOP && !FSBM_OK(G.chk, k + 1, n)) on = false;
  TargetOf<T> tgt;
  if (!TOP) tgt.init(on ? sm.Mt[o.c * n + k] : T(0), on ? sm.Mt[o.c * n + k + 1] : T(0), B, mt);
  const int kstride = n * S2 * P;  // table step from one of this part's distances to the next
  const int lgP = __ffs(P) - 1;
  int run = 0;  // FP32: pairs added to the open run since it was last folded into the totals
  for (int kap = 0; kap <= G.kappa_max; ++kap) {
    const int dlo = max(G.d_lo[kap], (int)o.dmin), dhi = G.d_hi[kap];
    const int m0 = max(TOP ? n - 1 - kap : k - kap, lo_l);
    const int m1 = on ? min(TOP ? n - 1 : k - kap, hi_l) : m0 - 1;
    for (int m = m0; m <= m1; ++m) {
      const int d0 = max(dlo, m - hi_s), d1 = min(dhi, m - lo_s);
      if (FSBM_CHECKED_BUILD && d0 <= d1 &&
          !(FSBM_OK(G.chk, d0, n) && FSBM_OK(G.chk, d1, n) && FSBM_OK(G.chk, m, n) && FSBM_OK(G.chk, m - d1, n) &&
            FSBM_OK(G.chk, m - d0, n) && FSBM_OK(G.chk, ((ptrdiff_t)d1 * n + m) * S2 + o.table, (ptrdiff_t)S2 * n * n)))
        continue;
      const T am = Ml[m] * dt;
      const T ll = LIMITED ? NLl[m].l : T(1);
      const T amll = am * ll;  // FP64 limited pairs whose ratio min is the larger bin's
      const ptrdiff_t e0 = (ptrdiff_t)((d0 + p) * n + m) * S2;
      const T* __restrict__ Kp = Kd + e0;
      const T* __restrict__ Kq = LEVELS ? Kdd + e0 : nullptr;
      // chunks of up to GainRun pairs; the open run is folded into the totals before a chunk
      // that would take it past GainRun pairs (and at the end of the item)
      for (int dc = d0 + p; dc <= d1; dc += GainRun<T>::value * P) {
        const int dce = min(d1, dc + (GainRun<T>::value - 1) * P);
        if (sizeof(T) == sizeof(float)) {
          const int len = ((dce - dc) >> lgP) + 1;
          if (run + len > GainRun<T>::value) {
            stay.flush();
            up.flush();
            run = 0;
          }
          run += len;
        }
        int d = dc;
        if (sizeof(T) == sizeof(float)) {
          // FP32: two pairs per iteration, so that two flux chains (each a string of dependent
          // SFU and FMA operations) are in flight per lane; the sums take them in pair order.
          // (FP64 runs one pair at a time: its double-precision pipe is already the bound, and
          // the unrolled form measured slower there.)
          for (; d + P <= dce; d += 2 * P, Kp += 2 * kstride) {
            const int i = m - d;
            T K0 = __ldg(Kp), K1 = __ldg(Kp + kstride);
            if (LEVELS) {
              K0 = fma(wl, __ldg(Kq), K0);
              K1 = fma(wl, __ldg(Kq + kstride), K1);
              Kq += 2 * kstride;
            }
            const NLPair<T> a0 = NLs[i], a1 = NLs[i - P];
            T dM0 = K0 * am * a0.n, dM1 = K1 * am * a1.n;
            if (LIMITED) {
              dM0 *= min_nonneg(a0.l, ll);
              dM1 *= min_nonneg(a1.l, ll);
            }
            stay.add(dM0);
            stay.add(dM1);
            if (!TOP) {
              const T f0 = tgt.flux(dM0, cds[d], mt), f1 = tgt.flux(dM1, cds[d + P], mt);
              up.add(f0);
              up.add(f1);
            }
          }
        }
        for (; d <= dce; d += P, Kp += kstride) {
          const int i = m - d;
          T K = __ldg(Kp);
          if (LEVELS) {
            K = fma(wl, __ldg(Kq), K);
            Kq += kstride;
          }
          const NLPair<T> a = NLs[i];
          T dM;
          if (LIMITED && sizeof(T) == sizeof(double)) {
            // min(l_i, l_m) N_i (M_m dt) as two multiplies: (N_i l_i)(M_m dt) when l_i <= l_m,
            // else N_i (M_m dt l_m), chosen on the bit patterns
            const bool own = !lt_nonneg(ll, a.l);
            dM = K * (own ? am : amll) * (own ? NLm[i] : a.n);
          } else {
            dM = K * am * a.n;
            if (LIMITED) dM *= min_nonneg(a.l, ll);
          }
          stay.add(dM);  // the pair's whole mass; the flux is taken back out at the end
          if (!TOP) {    // none out of the top bin
            const T c = cds[d];
            // c = 0 (the pair lands exactly on bin k): F = 0, skipped. Every d = 0 pair (two
            // equal bins: x_m + x_m = x_{m+s} exactly) forms a group of its own and comes
            // through here, so a warp skips it as a whole; the FP32 flux would give 0 too
            if (!is_zero(c)) up.add(tgt.flux(dM, c, mt));
          }
        }
      }
    }
  }
  typename Num<T>::Sum st = stay.sum(), u = up.sum();
  Num<T>::sub(st, u);
  *out_stay = st;
  *out_up = u;
}

template <typename T>
struct StoreOf { using type = T; };

// LEV: kernels at two pressure levels (a separate instantiation, so that the one-level kernel
// keeps its registers and instructions). The FP32 form is held to 64 registers (four CTAs of
// 256 threads per SM): it is bound by instruction issue and latency, and more resident warps
// hide more of it; the FP64 form is bound by the FP64 pipe and keeps what it needs.
template <typename T, bool LEV>
__global__ void __launch_bounds__(512, sizeof(T) == sizeof(float) ? 2 : 1) k_coal(Tables t, PointsDev pd, const int32_t* __restrict__ list, int32_t* counters, double dt,
                       int n_steps, int nmax) {
  using Store = typename StoreOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[33];
  __shared__ Orient ori[kMaxOrient];
  __shared__ int8_t s_plist[kMaxSpecies][kMaxOrient];  // orientations whose product is slot c
  __shared__ int s_np[kMaxSpecies];
  __shared__ int s_lo[kMaxSpecies], s_hi[kMaxSpecies], s_sp[kMaxSpecies];
  __shared__ int s_next;
  __shared__ int s_task;
  __shared__ int s_nlim;

  const int S = t.S;
  Smem<T> sm;
  sm.carve(smem_raw, nmax, S);
  const int tid = threadIdx.x, NT = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = NT >> 5;
  const int n_end = counters[2];
  const T dtT = (T)dt;

  for (;;) {
    if (tid == 0) s_next = atomicAdd(&counters[1], 1);
    __syncthreads();
    const int idx = s_next;
    __syncthreads();
    if (idx >= n_end) break;
    if (FSBM_CHECKED_BUILD && !FSBM_OK(t.chk, idx, counters[0])) break;
    const int p = list[idx];
    if (FSBM_CHECKED_BUILD && !FSBM_OK(t.chk, p, pd.n_points)) continue;
    const int g = pd.grid_id[p];
    if (FSBM_CHECKED_BUILD && !FSBM_OK(t.chk, g, t.G)) continue;
    const GridDev& G = t.g[g];
    const int n = G.n;
    const unsigned mask = pd.species_mask[p];
    const int ns = __popc(mask);
    if (FSBM_CHECKED_BUILD && !(FSBM_OK(t.chk, n - 1, nmax) && FSBM_OK(t.chk, ns - 1, S) &&
                                FSBM_OK(t.chk, pd.offset[p + 1] - pd.offset[p] - (int64_t)ns * n, 1)))
      continue;
    const int64_t off = pd.offset[p];
    Store* spec = reinterpret_cast<Store*>(pd.spectra) + off;
    const int E = ns * n;
    // kernels at two pressure levels: weight of the second at this point (0: the first alone)
    const double wlev = LEV ? level_weight(t, pd, p) : 0.0;
    const bool lev = LEV && wlev != 0.0;
    const T wT = (T)wlev;

    if (tid == 0) {
      int q = 0;
      for (int a = 0; a < S; ++a)
        if (mask >> a & 1u) s_sp[q++] = a;
    }
    // load the spectrum (FP64 on chip) and the bin masses
    bool bad = false;
    for (int e = tid; e < E; e += NT) {
      const double v = (double)spec[e];
      bad |= !(v >= 0.0) || !(v <= DBL_MAX);
      sm.M[e] = v;
    }
    for (int k = tid; k < n; k += NT) {
      sm.xs[k] = Sel<T>::x(G)[k];
      sm.cd[k] = Sel<T>::cd(G)[k];
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) {
        pd.status[p] = 2;
        pd.mass_budget[p] = 0.0;
        pd.mass_error[p] = 0.0;
      }
      continue;
    }
    // the budget, summed by one warp in the order the end-of-step totals use, so that a
    // step that changes nothing rescales by exactly 1
    if (warp == 0) {
      double b = 0.0;
      for (int e = lane; e < E; e += 32) b += sm.M[e];
      b = warp_sum(b);
      if (lane == 0) red[2] = b;
    }
    __syncthreads();
    const double B0 = red[2];
    if (!(B0 > 0.0)) {
      if (tid == 0) {
        pd.status[p] = 4;
        pd.mass_budget[p] = 0.0;
        pd.mass_error[p] = 0.0;
      }
      continue;
    }
    // orientation list: same species once; each cross pair in both index orders
    if (tid == 0) {
      int q = 0;
      for (int a = 0; a < ns; ++a)
        for (int b = a; b < ns; ++b) {
          const int ia = s_sp[a], ib = s_sp[b];
          const int prod = t.product[ia * S + ib];
          const int cs = (prod == ia) ? a : b;
          ori[q++] = Orient{(int8_t)a, (int8_t)b, 0, (int8_t)cs, ia * S + ib};
          if (a != b) ori[q++] = Orient{(int8_t)b, (int8_t)a, 1, (int8_t)cs, ib * S + ia};
        }
      for (int c = 0; c < ns; ++c) s_np[c] = 0;
      for (int o = 0; o < q; ++o) {  // ascending orientation order within every product slot
        const int c = ori[o].c;
        s_plist[c][s_np[c]++] = (int8_t)o;
      }
    }
    __syncthreads();
    const int O = ns * ns;
    // lanes per gain item: points with few items (one or two species) share each item's
    // pairs among up to 8 lanes, so that they fill more warps and more lanes of each; the
    // choice depends on the point's shape only, never on the CTA size
    int lgP = 0;
    if (t.gain_split > 0) {
      while ((2 << lgP) <= t.gain_split) ++lgP;
    } else {
      while (lgP < 3 && (n - 2) * O * (2 << lgP) <= kSplitLanes) ++lgP;
    }
    const int P = 1 << lgP;
    // the loss passes' items: (row pair, run of columns), rows 2h and 2h + 1 of one species
    const int H = (n + 1) >> 1, RP = ns * H;
    const unsigned inv_H = div_inv(H), inv_RP = div_inv(RP), inv_O = div_inv(O);

    int status = 0;
    double emax = 0.0;
    const double inv_B0 = 1.0 / B0;  // mass errors are relative to the budget
    for (int step = 0; step < n_steps; ++step) {
      // 1. budget and active ranges. The budget of every step is the point's mass B0: each
      //    step ends rescaled to it (the start-of-step total equals B0 to rounding).
      const double Bs = B0;
      for (int a = warp; a < ns; a += nw) {
        // non-negative doubles order like their bit patterns: the largest bin and the range
        // tests run on the integer pipes (a -0.0 left by the clamp reads as negative: empty)
        const long long* Ma = reinterpret_cast<const long long*>(sm.M + a * n);
        long long mx = 0;
        for (int k = lane; k < n; k += 32) mx = max(mx, Ma[k]);
        mx = warp_max_ll(mx);
        long long thr = 1;  // M > 0
        if (t.tau > 0.0) thr = max(thr, __double_as_longlong(t.tau * __longlong_as_double(mx)));
        int lo = n, hi = -1;
        for (int k = lane; k < n; k += 32) {
          if (Ma[k] >= thr) {
            lo = min(lo, k);
            hi = max(hi, k);
          }
        }
        lo = warp_min_i(lo);
        hi = warp_max_i(hi);
        if (lane == 0) {
          s_lo[a] = lo;
          s_hi[a] = hi;
        }
      }
      for (int e = tid; e < E; e += NT) {
        const int k = e - div_n(e, G.inv_n) * n;
        const T m = (T)sm.M[e];
        sm.NL[e].n = m * __ldg(Sel<T>::invx(G) + k);  // N = M / x through the table of 1 / x
        if (sizeof(T) != sizeof(double)) sm.Mt[e] = m;
      }
      __syncthreads();

      // 2. requested loss R and limiter ratios. The active columns (species b, bin j) are
      //    listed once in shared memory as (Kr offset, N), padded with zero entries to a
      //    multiple of 8; Kr is i-fastest, so for a fixed column the rows' entries are
      //    contiguous and the offset (b, j) is the same for every row. One item per (pair of
      //    adjacent rows of one species, run of the list): the two rows share each column's
      //    offset and N, and keep four partial sums each (eight loads in flight); the item parks
      //    its sums in the gain arrays (free until the gain pass); then one lane per row adds
      //    its runs in order and forms R and lambda in FP64.
      using Sum = typename Num<T>::Sum;
      Sum* const part = sm.stay;  // [run][E] partial row sums, reaching into sm.up, which follows
      bool limited = false;
      const T* __restrict__ Kr = Sel<T>::Kr(G);
      const T* __restrict__ Krd = lev ? Sel<T>::Kr_d(G) : nullptr;
      int NC = 0;  // active columns, then padded to a multiple of 8
      for (int b = 0; b < ns; ++b) NC += max(0, s_hi[b] - s_lo[b] + 1);
      const int NCp = (NC + 7) & ~7;
      for (int e = tid; e < max(E, NCp); e += NT) {
        if (e < E) {
          const int b = div_n(e, G.inv_n), j = e - b * n;
          if (j >= s_lo[b] && j <= s_hi[b]) {
            int pos = j - s_lo[b];
            for (int b2 = 0; b2 < b; ++b2) pos += max(0, s_hi[b2] - s_lo[b2] + 1);
            sm.loff[pos] = (s_sp[b] * n + j) * n;
            sm.lN[pos] = sm.NL[e].n;
          }
        }
        if (e >= NC && e < NCp) {
          sm.loff[e] = 0;
          sm.lN[e] = T(0);
        }
      }
      __syncthreads();
      {
        const int nch = loss_runs(NCp, ns), span = loss_span(NCp, nch);
        for (int it = tid; it < nch * RP; it += NT) {
          const int ch = div_by(it, RP, inv_RP), rp = it - ch * RP;
          const int a = div_by(rp, H, inv_H), i = 2 * (rp - a * H), r = a * n + i;
          Acc<T> acc0, acc1;
          if (((i >= s_lo[a] && i <= s_hi[a]) || (i + 1 < n && i + 1 >= s_lo[a] && i + 1 <= s_hi[a])) &&
              (!FSBM_CHECKED_BUILD || (FSBM_OK(t.chk, s_sp[a], S) && FSBM_OK(t.chk, nch * E - 1, 2 * S * S * nmax)))) {
            // rows i and i + 1 (which for i = n - 1 reads past the row into the next column, or
            // into the table's zero padding, and is dropped)
            const T* __restrict__ Krow = Kr + (size_t)s_sp[a] * S * n * n + i;
            const T* __restrict__ Krowd = lev ? Krd + (size_t)s_sp[a] * S * n * n + i : nullptr;
            const int qa = ch * span, qb = min(NCp, qa + span);
            for (int q0 = qa; q0 < qb; q0 += kLossRun) {
              const int q1 = min(qb, q0 + kLossRun);
              T p0[4], p1[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) p0[u] = p1[u] = T(0);
              for (int q = q0; q < q1; q += 8) {
                int o[8];
                T nj[8], k0[8], k1[8];
                lds8(sm.loff + q, o);
                lds8(sm.lN + q, nj);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  k0[u] = __ldg(Krow + o[u]);
                  k1[u] = __ldg(Krow + o[u] + 1);
                }
                if (lev) {
#pragma unroll
                  for (int u = 0; u < 8; ++u) {
                    k0[u] = fma(wT, __ldg(Krowd + o[u]), k0[u]);
                    k1[u] = fma(wT, __ldg(Krowd + o[u] + 1), k1[u]);
                  }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  p0[u & 3] = fma(k0[u], nj[u], p0[u & 3]);
                  p1[u & 3] = fma(k1[u], nj[u], p1[u & 3]);
                }
              }
              acc0.add((p0[0] + p0[1]) + (p0[2] + p0[3]));
              acc0.flush();
              acc1.add((p1[0] + p1[1]) + (p1[2] + p1[3]));
              acc1.flush();
            }
          }
          part[ch * E + r] = acc0.sum();
          if (i + 1 < n) part[ch * E + r + 1] = acc1.sum();
        }
        __syncthreads();
        bool fired = false;
        for (int r = tid; r < E; r += NT) {
          const int a = div_n(r, G.inv_n), i = r - a * n;
          double R = 0.0;
          double lamd = 1.0;
          if (i >= s_lo[a] && i <= s_hi[a]) {
            Sum tot = part[r];
            for (int ch = 1; ch < nch; ++ch) Num<T>::add(tot, part[ch * E + r]);
            R = dt * sm.M[r] * Num<T>::val(tot);
            if (R > sm.M[r]) {  // lambda = M / R < 1 (R > 0 here)
              lamd = sm.M[r] / R;
              fired = true;
            }
          }
          sm.loss[r] = R;
          sm.NL[r].l = (T)lamd;
          if (sizeof(T) == sizeof(double)) sm.nlam[r] = sm.NL[r].n * (T)lamd;
        }
        if (tid == 0) s_task = 0;
        limited = __syncthreads_or(fired);
      }
      if (limited) status |= 1;

      // 3. limited losses: loss_i = dt M_i sum_j K N_j min(lam_i, lam_j)
      //      = lam_i R_i + dt M_i sum_{j limited} K N_j (min(lam_i, lam_j) - lam_i),
      //    where lam_i R_i = M_i when lam_i < 1 and every term with lam_j >= lam_i is 0. The
      //    limited rows are listed in row order as columns (Kr offset, N, lambda), padded with
      //    zero entries to a multiple of 8; one item per (row pair, run of the list) as in the
      //    requested loss; then one lane per row adds its runs in order.
      if (limited) {
        if (warp == 0) {
          int cnt = 0;
          for (int r0 = 0; r0 < E; r0 += 32) {
            const int r = r0 + lane;
            const bool f = r < E && sm.NL[r].l < T(1);
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f && FSBM_OK(t.chk, cnt + __popc(bal & ((1u << lane) - 1u)), E))
              sm.lim[cnt + __popc(bal & ((1u << lane) - 1u))] = r;
            cnt += __popc(bal);
          }
          if (lane == 0) s_nlim = cnt;
        }
        __syncthreads();
        const int L = s_nlim, Lp = (L + 7) & ~7;
        for (int q = tid; q < Lp; q += NT) {
          if (q < L) {
            const int r = sm.lim[q];
            const int b = div_n(r, G.inv_n), j = r - b * n;
            sm.llam[q] = sm.NL[r].l;
            sm.lN[q] = sm.NL[r].n;
            sm.loff[q] = (s_sp[b] * n + j) * n;
            if (sizeof(T) == sizeof(double)) sm.lNl[q] = sm.nlam[r];
          } else {
            sm.llam[q] = T(1);
            sm.lN[q] = T(0);
            sm.loff[q] = 0;
            if (sizeof(T) == sizeof(double)) sm.lNl[q] = T(0);
          }
        }
        __syncthreads();
        const int nch = loss_runs(Lp, ns), span = loss_span(Lp, nch);
        for (int it = tid; it < nch * RP; it += NT) {
          const int ch = div_by(it, RP, inv_RP), rp = it - ch * RP;
          const int a = div_by(rp, H, inv_H), i = 2 * (rp - a * H), r = a * n + i;
          Acc<T> acc0, acc1;
          if (((i >= s_lo[a] && i <= s_hi[a]) || (i + 1 < n && i + 1 >= s_lo[a] && i + 1 <= s_hi[a])) &&
              (!FSBM_CHECKED_BUILD || (FSBM_OK(t.chk, s_sp[a], S) && FSBM_OK(t.chk, L, E + 1) &&
                                       FSBM_OK(t.chk, nch * E - 1, 2 * S * S * nmax)))) {
            const T li0 = sm.NL[r].l, li1 = i + 1 < n ? sm.NL[r + 1].l : T(1);
            const T* __restrict__ Krow = Kr + (size_t)s_sp[a] * S * n * n + i;
            const T* __restrict__ Krowd = lev ? Krd + (size_t)s_sp[a] * S * n * n + i : nullptr;
            const int qa = ch * span, qb = min(Lp, qa + span);
            for (int q0 = qa; q0 < qb; q0 += kLossRun) {
              const int q1 = min(qb, q0 + kLossRun);
              T p0[4], p1[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) p0[u] = p1[u] = T(0);
              for (int q = q0; q < q1; q += 8) {
                int o[8];
                T nj[8], lj[8], k0[8], k1[8];
                lds8(sm.loff + q, o);
                lds8(sm.lN + q, nj);
                lds8(sm.llam + q, lj);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  k0[u] = __ldg(Krow + o[u]);
                  k1[u] = __ldg(Krow + o[u] + 1);
                }
                if (lev) {
#pragma unroll
                  for (int u = 0; u < 8; ++u) {
                    k0[u] = fma(wT, __ldg(Krowd + o[u]), k0[u]);
                    k1[u] = fma(wT, __ldg(Krowd + o[u] + 1), k1[u]);
                  }
                }
                if (sizeof(T) == sizeof(double)) {
                  // FP64: (min(l_i, l_j) - l_i) N_j is 0 for l_j >= l_i and N_j l_j - l_i N_j
                  // otherwise: one multiply-add on the listed N_j l_j and a select on the bit
                  // patterns (non-negative ratios order like integers), two FP64 operations a term
                  T nlj[8];
                  lds8(sm.lNl + q, nlj);
#pragma unroll
                  for (int u = 0; u < 8; ++u) {
                    const T t0 = lt_nonneg(lj[u], li0) ? fma(-li0, nj[u], nlj[u]) : T(0);
                    const T t1 = lt_nonneg(lj[u], li1) ? fma(-li1, nj[u], nlj[u]) : T(0);
                    p0[u & 3] = fma(k0[u], t0, p0[u & 3]);
                    p1[u & 3] = fma(k1[u], t1, p1[u & 3]);
                  }
                } else {
#pragma unroll
                  for (int u = 0; u < 8; ++u) {
                    p0[u & 3] = fma((min_nonneg(li0, lj[u]) - li0) * k0[u], nj[u], p0[u & 3]);
                    p1[u & 3] = fma((min_nonneg(li1, lj[u]) - li1) * k1[u], nj[u], p1[u & 3]);
                  }
                }
              }
              acc0.add((p0[0] + p0[1]) + (p0[2] + p0[3]));
              acc0.flush();
              acc1.add((p1[0] + p1[1]) + (p1[2] + p1[3]));
              acc1.flush();
            }
          }
          part[ch * E + r] = acc0.sum();
          if (i + 1 < n) part[ch * E + r + 1] = acc1.sum();
        }
        __syncthreads();
        for (int r = tid; r < E; r += NT) {
          const int a = div_n(r, G.inv_n), i = r - a * n;
          if (i < s_lo[a] || i > s_hi[a]) continue;
          Sum tot = Num<T>::zero();
          for (int ch = 0; ch < nch; ++ch) Num<T>::add(tot, part[ch * E + r]);
          const T li = sm.NL[r].l;
          const double base = li < T(1) ? sm.M[r] : sm.loss[r];
          sm.loss[r] = base + dt * sm.M[r] * Num<T>::val(tot);
        }
        __syncthreads();  // the partial sums live in the gain arrays
      }

      // 4. gains. Lanes run over the flattened list of (target bin 1..n-2, orientation)
      //    items, orientation fastest: a warp covers about 32/O consecutive targets, whose
      //    distance ranges differ by a few steps at most, so nearly every lane stays busy,
      //    and the lanes of one (d, m) read one contiguous run of Kd. The top bin's items
      //    (the most pairs, but no flux) get warp tasks of their own, so that no warp runs
      //    its flux for a few lanes while the rest walk the top bin; the list is padded at
      //    its cheap end (low k), where a partly filled warp costs least. Warps claim the
      //    top tasks first, then the others costliest first (the cost grows with k).
      {
        const int n_reg = ((n - 2) * O) << lgP;  // lanes: P per item, an item's parts adjacent
        const int n_reg_tasks = (n_reg + 31) >> 5;
        const int pad = n_reg_tasks * 32 - n_reg;  // a multiple of P: parts never straddle warps
        const int n_top_tasks = ((O << lgP) + 31) >> 5;
        const int n_tasks = n_top_tasks + n_reg_tasks;
        for (;;) {
          int q = 0;
          if (lane == 0) q = atomicAdd(&s_task, 1);
          q = __shfl_sync(0xffffffffu, q, 0);
          if (q >= n_tasks) break;
          bool on;
          int ol, k, part;
          if (q < n_top_tasks) {
            const int f = q * 32 + lane;
            on = f < (O << lgP);
            ol = on ? f >> lgP : 0;
            part = f & (P - 1);
            k = n - 1;
          } else {
            const int f = (n_reg_tasks - 1 - (q - n_top_tasks)) * 32 + lane - pad;
            on = f >= 0;
            const int it = on ? f >> lgP : 0;
            const int kq = div_by(it, O, inv_O);
            ol = it - kq * O;
            part = on ? f & (P - 1) : 0;
            k = kq + 1;
          }
          typename Num<T>::Sum st_, up_;
#define FSBM_GAIN(LIM, LV, TP)                                                                          \
  gain_task<T, LIM, LV, TP>(G, S * S, sm, ori[ol], s_lo, s_hi, k, on, part, P, dtT, Bs, t.math, wT, &st_, \
                            &up_)
          const bool top_task = q < n_top_tasks;
          if (LEV && lev) {
            if (limited) {
              if (top_task) FSBM_GAIN(true, LEV, true); else FSBM_GAIN(true, LEV, false);
            } else {
              if (top_task) FSBM_GAIN(false, LEV, true); else FSBM_GAIN(false, LEV, false);
            }
          } else {
            if (limited) {
              if (top_task) FSBM_GAIN(true, false, true); else FSBM_GAIN(true, false, false);
            } else {
              if (top_task) FSBM_GAIN(false, false, true); else FSBM_GAIN(false, false, false);
            }
          }
#undef FSBM_GAIN
          // the parts' sums, added pairwise across adjacent lanes (a fixed order); part 0 keeps them
          for (int off = 1; off < P; off <<= 1) {
            shfl_add<T>(st_, off);
            shfl_add<T>(up_, off);
          }
          if (on && part == 0 && FSBM_OK(t.chk, ol * n + k, O * n)) {
            sm.stay[ol * n + k] = st_;
            sm.up[ol * n + k] = up_;
          }
        }
      }
      if (tid < O) {  // bin 0 of every orientation receives nothing
        sm.stay[tid * n] = Num<T>::zero();
        sm.up[tid * n] = Num<T>::zero();
      }
      __syncthreads();

      // 5. update, mass error, clamp, renormalise (FP64). The pre-clamp values go to `loss`
      //    (no longer needed) so that one warp forms both totals in a fixed order.
      for (int e = tid; e < E; e += NT) {
        const int c = div_n(e, G.inv_n), k = e - c * n;
        typename Num<T>::Sum gsum = Num<T>::zero();
        for (int qq = 0; qq < s_np[c]; ++qq) {
          const int q = s_plist[c][qq];
          if (FSBM_CHECKED_BUILD && !FSBM_OK(t.chk, (size_t)q * n + k, (size_t)O * n)) continue;
          Num<T>::add(gsum, sm.stay[q * n + k]);
          if (k > 0) Num<T>::add(gsum, sm.up[q * n + k - 1]);
        }
        const double v = sm.M[e] - sm.loss[e] + Num<T>::val(gsum);
        sm.loss[e] = v;
        sm.M[e] = v < 0.0 ? 0.0 : v;
      }
      __syncthreads();
      if (warp == 0) {
        double pre = 0.0, post = 0.0;
        for (int e = lane; e < E; e += 32) {
          pre += sm.loss[e];
          post += sm.M[e];
        }
        pre = warp_sum(pre);
        post = warp_sum(post);
        if (lane == 0) {
          emax = fmax(emax, fabs(pre - Bs) * inv_B0);  // thread 0 keeps the running maximum
          red[1] = Bs / post;
        }
      }
      __syncthreads();
      const double scale = red[1];
      for (int e = tid; e < E; e += NT) sm.M[e] = sm.M[e] * scale;
      __syncthreads();
    }

    for (int e = tid; e < E; e += NT) spec[e] = (Store)sm.M[e];
    if (tid == 0) {
      pd.status[p] = status;
      pd.mass_budget[p] = B0;
      pd.mass_error[p] = emax;
    }
    (void)lane;
  }
}

template <typename T, bool LEV>
cudaError_t plan_t(const Tables& t, int block_dim, int n_sms, CoalLaunch* out) {
  int nmax = 0;
  for (int g = 0; g < t.G; ++g) nmax = t.g[g].n > nmax ? t.g[g].n : nmax;
  const size_t smem = Smem<T>::bytes(nmax, t.S);
  auto* kern = k_coal<T, LEV>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // Give shared memory what the register-limited number of resident CTAs needs and leave the
  // rest of the SM's 256 KB to L1 (the kernel and math tables are read through it).
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  int dev = 0, regs_sm = 0, smem_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  const int regs_cta = ((fa.numRegs * 32 + 255) / 256 * 256) * (block_dim / 32);  // per-warp allocation unit 256
  const int by_regs = std::max(regs_cta > 0 ? regs_sm / regs_cta : 1, 1);
  const size_t need = (size_t)by_regs * (smem + fa.sharedSizeBytes + 1024);
  const int carve = (int)std::min<size_t>(100, (need * 100 + smem_sm - 1) / std::max(smem_sm, 1));
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve)) != cudaSuccess)
    return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block_dim, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  out->block_dim = block_dim;
  out->grid_dim = per_sm * n_sms;
  out->smem = smem;
  return cudaSuccess;
}

}  // namespace

namespace {
__global__ void k_math_check(MathTabs mt, double* out) {
  // sweep: log over [1e-300, 1e300] geometrically, exp/expm1 over [-700, 700] and densely near 0
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = gridDim.x * blockDim.x;
  double el = 0.0, ee = 0.0, em = 0.0, es = 0.0, er = 0.0;
  for (int q = tid; q < (1 << 20); q += n) {
    const double u = (q + 0.5) / (double)(1 << 20);
    const double x = exp((u - 0.5) * 1381.0);            // 1e-300 .. 1e300
    const double rl = log(x);
    el = fmax(el, fabs(fsbm_log(x, mt) - rl) / fmax(fabs(rl), 1.0));  // absolute near x = 1
    const double y = (u - 0.5) * 1400.0;
    double ex, e1;
    fsbm_exp_em1(y, mt, &ex, &e1);
    ee = fmax(ee, fabs(ex - exp(y)) / exp(y));
    const double ys = (u - 0.5) * 1e-3 * ((q & 7) + 1);
    fsbm_exp_em1(ys, mt, &ex, &e1);
    const double r1 = expm1(ys);
    if (r1 != 0.0) em = fmax(em, fabs(e1 - r1) / fabs(r1));
    fsbm_exp_em1(y * 1e-2, mt, &ex, &e1);
    const double r2 = expm1(y * 1e-2);
    if (r2 != 0.0) em = fmax(em, fabs(e1 - r2) / fabs(r2));
    es = fmax(es, fabs(fsbm_rsqrt(x) - rsqrt(x)) * sqrt(x));
    const double xr = (q & 1) ? -x : x;
    er = fmax(er, fabs(fsbm_rcp(xr) * xr - 1.0));
  }
  __shared__ double red[5][256];
  red[0][threadIdx.x] = el;
  red[1][threadIdx.x] = ee;
  red[2][threadIdx.x] = em;
  red[3][threadIdx.x] = es;
  red[4][threadIdx.x] = er;
  __syncthreads();
  if (threadIdx.x < 5) {
    double m = 0.0;
    for (int i = 0; i < blockDim.x; ++i) m = fmax(m, red[threadIdx.x][i]);
    // blocks combine through a CAS-free max on the bit pattern (non-negative doubles order
    // like their bit patterns)
    atomicMax(reinterpret_cast<unsigned long long*>(out) + threadIdx.x,
              (unsigned long long)__double_as_longlong(m));
  }
}
}  // namespace

cudaError_t launch_math_check(const Tables& t, double* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, 5 * sizeof(double), stream);
  if (e != cudaSuccess) return e;
  k_math_check<<<64, 256, 0, stream>>>(t.math, out);
  return cudaGetLastError();
}

size_t coal_smem_bytes(const Tables& t, int precision) {
  int nmax = 0;
  for (int g = 0; g < t.G; ++g) nmax = t.g[g].n > nmax ? t.g[g].n : nmax;
  return precision == 0 ? Smem<double>::bytes(nmax, t.S) : Smem<float>::bytes(nmax, t.S);
}

cudaError_t coal_plan(const Tables& t, int precision, int block_dim, int n_sms, CoalLaunch* out) {
  if (t.mode == 1) return sweep_plan(block_dim, n_sms, out);
  if (t.levels)
    return precision == 0 ? plan_t<double, true>(t, block_dim, n_sms, out) : plan_t<float, true>(t, block_dim, n_sms, out);
  return precision == 0 ? plan_t<double, false>(t, block_dim, n_sms, out) : plan_t<float, false>(t, block_dim, n_sms, out);
}

cudaError_t launch_coal(const Tables& t, int precision, const PointsDev& p, const Scratch& s, double dt,
                        int n_steps, const CoalLaunch& plan, cudaStream_t stream) {
  if (t.mode == 1) return launch_sweep(t, p, s, dt, n_steps, plan, stream);
  int nmax = 0;
  for (int g = 0; g < t.G; ++g) nmax = t.g[g].n > nmax ? t.g[g].n : nmax;
  // all four instantiations share one signature
  void (*kern)(Tables, PointsDev, const int32_t*, int32_t*, double, int, int) =
      precision == 0 ? (t.levels ? k_coal<double, true> : k_coal<double, false>)
                     : (t.levels ? k_coal<float, true> : k_coal<float, false>);
  kern<<<plan.grid_dim, plan.block_dim, plan.smem, stream>>>(t, p, s.active_list, s.counters, dt, n_steps, nmax);
  return cudaGetLastError();
}

}  // namespace fsbm
