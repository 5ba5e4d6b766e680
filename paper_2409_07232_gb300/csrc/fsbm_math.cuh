// fsbm_math.cuh -- table-driven FP64 logarithm and exponential for the FP64 pair flux.
//
// GB300 runs FP64 at about 1/64 of its FP32 rate, so the FP64 form of the collision kernel is
// bound by FP64 instructions per bin pair, most of which go to the logarithm and the
// exponential of Bott's flux. These routines follow P. T. P. Tang's table-driven methods
// ("Table-driven implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989; "... the logarithm function ...", ACM TOMS 16(4),
// 1990; "... the expm1 function ...", ACM TOMS 18(2), 1992): a table reduces the argument to
// a short interval, a low-degree Taylor polynomial finishes it, and integer operations
// handle the binary exponent, the table index and the reduced argument's table point (the
// integer pipes are idle in this kernel, the FP64 pipe is not). The tables are large enough
// that degree-4 polynomials reach what the flux needs (its result must agree to 1e-12):
// about 2e-16 absolute for ln (the flux only uses differences of logarithms), 4e-16 relative
// for e^y and 3e-14 relative for e^y - 1 (near y = 0, where the series' r^4/120 decides),
// checked against CUDA's log/exp/expm1 by fsbm_coal_math_check.
//
// Tables (built on the host in extended precision, rounded to FP64, copied to the device once
// per context), each read as one 16-byte load per call:
//   logtab[j] = (1 / F_j, ln F_j) for F_j = 1 + j/512, j = 0..512
//   etab[b]   = (e ln2_hi, e ln2_lo) for e = b - 1023, b = 0..2047 (e ln2_hi exact)
//   exptab[j] = (hi, lo) with hi + lo = 2^(j/256), j = 0..255 (lo: the rounding error of hi)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fsbm {

constexpr int kLogTab = 513;
constexpr int kExpTab = 256;

// ln 2 = hi + lo with the 32 low mantissa bits of hi cleared, so that e * hi is exact for
// |e| < 2^11 and N * hi / 256 for |N| < 2^20; and 256 / ln 2. Built on the host.
struct MathTabs {
  const double2* logtab;   // [kLogTab]
  const double2* exptab;   // [kExpTab]
  const double2* etab;     // [2048] (e ln2_hi, e ln2_lo) for the biased exponent e + 1023
  double ln2_hi, ln2_lo;   // ln 2 = hi + lo
  double l256_hi, l256_lo; // (ln 2) / 256 = hi + lo (the above divided by 256, exactly)
  double inv_l256;         // 256 / ln 2
  double ln_eps, sqrt_eps; // ln(1e-60) and e^{ln(1e-60)/2}: Bott's constant in the flux
};

// ln x for normal x > 0 (callers guarantee x >= 1e-300), absolute error about 2e-16 plus the
// rounding of the result. x = 2^e m with m in [1, 2); F = 1 + j/512 is the table point
// nearest m, built from the index bits (so m - F is exact, |m - F| <= 2^-10) and
// ln x = e ln2 + ln F + ln(1 + u) with u = (m - F) / F, |u| <= 2^-10. e ln2 comes from a
// table indexed by the exponent bits (a load instead of an integer-to-FP64 conversion,
// which would take an FP64-pipe slot).
__device__ __forceinline__ double fsbm_log(double x, const MathTabs& mt) {
  const int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  const int mb = hi & 0x000fffff;
  const int j = (mb + 0x400) >> 11;                         // nearest j / 512, in [0, 512]
  const double m = __hiloint2double(mb | 0x3ff00000, lo);   // in [1, 2)
  const double F = __hiloint2double(0x3ff00000 + (j << 11), 0);
  const double2 t = __ldg(mt.logtab + j);
  const double u = (m - F) * t.x;
  // ln(1 + u) = u - u^2/2 + u^3/3 - u^4/4; the next term is below 2^-50 / 5 = 1.8e-16
  double q = fma(u, -0.25, 1.0 / 3.0);
  q = fma(q, u, -0.5);
  const double lp = fma(u * u, q, u);
  const double2 te = __ldg(mt.etab + (hi >> 20));
  return (te.x + t.y) + (te.y + lp);
}

// e^y (*ex) and e^y - 1 (*em1) for |y| <= 700, from one reduction:
// y = (256 M + j) ln2/256 + r, |r| <= ln2/512, e^y = 2^M 2^(j/256) (1 + p(r)).
// e^y - 1 = (s - 1) + s p with s = 2^M 2^(j/256); s - 1 is exact whenever the result is
// small (M = 0, j = 0 near y = 0), which is what keeps e^y - 1 accurate there.
__device__ __forceinline__ void fsbm_exp_em1(double y, const MathTabs& mt, double* ex, double* em1) {
  // N = nearest integer to 256 y / ln2: adding 1.5 * 2^52 rounds it into the low word
  constexpr double kShift = 6755399441055744.0;  // 1.5 * 2^52
  const double kd = fma(y, mt.inv_l256, kShift);
  const int N = __double2loint(kd);
  const double Nd = kd - kShift;
  double r = fma(-Nd, mt.l256_hi, y);
  r = fma(-Nd, mt.l256_lo, r);
  // e^r - 1 = r + r^2/2 + r^3/6 + r^4/24; the next term is r^4/120 <= 2.8e-14 of the
  // result (|r| <= ln2/512), which bounds e^y - 1's relative error near y = 0
  double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(r * r, p, r);
  const int jj = N & 255;
  const int M = N >> 8;                            // floor division
  // s = 2^M * 2^(jj/256) = s_hi + s_lo: add M to the exponent field of both table parts.
  // lo is 0 at jj = 0; where lo 2^M would leave the normal range it is below 2^-1022 and
  // is dropped.
  const double2 t = __ldg(mt.exptab + jj);
  const int sh = (int)((unsigned)M << 20);
  const double s_hi = __hiloint2double(__double2hiint(t.x) + sh, __double2loint(t.x));
  const int lh = __double2hiint(t.y);
  const int le = (lh >> 20) & 0x7ff;
  const double s_lo = (le != 0 && le + M > 0) ? __hiloint2double(lh + sh, __double2loint(t.y)) : 0.0;
  const double tail = fma(s_hi, p, s_lo);          // s p + s_lo (s_lo p is below 2^-60 s)
  *ex = s_hi + tail;
  *em1 = (s_hi - 1.0) + tail;                      // s_hi - 1 is exact when the result is small
}

__device__ __forceinline__ double fsbm_exp(double y, const MathTabs& mt) {
  double ex, em1;
  fsbm_exp_em1(y, mt, &ex, &em1);
  return ex;
}

}  // namespace fsbm
