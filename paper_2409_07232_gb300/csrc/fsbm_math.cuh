// fsbm_math.cuh -- table-driven FP64 logarithm and exponential for the FP64 pair flux.
//
// GB300 runs FP64 at about 1/64 of its FP32 rate, so the FP64 form of the collision kernel is
// bound by FP64 instructions per bin pair, most of which go to the logarithm and the two
// exponentials of Bott's flux. These routines follow P. T. P. Tang's table-driven methods
// ("Table-driven implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989; "... the logarithm function ...", ACM TOMS 16(4),
// 1990; "... the expm1 function ...", ACM TOMS 18(2), 1992): a table reduces the argument to
// a short interval, a low-degree Taylor polynomial finishes it, and integer operations
// handle the binary exponent. The polynomial degrees are cut to what the flux needs (its
// result must agree to 1e-12): about 1e-16 absolute for ln, 1e-15 relative for e^y and
// e^y - 1, checked against CUDA's log/exp/expm1 by fsbm_coal_math_check.
//
// Tables (built on the host in FP64, copied to the device once per context):
//   logtab[2*(j+75)], logtab[2*(j+75)+1] = 1 / F_j, ln F_j for F_j = 1 + j/256, j = -75..106
//                                           (F covers [1/sqrt2, sqrt2], the reduced mantissa)
//   exptab[2*j], exptab[2*j+1]  = 2^(j/64) = hi + lo (lo: the rounding error of hi)
#pragma once
#include <cstdint>

namespace fsbm {

constexpr int kLogTabLo = -75;
constexpr int kLogTab = 182;
constexpr int kExpTab = 64;

// The constants: ln 2 = hi + lo with the 32 low mantissa bits of hi cleared, so that e * hi is
// exact for |e| < 2^11 and N * hi / 64 for |N| < 2^17; and 64 / ln 2. Built on the host.
struct MathTabs {
  const double* logtab;   // [2 * kLogTab]
  const double* exptab;   // [2 * kExpTab]
  double ln2_hi, ln2_lo;   // ln 2 = hi + lo
  double l64_hi, l64_lo;   // (ln 2) / 64 = hi + lo (the above divided by 64, exactly)
  double inv_l64;          // 64 / ln 2
  double ln_eps, sqrt_eps; // ln(1e-60) and e^{ln(1e-60)/2}: Bott's constant in the flux
};

// ln x for normal x > 0 (callers guarantee x >= 1e-300). x = 2^e m with m in
// [1/sqrt2, sqrt2), so e = 0 near x = 1 and no table rounding is left to cancel there.
__device__ __forceinline__ double fsbm_log(double x, const MathTabs& mt) {
  const double* __restrict__ logtab = mt.logtab;
  const int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  int e = (hi >> 20) - 1023;
  const int mb = hi & 0x000fffff;
  int j;
  double m;
  if (mb >= 0x6a09e) {                              // mantissa >= sqrt2: halve it
    e += 1;
    m = __hiloint2double(mb | 0x3fe00000, lo);      // in [1/sqrt2, 1)
    j = ((mb - 0x100000) + 0x1000) >> 13;           // nearest (m - 1) * 256, in [-75, 0]
  } else {
    m = __hiloint2double(mb | 0x3ff00000, lo);      // in [1, sqrt2)
    j = (mb + 0x800) >> 12;                         // nearest (m - 1) * 256, in [0, 106]
  }
  const double F = fma((double)j, 1.0 / 256.0, 1.0);
  const double f = m - F;                           // exact: |f| <= 1/512
  const int t = 2 * (j - kLogTabLo);
  const double u = f * __ldg(logtab + t);           // f / F, |u| <= 2^-8.5
  // ln(1 + u) = u - u^2/2 + u^3/3 - u^4/4 + u^5/5; the next term is below 2^-51 / 6 = 7e-17
  // (absolute), which is the accuracy the flux needs: it uses differences of logarithms.
  double q = fma(u, 1.0 / 5.0, -0.25);
  q = fma(q, u, 1.0 / 3.0);
  q = fma(q, u, -0.5);
  const double lp = fma(u * u, q, u);
  const double de = (double)e;
  return fma(de, mt.ln2_hi, __ldg(logtab + t + 1)) + fma(de, mt.ln2_lo, lp);
}

// e^y (*ex) and e^y - 1 (*em1) for |y| <= 700, from one reduction:
// y = (64 M + j) ln2/64 + r, |r| <= ln2/128, e^y = 2^M 2^(j/64) (1 + p(r)).
// e^y - 1 = (s - 1) + s p with s = 2^M 2^(j/64); s - 1 is exact whenever the result is
// small (M = 0, j = 0 near y = 0), which is what keeps e^y - 1 accurate there.
__device__ __forceinline__ void fsbm_exp_em1(double y, const MathTabs& mt, double* ex, double* em1) {
  const double* __restrict__ exptab = mt.exptab;
  const double t = y * mt.inv_l64;
  const double Nd = rint(t);
  const int N = (int)Nd;
  double r = fma(-Nd, mt.l64_hi, y);
  r = fma(-Nd, mt.l64_lo, r);
  // e^r - 1 = r + r^2/2 + r^3/6 + r^4/24 + r^5/120; the next term is below 7e-15 of the
  // result (|r| <= ln2/128), the relative accuracy the flux needs for e^y - 1 near y = 0
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(r * r, p, r);
  const int jj = N & 63;
  const int M = N >> 6;                            // floor division
  // s = 2^M * 2^(jj/64) = s_hi + s_lo: add M to the exponent field of both table parts
  const double th = __ldg(exptab + 2 * jj), tl = __ldg(exptab + 2 * jj + 1);
  const int sh = (int)((unsigned)M << 20);
  const double s_hi = __hiloint2double(__double2hiint(th) + sh, __double2loint(th));
  const double s_lo = tl * __hiloint2double((M + 1023) << 20, 0);  // tl 2^M (tl is tiny: scale by multiply)
  const double tail = fma(s_hi, p, s_lo * (1.0 + p));  // s p + s_lo, the small part
  *ex = s_hi + tail;
  *em1 = (s_hi - 1.0) + tail;                      // s_hi - 1 is exact when the result is small
}

__device__ __forceinline__ double fsbm_exp(double y, const MathTabs& mt) {
  double ex, em1;
  fsbm_exp_em1(y, mt, &ex, &em1);
  return ex;
}

}  // namespace fsbm
