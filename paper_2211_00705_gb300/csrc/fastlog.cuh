// Low-latency FP64 natural logarithm for the boundary solves (whose chains are latency bound):
// Tang's table-driven method (P. T. P. Tang, "Table-driven implementation of the logarithm function in
// IEEE floating-point arithmetic", ACM TOMS 16(4), 1990). x = 2^k m with m in [sqrt(1/2), sqrt(2));
// c = j/128 is the grid point nearest m, r = (m - c)/c (m - c is exact), and
// ln x = k ln2 + ln c + ln(1 + r), where ln(1 + r) is the Taylor series to r^8 (|r| < 0.0056 keeps the
// truncation below 2^-60 relative) evaluated with Estrin's scheme. ln c and k ln2 are carried as
// high/low pairs. Valid for positive normal finite x; anything else goes to the library log.
#pragma once

namespace imexds {

constexpr int kLogJ0 = 90;    // first table index (90/128 < sqrt(1/2))
constexpr int kLogJN = 93;    // entries for j = 90 .. 182
struct LogTable {
  double c[kLogJN];           // j / 128 (exact)
  double inv_c[kLogJN];       // 128 / j rounded
  double lnc_hi[kLogJN];      // ln(j/128) rounded to double ...
  double lnc_lo[kLogJN];      // ... and the remainder
};

__device__ LogTable g_logtab;  // filled by the host before the first kernel that uses fast_log

__device__ __forceinline__ double fast_log(double x) {
  int hi = __double2hiint(x);
  int lo = __double2loint(x);
  int e = (hi >> 20) & 0x7ff;
  if (e == 0 || e == 0x7ff || hi < 0) return log(x);  // zero, subnormal, inf, nan, negative
  int k = e - 1023;
  int frac = hi & 0x000fffff;                        // top 20 bits of the fraction f of m = 1 + f
  int mhi = frac | 0x3ff00000;                       // m in [1, 2)
  int j;
  if (frac >= 0x6a09e) {                             // m >= sqrt(2) (to 20 bits): use m/2, k + 1
    mhi -= 0x00100000;
    k += 1;
    j = 64 + ((frac + (1 << 13)) >> 14);             // round(64 (1 + f)), integer arithmetic only
  } else {
    j = 128 + ((frac + (1 << 12)) >> 13);            // round(128 (1 + f))
  }
  double m = __hiloint2double(mhi, lo);
  int t = j - kLogJ0;
  double r = (m - __ldg(&g_logtab.c[t])) * __ldg(&g_logtab.inv_c[t]);
  // ln(1 + r) = r - r^2/2 + r^3/3 - ... - r^8/8 by Estrin's scheme
  double r2 = r * r;
  double r4 = r2 * r2;
  double a = __fma_rn(-0.5, r, 1.0);
  double b = __fma_rn(-0.25, r, 1.0 / 3.0);
  double cc = __fma_rn(-1.0 / 6.0, r, 0.2);
  double dd = __fma_rn(-0.125, r, 1.0 / 7.0);
  double p = r * __fma_rn(r4, __fma_rn(r2, dd, cc), __fma_rn(r2, b, a));
  const double LN2_HI = 6.93147180369123816490e-01;  // ln 2 with the low 21 bits zero (k LN2_HI is exact)
  const double LN2_LO = 1.90821492927058770002e-10;  // ln 2 - LN2_HI
  double kd = (double)k;
  double s_hi = __fma_rn(kd, LN2_HI, __ldg(&g_logtab.lnc_hi[t]));
  double s_lo = __fma_rn(kd, LN2_LO, __ldg(&g_logtab.lnc_lo[t]));
  return s_hi + (s_lo + p);
}

}  // namespace imexds
