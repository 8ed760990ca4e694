// vc_maps.cuh -- device arithmetic of the cipher's chaotic generators.
//
// Every floating-point operation is an explicit IEEE-754 binary64
// round-to-nearest intrinsic (__dadd_rn, __dmul_rn, __ddiv_rn, ...), so the
// compiler can neither contract a multiply-add into an FMA nor reorder
// anything: the results are bit-identical to any other binary64 evaluation in
// the same operation order.
#pragma once
#include <cstdint>

#include "vc_ieee.cuh"

namespace vc {

// ---- the cipher's sine (reading of "sin" in Eq. 1 and Eq. 6) ----------------
// k = floor(t * 2/pi + 1/2); r = (t - k*PIO2_HI) - k*PIO2_LO (Cody-Waite, 33-bit
// head so k*PIO2_HI is exact); quadrant k mod 4 selects +-sin(r) / +-cos(r);
// Taylor polynomials in r^2 by Horner, sin to degree 17, cos to degree 16.
static constexpr double kPi = 0x1.921fb54442d18p+1;       // nearest double to pi
static constexpr double kTwoPi = 0x1.921fb54442d18p+2;    // nearest double to 2 pi
static constexpr double kTwoOverPi = 0x1.45f306dc9c883p-1; // nearest double to 2/pi
static constexpr double kPio2Hi = 0x1.921fb544p+0;
static constexpr double kPio2Lo = 0x1.0b4611a626331p-34;
static_assert(kPio2Hi == 0x1921fb544p-32, "the 33-bit head of pi/2 as an integer times 2^-32");

// (-1)^k / (2k+1)!  and  (-1)^k / (2k)!, k = 1..8: each a quotient of exactly
// representable integers, rounded once by the compiler's constant folding.
#define VC_S(k, f) ((((k) & 1) ? -1.0 : 1.0) / (f))
static constexpr double kSin1 = VC_S(1, 6.0);
static constexpr double kSin2 = VC_S(2, 120.0);
static constexpr double kSin3 = VC_S(3, 5040.0);
static constexpr double kSin4 = VC_S(4, 362880.0);
static constexpr double kSin5 = VC_S(5, 39916800.0);
static constexpr double kSin6 = VC_S(6, 6227020800.0);
static constexpr double kSin7 = VC_S(7, 1307674368000.0);
static constexpr double kSin8 = VC_S(8, 355687428096000.0);
static constexpr double kCos1 = VC_S(1, 2.0);
static constexpr double kCos2 = VC_S(2, 24.0);
static constexpr double kCos3 = VC_S(3, 720.0);
static constexpr double kCos4 = VC_S(4, 40320.0);
static constexpr double kCos5 = VC_S(5, 3628800.0);
static constexpr double kCos6 = VC_S(6, 479001600.0);
static constexpr double kCos7 = VC_S(7, 87178291200.0);
static constexpr double kCos8 = VC_S(8, 20922789888000.0);
#undef VC_S

// sin(r) = r + (r*r^2) * S(r^2) and cos(r) = 1 + (1*r^2) * C(r^2), both as
// A + (m*r^2) * Horner(coefficients; r^2): the lanes of a warp pick their
// coefficient set by quadrant instead of branching, so a warp whose lanes sit
// in different quadrants still evaluates one polynomial.  (1*r^2 == r^2
// exactly, so the cosine is the same binary64 value as 1 + r^2*C(r^2).)
__device__ __forceinline__ double csin_poly(double r, long long k) {
  const int quad = (int)(k & 3);  // two's complement: the mathematical k mod 4
  const bool c = (quad & 1) != 0;
  const double r2 = __dmul_rn(r, r);
  double s = c ? kCos8 : kSin8;
  s = __dadd_rn(__dmul_rn(s, r2), c ? kCos7 : kSin7);
  s = __dadd_rn(__dmul_rn(s, r2), c ? kCos6 : kSin6);
  s = __dadd_rn(__dmul_rn(s, r2), c ? kCos5 : kSin5);
  s = __dadd_rn(__dmul_rn(s, r2), c ? kCos4 : kSin4);
  s = __dadd_rn(__dmul_rn(s, r2), c ? kCos3 : kSin3);
  s = __dadd_rn(__dmul_rn(s, r2), c ? kCos2 : kSin2);
  s = __dadd_rn(__dmul_rn(s, r2), c ? kCos1 : kSin1);
  const double a = c ? 1.0 : r;
  const double v = __dadd_rn(a, __dmul_rn(__dmul_rn(a, r2), s));
  return (quad & 2) ? -v : v;
}

// The reduction with every step on the binary64 pipe: the shortest dependency
// chain (used where few chains run per SM and latency binds).
__device__ __forceinline__ double csin_b64(double t) {
  const double kd = floor(__dadd_rn(__dmul_rn(t, kTwoOverPi), 0.5));
  const double r = __dsub_rn(__dsub_rn(t, __dmul_rn(kd, kPio2Hi)), __dmul_rn(kd, kPio2Lo));
  return csin_poly(r, __double2ll_rz(kd));
}

// The same values with the rounding and floor of u + 1/2 and the exact
// t - k*PIO2_HI on the integer pipes (vc_ieee.cuh): five binary64 operations
// and conversions fewer per sine, for kernels where many chains share the
// SMs' binary64 pipes; arguments outside the integer forms' range
// (|t| >= 2^8 pi/2) take csin_b64.
__device__ __forceinline__ double csin(double t) {
  constexpr uint64_t kPio2HiM = 0x1921fb544ull;  // kPio2Hi = kPio2HiM 2^-32
  const double u = __dmul_rn(t, kTwoOverPi);
  bool ok1 = false, ok2 = false;
  const int k = round_half_floor_int(ieee_bits(u), ok1);
  const uint64_t db = sub_kh_bits(ieee_bits(t), k, kPio2HiM, ok2);
  if (!ok1 || (k != 0 && !ok2)) return csin_b64(t);
  const double d = k == 0 ? t : ieee_double(db);
  const double r = __dsub_rn(d, __dmul_rn(ieee_double(small_int_bits(k)), kPio2Lo));
  return csin_poly(r, k);
}

// ---- PLCM, Eq. 5 ------------------------------------------------------------
// x in [0,1]; p in (0,1/2); q = RN(1/2 - p) (the same value the map computes
// each step).  Reflect above 1/2 (exact), then one correctly rounded division.
// Branch-free so a warp never executes both divisions.
__device__ __forceinline__ double plcm_step(double x, double p, double q) {
  const double xr = (x > 0.5) ? __dsub_rn(1.0, x) : x;
  const bool lo = xr < p;
  const double num = lo ? xr : __dsub_rn(xr, p);
  const double den = lo ? p : q;
  return __ddiv_rn(num, den);
}

// The same PLCM step evaluated on the integer pipes (vc_ieee.cuh): identical
// binary64 results; the rare operands outside the normal range (x = 0 or 1,
// x = p, subnormal quotients) take the hardware path above.
struct PlcmMap {
  double p, q;    // p and RN(1/2 - p)
  Divisor dp, dq;
};

__device__ __forceinline__ PlcmMap make_plcm(double p, double q) {
  PlcmMap m;
  m.p = p;
  m.q = q;
  m.dp = make_divisor(p);
  m.dq = make_divisor(q);
  return m;
}

__device__ __forceinline__ double plcm_step_int(double x, const PlcmMap& m) {
  const uint64_t xb = ieee_bits(x);
  const bool refl = xb > 0x3FE0000000000000ull;  // x > 1/2 (positive doubles order like their bits)
  bool ok1 = true, ok2 = true, ok3 = true;
  const double om = one_minus_int(x, ok1);
  const double xr = refl ? om : x;
  const bool lo = ieee_bits(xr) < ieee_bits(m.p);
  const double sb = sub_rn_int(xr, m.p, ok2);
  const double a = lo ? xr : sb;
  Divisor d;
  d.mb = lo ? m.dp.mb : m.dq.mb;
  d.inv = lo ? m.dp.inv : m.dq.inv;
  d.eb = lo ? m.dp.eb : m.dq.eb;
  double r = div_rn_int(a, d, ok3);
  if ((refl && !ok1) || (!lo && !ok2) || !ok3) r = plcm_step(x, m.p, m.q);
  return r;
}

// ---- the logistic map, a third map for the same strategy -------------------
// x' = (r x)(1 - x), left to right; r in [3.9, 4].
__device__ __forceinline__ double logistic_step(double x, double r) {
  return __dmul_rn(__dmul_rn(r, x), __dsub_rn(1.0, x));
}

// ---- 2DLASM, Eq. 6 ----------------------------------------------------------
// pm = RN(pi * mu).  x' = csin(((pm*(y+3))*x)*(1-x)); y' uses the new x'.
// SINE_B64 selects the all-binary64 reduction of the sine (same values).
template <bool SINE_B64 = false>
__device__ __forceinline__ void lasm_step(double& x, double& y, double pm) {
  const double tx = __dmul_rn(__dmul_rn(__dmul_rn(pm, __dadd_rn(y, 3.0)), x), __dsub_rn(1.0, x));
  const double xn = SINE_B64 ? csin_b64(tx) : csin(tx);
  const double ty = __dmul_rn(__dmul_rn(__dmul_rn(pm, __dadd_rn(xn, 3.0)), y), __dsub_rn(1.0, y));
  const double yn = SINE_B64 ? csin_b64(ty) : csin(ty);
  x = xn;
  y = yn;
}

// ---- Sec. 3: six mantissa bytes = low 48 bits of the pattern, LSB first -----
__device__ __forceinline__ uint64_t mant48(double v) {
  return (uint64_t)__double_as_longlong(v) & 0xFFFFFFFFFFFFull;
}

}  // namespace vc
