// vc_ieee.cuh -- IEEE-754 binary64 round-to-nearest-even subtraction and
// division evaluated on the integer pipes.
//
// GB300 executes binary64 at 2 lanes per clock per SM with ~63-cycle latency,
// while 32-bit integer multiply-adds run at 64 lanes per clock.  The PLCM
// (Eq. 5) needs one binary64 division per iteration by one of two constants
// of its chain (p or 1/2 - p).  These routines return exactly the correctly
// rounded binary64 result (the value __ddiv_rn / __dsub_rn return) from
// integer arithmetic:
//  * division by a constant divisor b = mb 2^e: a precomputed reciprocal
//    inv = floor(2^115 / mb) gives a quotient estimate within one unit
//    (Granlund & Montgomery, "Division by invariant integers using
//    multiplication", PLDI 1994), one correction step makes it exact, and the
//    remainder decides round-to-nearest-even; the PLCM step instead carries
//    the reciprocal to 128 bits, rounded up, so that the product alone
//    decides the rounding (no correction step);
//  * subtraction a - b, a >= b > 0: alignment with 10 guard bits and a sticky
//    bit, then rounding of the dropped bits (the classical guard/round/sticky
//    scheme of IEEE adders).
// Operands or results outside the normal range are reported through `ok`
// (false) and the caller falls back to the hardware operation, so the result
// is correctly rounded for every input.
#pragma once
#include <cstdint>
#include <cstring>

namespace vc {

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ uint64_t ieee_bits(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ double ieee_double(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ uint64_t ieee_mulhi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }
__device__ __forceinline__ int ieee_clz64(uint64_t v) { return __clzll((long long)v); }
// Leading zeros of v when its high word is non-zero, from the exponent of the
// high word converted to binary32 with truncation (exact: floor(log2)).  The
// conversion is several times faster than the integer leading-zero count on
// this GPU.
__device__ __forceinline__ int lz64_hi(uint64_t v) {
  return 158 - (int)(__float_as_uint(__uint2float_rz((uint32_t)(v >> 32))) >> 23);
}
// Number of significant bits of v (floor(log2 v) + 1) by the same conversion;
// v = 0 gives -126.
__device__ __forceinline__ int ieee_bitlen32(uint32_t v) {
  return (int)(__float_as_uint(__uint2float_rz(v)) >> 23) - 126;
}
#else
inline uint64_t ieee_bits(double v) {
  uint64_t b;
  std::memcpy(&b, &v, 8);
  return b;
}
inline double ieee_double(uint64_t b) {
  double v;
  std::memcpy(&v, &b, 8);
  return v;
}
inline uint64_t ieee_mulhi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
inline int ieee_clz64(uint64_t v) { return v ? __builtin_clzll(v) : 64; }
inline int lz64_hi(uint64_t v) { return __builtin_clz((uint32_t)(v >> 32)); }
inline int ieee_bitlen32(uint32_t v) { return v ? 32 - __builtin_clz(v) : -126; }
#endif

constexpr uint64_t kMant52 = (1ull << 52) - 1;

// A positive normal binary64 divisor: mantissa with the hidden bit, biased
// exponent, inv = floor(2^115 / mb) (in (2^62, 2^63]) and the 128-bit
// reciprocal rc_hi 2^64 + rc_lo = ceil(2^179 / mb) (in (2^126, 2^127]).
struct Divisor {
  uint64_t mb;
  uint64_t inv;
  uint64_t rc_hi, rc_lo;
  int eb;
};

// floor(2^115 / m) for m in [2^52, 2^53): restoring long division, 63
// quotient bits (used once per chain, off the hot loop).
__host__ __device__ inline uint64_t recip115(uint64_t m) {
  // 2^115 / m = 2^62 * (2^53 / m); start from the remainder of 2^53 / m.
  uint64_t q = 1;           // 2^53 / m >= 1 (m < 2^53), first quotient bit
  uint64_t r = (1ull << 53) - m;
  for (int i = 0; i < 62; i++) {
    r <<= 1;
    q <<= 1;
    if (r >= m) {
      r -= m;
      q |= 1;
    }
  }
  return q;
}

// ceil(2^179 / m) for m in [2^52, 2^53) as two words, from inv = floor(2^115 / m):
// 64 more quotient bits of the long division, rounded up if a remainder is left.
__host__ __device__ inline void recip179_ceil(uint64_t m, uint64_t inv, uint64_t& hi, uint64_t& lo) {
  uint64_t r = 0 - inv * m;  // 2^115 - inv m, exact: it lies in [0, m) and 2^115 is 0 mod 2^64
  uint64_t q = 0;
  for (int i = 0; i < 64; i++) {
    r <<= 1;
    q <<= 1;
    if (r >= m) {
      r -= m;
      q |= 1;
    }
  }
  hi = inv;
  lo = q;
  if (r != 0) {
    lo++;
    if (lo == 0) hi++;
  }
}

__host__ __device__ inline Divisor make_divisor(double b) {
  const uint64_t bb = ieee_bits(b);
  Divisor d;
  d.eb = (int)(bb >> 52);
  d.mb = (bb & kMant52) | (1ull << 52);
  d.inv = recip115(d.mb);
  recip179_ceil(d.mb, d.inv, d.rc_hi, d.rc_lo);
  return d;
}

// RN(a / b) for a > 0 normal and b = d (positive normal).  ok = false when a is
// zero/subnormal or the quotient is not a normal number.
__host__ __device__ __forceinline__ double div_rn_int(double a, const Divisor& d, bool& ok) {
  const uint64_t ab = ieee_bits(a);
  const int ea = (int)(ab >> 52);
  const uint64_t ma = (ab & kMant52) | (1ull << 52);
  const bool lt = ma < d.mb;
  const int s = lt ? 53 : 52;
  // q = floor(ma * inv / 2^(115 - s)), within one of floor(ma 2^s / mb)
  const uint64_t lo = ma * d.inv;
  const uint64_t hi = ieee_mulhi(ma, d.inv);
  const int sh = 115 - s;  // 62 or 63
  uint64_t q = (hi << (64 - sh)) | (lo >> sh);
  uint64_t rem = (ma << s) - q * d.mb;  // exact: the true value lies in [0, 2 mb)
  if (rem >= d.mb) {
    q++;
    rem -= d.mb;
  }
  const uint64_t twice = rem << 1;
  q += (twice > d.mb || (twice == d.mb && (q & 1))) ? 1 : 0;
  int e = ea - d.eb + 1023 - (lt ? 1 : 0);
  if (q == (1ull << 53)) {
    q >>= 1;
    e++;
  }
  ok = (ea >= 1) && (e >= 1) && (e <= 2046);
  return ieee_double(((uint64_t)(e & 0x7FF) << 52) | (q & kMant52));
}

// RN(a - b) for a >= b > 0, both normal.  ok = false when the result is
// zero/subnormal (a == b, or a tiny difference) or an operand is not normal.
__host__ __device__ __forceinline__ double sub_rn_int(double a, double b, bool& ok) {
  const uint64_t ab = ieee_bits(a), bb = ieee_bits(b);
  const int ea = (int)(ab >> 52), eb = (int)(bb >> 52);
  const uint64_t A = ((ab & kMant52) | (1ull << 52)) << 10;  // 63 bits
  const uint64_t Bf = ((bb & kMant52) | (1ull << 52)) << 10;
  const int shift = ea - eb;  // >= 0
  uint64_t B, sticky;
  if (shift >= 64) {
    B = 0;
    sticky = 1;
  } else if (shift == 0) {
    B = Bf;
    sticky = 0;
  } else {
    B = Bf >> shift;
    sticky = (Bf << (64 - shift)) != 0 ? 1 : 0;
  }
  // D = floor(true difference) in units of 2^(ea - 1085); sticky: a fraction remains
  const uint64_t D = A - B - sticky;
  const int L = 64 - ieee_clz64(D);  // bit length (0 if D == 0)
  const int k = L - 53;              // bits to drop (> 8 whenever sticky is set)
  uint64_t q;
  if (k > 0) {
    q = D >> k;
    const uint64_t R = D & ((1ull << k) - 1);
    const uint64_t half = 1ull << (k - 1);
    q += (R > half || (R == half && (sticky || (q & 1)))) ? 1 : 0;
  } else {
    q = D << (-k);  // exact (no sticky possible here)
  }
  int e = k + ea - 10;
  if (q == (1ull << 53)) {
    q >>= 1;
    e++;
  }
  ok = (ea >= 1) && (eb >= 1) && (ab >= bb) && (L > 0) && (e >= 1);
  return ieee_double(((uint64_t)(e & 0x7FF) << 52) | (q & kMant52));
}

// PLCM (Eq. 5) step on the integer pipes in Q0.64 fixed point, for a chain
// whose p and q = RN(1/2 - p) are both >= 2^-11 (true of every derived
// parameter, p in [0.05, 0.45]).  Every double in [2^-12, 1) is an exact Q0.64
// number, so the reflection 1 - x and the difference x - p are exact integer
// operations; RN(x - p) is the 53-bit rounding of that integer, and the
// quotient uses the reciprocal division above.  Operates on the bit pattern
// of x; returns the bit pattern of F(x) with ok = false for the few operands
// it does not cover (x = 0, x = 1, x = p, tiny quotients).
struct PlcmFx {
  uint64_t P;      // p 2^64
  Divisor dp, dq;  // p and q as divisors
};

__host__ __device__ inline bool make_plcm_fx(double p, double q, PlcmFx& F) {
  const uint64_t pb = ieee_bits(p), qb = ieee_bits(q);
  const int ep = (int)(pb >> 52), eq = (int)(qb >> 52);
  F.dp = make_divisor(p);
  F.dq = make_divisor(q);
  if (ep < 1012 || ep > 1021 || eq < 1012 || eq > 1021) {  // need 2^-11 <= p, q < 1/2
    F.P = 0;
    return false;
  }
  F.P = F.dp.mb << (ep - 1011);
  return true;
}

__host__ __device__ __forceinline__ uint64_t plcm_fx_step(uint64_t xb, const PlcmFx& F, bool& ok) {
  const int ex = (int)(xb >> 52);
  const uint64_t m = (xb & kMant52) | (1ull << 52);
  const int sx = ex - 1011;                 // x = m 2^(sx - 64) in Q0.64 when 0 <= sx <= 11
  const bool small = sx < 0;                // x < 2^-12 < p: always the x/p branch, operand x itself
  const uint64_t X = m << (sx & 15);
  const bool refl = xb > 0x3FE0000000000000ull;  // x > 1/2
  const uint64_t XR = refl ? (0ull - X) : X;      // 1 - x, exact
  const bool lo = small || XR < F.P;
  const uint64_t A = lo ? XR : XR - F.P;          // x (or 1 - x), or the exact x - p
  const bool wide = (A >> 32) != 0;               // operand >= 2^-32 (else the hardware path)
  const int lz = lz64_hi(wide ? A : (1ull << 32));
  const uint64_t An = A << (lz & 63);
  // RN to 53 significant bits: add just under half a unit plus the unit's
  // parity (ties to even); a carry out of bit 63 (rounding up to the next
  // binade, about 2^-42 per step) is left to the hardware path
  const uint64_t Ar = An + (0x3FFull + ((An >> 11) & 1));
  const bool carry = Ar < An;
  const uint64_t ma = small ? m : (Ar >> 11);
  const int ea = small ? ex : 1022 - lz;
  // RN(a / b), b = p on the x/p branch, q on the (x - p)/q branch.  With
  // t = ma 2^53 / mb and RC = ceil(2^179 / mb), v = ma RC / 2^126 = t + eps,
  // 0 <= eps < ma / 2^126 < 2^-73.  The fraction of t is a multiple of 1/mb
  // (> 2^-53) and never 1/2 (that would need 2^54 | mb), so floor(v) =
  // floor(t) and frac(v) >= 1/2 iff frac(t) > 1/2.  ma >= mb (t >= 2^53): the
  // result is (floor(t) + 1) >> 1 (a quotient of two 53-bit numbers is never
  // halfway); ma < mb: floor(t) rounded up iff frac(t) > 1/2.  A quotient
  // that rounds up to 2^53 (the next binade) is left to the hardware path.
  const uint64_t mb = lo ? F.dp.mb : F.dq.mb;
  const uint64_t rh = lo ? F.dp.rc_hi : F.dq.rc_hi;
  const uint64_t rl = lo ? F.dp.rc_lo : F.dq.rc_lo;
  const int eb = lo ? F.dp.eb : F.dq.eb;
  const bool big = ma >= mb;
  // ma RC = hi1 2^128 + (lo1 + hi2) 2^64 + (low word, not needed)
  const uint64_t lo1 = ma * rh, hi1 = ieee_mulhi(ma, rh);
  const uint64_t hi2 = ieee_mulhi(ma, rl);
  const uint64_t mid = lo1 + hi2;
  const uint64_t top = hi1 + (mid < lo1 ? 1 : 0);
  uint64_t q = (top << 2) | (mid >> 62);  // floor(v)
  q = big ? ((q >> 1) + (q & 1)) : (q + ((mid >> 61) & 1));
  const int e = ea - eb + (big ? 1023 : 1022);
  ok = (ex >= 1) && (ex <= 1022) && (small || (wide && !carry)) && (q < (1ull << 53)) && (e >= 1);
  return ((uint64_t)(e & 0x7FF) << 52) | (q & kMant52);
}

// 1 - x for x in (1/2, 1): exact; x = mx 2^-53 with mx in (2^52, 2^53).
__host__ __device__ __forceinline__ double one_minus_int(double x, bool& ok) {
  const uint64_t xb = ieee_bits(x);
  const int ex = (int)(xb >> 52);
  const uint64_t y = (1ull << 53) - ((xb & kMant52) | (1ull << 52));  // in (0, 2^52)
  const int L = 64 - ieee_clz64(y);
  const uint64_t m = y << (53 - L);
  const int e = 1022 - (53 - L);
  ok = (ex == 1022) && (y != 0);
  return ieee_double(((uint64_t)e << 52) | (m & kMant52));
}

// ---- argument reduction of the cipher's sine on the integer pipes ----------
// The sine reduces t by k pi/2 with k = floor(RN(RN(t 2/pi) + 1/2)) and
// r = RN(RN(t - k HI) - RN(k LO)), HI = pi/2 to 33 bits (Cody-Waite).  Two of
// those steps have exact integer forms: the rounding of u + 1/2 followed by
// the floor, and t - k HI (k HI is exact, and so is the difference formed in
// fixed point below).  Both return the values the binary64 operations return,
// with five binary64 operations and conversions fewer per sine (the binary64
// pipe is the scarce one when many chains share the SMs) but a longer
// dependency chain (25 to 35 integer instructions against four binary64
// operations).

// floor(RN(u + 1/2)) from the bits of the binary64 u.  ok = false when
// |u| >= 256 or u is not finite (the caller uses the binary64 operations).
__host__ __device__ __forceinline__ int round_half_floor_int(uint64_t ub, bool& ok) {
  const int eu = (int)((ub >> 52) & 0x7FF);
  ok = eu <= 1030;
  const bool neg = (ub >> 63) != 0;
  const uint64_t mu = (ub & kMant52) | (1ull << 52);
  const uint64_t U = mu << ((eu - 1021) & 15);  // |u| 2^54 when 1/4 <= |u| < 256 (below 2^62)
  const uint64_t h = 1ull << 53;                 // 1/2 in units of 2^-54
  const bool sneg = neg && U > h;                // u + 1/2 < 0
  const uint64_t A = neg ? (sneg ? U - h : h - U) : U + h;  // |u + 1/2| 2^54, exact
  // RN to 53 significant bits: d = dropped bits (0 when A < 2^53)
  int d = 32 + ieee_bitlen32((uint32_t)(A >> 32)) - 53;
  d = d < 0 ? 0 : d;
  const uint64_t half = (1ull << d) >> 1;
  const uint64_t inc = d ? half - 1 + ((A >> d) & 1) : 0;  // ties to even
  const uint64_t Ar = ((A + inc) >> d) << d;
  const int fl = sneg ? -(int)((Ar + ((1ull << 54) - 1)) >> 54) : (int)(Ar >> 54);
  // |u| < 1/4: u + 1/2 lies in (1/4, 3/4) and so does its rounding: floor 0
  return eu < 1021 ? 0 : fl;
}

// Bits of RN(t - k H) for H = hm 2^-32 (hm below 2^34), from the bits of the
// binary64 t: t and k H are both multiples of 2^-53 when |t| >= 1/2, so their
// difference is formed exactly as an integer in units of 2^-53 and rounded
// once to 53 significant bits.  ok = false unless 1/2 <= |t| < 512 and
// |k| <= 256 (the caller uses the binary64 operations).
__host__ __device__ __forceinline__ uint64_t sub_kh_bits(uint64_t tb, int k, uint64_t hm, bool& ok) {
  const int et = (int)((tb >> 52) & 0x7FF);
  ok = et >= 1022 && et <= 1031 && k >= -256 && k <= 256;
  const uint64_t T = ((tb & kMant52) | (1ull << 52)) << ((et - 1022) & 15);  // |t| 2^53, below 2^62
  const uint64_t ak = (uint64_t)(k < 0 ? -k : k) & 511;
  const uint64_t KH = (ak * hm) << 21;                                         // |k| H 2^53
  const uint64_t sT = (tb >> 63) ? 0ull - T : T;
  const uint64_t sK = k < 0 ? 0ull - KH : KH;
  const uint64_t D = sT - sK;  // two's complement of (t - k H) 2^53; |.| < 2^63 in range
  const bool dneg = (int64_t)D < 0;
  const uint64_t A = dneg ? 0ull - D : D;
  const uint32_t ahi = (uint32_t)(A >> 32);
  const int b = ahi ? 32 + ieee_bitlen32(ahi) : ieee_bitlen32((uint32_t)A);  // significant bits of A
  const int d = b > 53 ? b - 53 : 0;
  const uint64_t half = (1ull << d) >> 1;
  const uint64_t inc = d ? half - 1 + ((A >> d) & 1) : 0;  // ties to even
  uint64_t M = (A + inc) >> d;
  const bool carry = (M >> 53) != 0;  // rounded up to the next power of two
  M = carry ? (M >> 1) : M;
  M = b < 53 ? (A << ((53 - b) & 63)) : M;
  const uint64_t e = (uint64_t)(b + 969 + (carry ? 1 : 0));  // biased exponent of A 2^-53
  const uint64_t bits = ((uint64_t)dneg << 63) | (e << 52) | (M & kMant52);
  return A == 0 ? 0ull : bits;  // t = k H exactly: +0
}

// Bits of the binary64 value of the integer k, |k| < 2^24.
__host__ __device__ __forceinline__ uint64_t small_int_bits(int k) {
  const uint32_t a = (uint32_t)(k < 0 ? -k : k);
  const int b = ieee_bitlen32(a);
  const uint64_t m = ((uint64_t)a << ((53 - b) & 63)) & kMant52;
  const uint64_t bits = ((uint64_t)(k < 0) << 63) | ((uint64_t)(1022 + b) << 52) | m;
  return a == 0 ? 0ull : bits;
}

}  // namespace vc
