// Host-side check of the integer-pipe binary64 routines of the CUDA library
// (csrc/vc_ieee.cuh) against the host CPU's IEEE-754 arithmetic, which rounds
// every operation to nearest even.  Compiled by nvcc as host code and run by
// tests/test_ieee_emulation.py.  Prints "mismatches <n>" per routine.
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <random>

#include "vc_ieee.cuh"

static double from_bits(uint64_t b) { double v; std::memcpy(&v, &b, 8); return v; }
static uint64_t to_bits(double v) { uint64_t b; std::memcpy(&b, &v, 8); return b; }

int main(int argc, char** argv) {
  const long long n = argc > 1 ? atoll(argv[1]) : 10000000LL;
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  long long bad_div = 0, bad_sub = 0, bad_om = 0, fb_div = 0, fb_sub = 0, checked_div = 0, checked_sub = 0;
  for (long long i = 0; i < n; i++) {
    // divisor: PLCM-like p in (0, 1/2) or an arbitrary positive normal
    double b;
    switch (i & 3) {
      case 0: b = 0.01 + 0.48 * U(g); break;
      case 1: b = 0.5 - (0.01 + 0.48 * U(g)); break;
      case 2: b = from_bits((g() & ((1ull << 52) - 1)) | ((uint64_t)(900 + g() % 200) << 52)); break;
      default: b = from_bits((g() & ((1ull << 52) - 1)) | (1022ull << 52)); break;
    }
    double a;
    switch ((i >> 2) & 3) {
      case 0: a = U(g) * b; break;                       // x < p branch
      case 1: a = from_bits(g() & 0x3FEFFFFFFFFFFFFFull); break;  // any value below 1
      case 2: a = from_bits((g() & ((1ull << 52) - 1)) | ((uint64_t)(1 + g() % 1022) << 52)); break;
      default: a = b * (1.0 + 1e-12 * (U(g) - 0.5)); break;  // quotient near 1
    }
    if (a > 0) {
      const vc::Divisor d = vc::make_divisor(b);
      bool ok = false;
      const double q = vc::div_rn_int(a, d, ok);
      if (ok) {
        checked_div++;
        if (to_bits(q) != to_bits(a / b)) {
          if (bad_div < 5) printf("div a=%a b=%a got %a want %a\n", a, b, q, a / b);
          bad_div++;
        }
      } else {
        fb_div++;
      }
    }
    // subtraction a >= b > 0 with nearby exponents
    double x = from_bits(to_bits(0.5 * U(g) + 1e-300));
    double y;
    switch ((i >> 4) & 3) {
      case 0: y = U(g) * x; break;
      case 1: y = x * (1.0 - std::ldexp(U(g), -(int)(g() % 60))); break;
      case 2: y = std::ldexp(x, -(int)(g() % 70)) * (0.5 + 0.5 * U(g)); break;
      default: y = from_bits(to_bits(x) - (g() % 4)); break;
    }
    if (y > 0 && y <= x) {
      bool ok = false;
      const double s = vc::sub_rn_int(x, y, ok);
      if (ok) {
        checked_sub++;
        if (to_bits(s) != to_bits(x - y)) {
          if (bad_sub < 5) printf("sub a=%a b=%a got %a want %a\n", x, y, s, x - y);
          bad_sub++;
        }
      } else {
        fb_sub++;
      }
    }
    // 1 - x on (1/2, 1)
    double z = from_bits((g() & ((1ull << 52) - 1)) | (1022ull << 52));
    if (z > 0.5) {
      bool ok = false;
      const double o = vc::one_minus_int(z, ok);
      if (!ok || to_bits(o) != to_bits(1.0 - z)) bad_om++;
    }
  }
  // PLCM step in Q0.64 (derived parameter range p in [0.05, 0.45]) against the
  // map of Eq. 5 evaluated in the host's binary64 arithmetic
  long long bad_plcm = 0, fb_plcm = 0, checked_plcm = 0;
  for (long long i = 0; i < n; i++) {
    const double p = 0.05 + 0.4 * U(g);
    const double q = 0.5 - p;
    vc::PlcmFx F;
    if (!vc::make_plcm_fx(p, q, F)) { bad_plcm++; continue; }
    double x;
    switch (i & 7) {
      case 0: x = U(g); break;
      case 1: x = U(g) * 1e-3; break;
      case 2: x = 1.0 - U(g) * 1e-9; break;
      case 3: x = p * (1.0 + 1e-13 * (U(g) - 0.5)); break;
      case 4: x = std::ldexp(U(g), -(int)(g() % 1000)); break;
      case 5: x = 0.5 + 1e-12 * (U(g) - 0.5); break;
      case 6: x = (1.0 - p) * (1.0 + 1e-13 * (U(g) - 0.5)); break;
      case 7:
        if ((i & 8) && (i & 64)) {  // exact quotients: x / p or (x - p) / q a power of two
          const int k = 1 + (int)(g() % 6);
          x = (i & 16) ? std::ldexp(p, -k) : p + std::ldexp(q, -k);
          if (i & 32) x = 1.0 - x;
        } else if (i & 8) {  // x / p (or (x - p) / q) close to a rounding midpoint or a binade edge
          const double y = 0.5 + 0.5 * U(g);
          const double yh = y + std::ldexp(1.0, -54) * (1.0 + (double)(g() % 5) - 2.0);
          x = (i & 16) ? yh * p : p + yh * q;
          if (i & 32) x = 1.0 - x;
        } else {
          x = from_bits(g() & 0x3FEFFFFFFFFFFFFFull);
        }
        break;
      default: x = U(g); break;
    }
    double xr = x > 0.5 ? 1.0 - x : x;
    const double want = xr < p ? xr / p : (xr - p) / q;
    bool ok = false;
    const uint64_t got = vc::plcm_fx_step(to_bits(x), F, ok);
    if (!ok) { fb_plcm++; continue; }
    checked_plcm++;
    if (got != to_bits(want)) {
      if (bad_plcm < 5) printf("plcm x=%a p=%a got %a want %a\n", x, p, from_bits(got), want);
      bad_plcm++;
    }
  }
  // argument reduction of the cipher's sine: k = floor(RN(u + 1/2)) and
  // RN(t - k*HI) against the host's binary64 operations, and the binary64
  // value of a small integer
  const double HI = 0x1.921fb544p+0;
  const double TWO_OVER_PI = 0x1.45f306dc9c883p-1;
  long long bad_kr = 0, fb_kr = 0, checked_kr = 0, bad_skh = 0, fb_skh = 0, checked_skh = 0, bad_int = 0;
  for (long long i = 0; i < n; i++) {
    double u;
    switch (i & 7) {
      case 0: u = 600.0 * (U(g) - 0.5); break;
      case 1: u = 40.0 * (U(g) - 0.5); break;
      case 2: {  // within a few units in the last place of a half-integer
        const double m = (double)((long long)(g() % 521) - 260) + 0.5;
        u = from_bits(to_bits(m) + (g() % 7) - 3);
        break;
      }
      case 3: u = std::ldexp(U(g) - 0.5, -(int)(g() % 80)); break;
      case 4: u = from_bits(g()); break;  // any bit pattern (ok must exclude the unsupported ones)
      case 5: u = (double)((long long)(g() % 601) - 300) * 0.5; break;  // exact halves and integers
      case 6: u = 0.5 - std::ldexp(1.0, -(int)(50 + g() % 6)); break;  // just below 1/2
      default: u = -0.5 - std::ldexp(1.0, -(int)(50 + g() % 6)) * (double)(g() % 3); break;
    }
    bool ok = false;
    const int k = vc::round_half_floor_int(to_bits(u), ok);
    if (!ok) {
      fb_kr++;
    } else {
      checked_kr++;
      const double want = std::floor(u + 0.5);
      if ((double)k != want) {
        if (bad_kr < 5) printf("kround u=%a got %d want %a\n", u, k, want);
        bad_kr++;
      }
    }
    // t near k pi/2 (the sine's arguments), at a multiple of HI, or anywhere
    double t;
    switch ((i >> 3) & 3) {
      case 0: t = 1200.0 * (U(g) - 0.5); break;
      case 1: t = 50.0 * (U(g) - 0.5); break;
      case 2: {
        const double kk = (double)((long long)(g() % 513) - 256);
        t = from_bits(to_bits(kk * HI) + (g() % 9) - 4);
        break;
      }
      default: t = (double)((long long)(g() % 513) - 256) * HI; break;
    }
    const double kd = std::floor(t * TWO_OVER_PI + 0.5);
    const int kt = (int)kd;
    if (std::fabs(kd) <= 256.0) {
      bool ok2 = false;
      const uint64_t got = vc::sub_kh_bits(to_bits(t), kt, 0x1921fb544ull, ok2);
      if (!ok2) {
        fb_skh++;
      } else {
        checked_skh++;
        const double want = t - kd * HI;
        if (got != to_bits(want)) {
          if (bad_skh < 5) printf("t-kHI t=%a k=%d got %a want %a\n", t, kt, from_bits(got), want);
          bad_skh++;
        }
      }
    }
    const int ki = (int)(g() % (1u << 21)) - (1 << 20);
    if (vc::small_int_bits(ki) != to_bits((double)ki)) bad_int++;
  }
  for (int ki = -300; ki <= 300; ki++)
    if (vc::small_int_bits(ki) != to_bits((double)ki)) bad_int++;
  printf("kround checked %lld fallback %lld mismatches %lld\n", checked_kr, fb_kr, bad_kr);
  printf("t-kHI checked %lld fallback %lld mismatches %lld\n", checked_skh, fb_skh, bad_skh);
  printf("small_int mismatches %lld\n", bad_int);
  printf("plcm_fx checked %lld fallback %lld mismatches %lld\n", checked_plcm, fb_plcm, bad_plcm);
  printf("div checked %lld fallback %lld mismatches %lld\n", checked_div, fb_div, bad_div);
  printf("sub checked %lld fallback %lld mismatches %lld\n", checked_sub, fb_sub, bad_sub);
  printf("one_minus mismatches %lld\n", bad_om);
  return (bad_div || bad_sub || bad_om || bad_plcm || bad_kr || bad_skh || bad_int) ? 1 : 0;
}
