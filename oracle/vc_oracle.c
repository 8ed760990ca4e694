/*
 * vc_oracle.c -- plain, single-threaded CPU oracle of the chaotic video cipher
 * of "Real-time chaotic video encryption based on multithreaded parallel
 * confusion and diffusion" (Jiang, Yuan, Li, Lu; arXiv 2302.07411).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or constant table
 * with the CUDA path.
 *
 * Every step is written in the order the paper states it:
 *   Eq. 5      PLCM map                          -> plcm_step()
 *   Eq. 6      2DLASM map                        -> lasm_step()
 *   Sec. 7 iii a third map, the logistic map (parity unpinned by the paper:
 *              it names no other map; pinned by closed forms)
 *                                                 -> logistic_step()
 *   Sec. 3     PRBG byte construction (6 mantissa bytes per iterate, XOR of the
 *              two maps' byte streams)           -> prbg_*()
 *   Alg. 1     main thread: PRBG_m keyed by K, parameters P_m, per-frame s_c
 *                                                 -> orc_ctx_init(), next_sc()
 *   Eq. 1      confusion (discretised Chirikov)  -> orc_confuse()
 *   Eq. 2      inverse confusion                 -> orc_unconfuse()
 *   Eq. 3      diffusion with ciphertext feedback, seed s_d from the last pixel
 *              of subframe (i+1) mod n (Alg. 2)  -> orc_diffuse()
 *   Eq. 4      inverse diffusion                 -> orc_undiffuse()
 *   Eq. 3/4, the per-channel reading (one chain per colour channel; a variant
 *              kept beside the default byte chains) -> orc_diffuse_pc(),
 *                                                    orc_undiffuse_pc()
 *   Alg. 1/2   r rounds of confusion then diffusion per frame
 *                                                 -> orc_encrypt_frame()
 *
 * Floating point: IEEE-754 binary64, round-to-nearest-even, one rounding per
 * operation.  Build with -ffp-contract=off (no fused multiply-add) and without
 * -ffast-math.  The paper's "sin" is the deterministic csin() below (Cody-Waite
 * reduction + Taylor polynomials by Horner), so results do not depend on a libm.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#include "vc_oracle.h"

/* ------------------------------------------------------------------------ */
/* csin: the cipher's sine (reading of "sin" in Eq. 1 and Eq. 6).           */
/* ------------------------------------------------------------------------ */

/* Nearest doubles to pi, 2*pi and 2/pi; pi/2 split into a 33-bit head (so that
 * k*head is exact for |k| < 2^20) and the nearest double to the remainder. */
static const double ORC_PI = 0x1.921fb54442d18p+1;
static const double ORC_TWO_PI = 0x1.921fb54442d18p+2;
static const double ORC_TWO_OVER_PI = 0x1.45f306dc9c883p-1;
static const double ORC_PIO2_HI = 0x1.921fb544p+0;
static const double ORC_PIO2_LO = 0x1.0b4611a626331p-34;

#define ORC_SIN_TERMS 8 /* odd terms r^3 .. r^17  */
#define ORC_COS_TERMS 8 /* even terms r^2 .. r^16 */

static double sin_coef[ORC_SIN_TERMS + 1]; /* [k] = (-1)^k / (2k+1)!, k>=1 */
static double cos_coef[ORC_COS_TERMS + 1]; /* [k] = (-1)^k / (2k)!,   k>=1 */
static int coef_ready = 0;

static void init_coefs(void) {
  /* n! is exact in binary64 for n <= 22, so 1.0/n! is the correctly rounded
   * reciprocal of the factorial. */
  double fact = 1.0;
  int n;
  for (n = 1; n <= 2 * ORC_SIN_TERMS + 1; n++) {
    fact = fact * (double)n;
    if (n % 2 == 1 && n >= 3) {
      int k = (n - 1) / 2;
      double c = 1.0 / fact;
      sin_coef[k] = (k % 2) ? -c : c;
    }
    if (n % 2 == 0 && n / 2 <= ORC_COS_TERMS) {
      int k = n / 2;
      double c = 1.0 / fact;
      cos_coef[k] = (k % 2) ? -c : c;
    }
  }
  coef_ready = 1;
}

double orc_sin_coef(int k) { if (!coef_ready) init_coefs(); return (k >= 1 && k <= ORC_SIN_TERMS) ? sin_coef[k] : 0.0; }
double orc_cos_coef(int k) { if (!coef_ready) init_coefs(); return (k >= 1 && k <= ORC_COS_TERMS) ? cos_coef[k] : 0.0; }

void orc_constants(double* out5) {
  out5[0] = ORC_PI; out5[1] = ORC_TWO_PI; out5[2] = ORC_TWO_OVER_PI;
  out5[3] = ORC_PIO2_HI; out5[4] = ORC_PIO2_LO;
}

/* sin(r) on |r| <= pi/4:  r + (r*r^2) * (S1 + r^2*(S2 + ... r^2*S8)) */
static double sin_poly(double r) {
  double r2 = r * r;
  double s = sin_coef[ORC_SIN_TERMS];
  int k;
  for (k = ORC_SIN_TERMS - 1; k >= 1; k--) s = s * r2 + sin_coef[k];
  return r + (r * r2) * s;
}

/* cos(r) on |r| <= pi/4:  1 + r^2 * (C1 + r^2*(C2 + ... r^2*C8)) */
static double cos_poly(double r) {
  double r2 = r * r;
  double c = cos_coef[ORC_COS_TERMS];
  int k;
  for (k = ORC_COS_TERMS - 1; k >= 1; k--) c = c * r2 + cos_coef[k];
  return 1.0 + r2 * c;
}

double orc_csin(double t) {
  double kd, r;
  long long k;
  if (!coef_ready) init_coefs();
  kd = floor(t * ORC_TWO_OVER_PI + 0.5);  /* nearest multiple of pi/2 */
  r = (t - kd * ORC_PIO2_HI) - kd * ORC_PIO2_LO; /* Cody-Waite reduction */
  k = (long long)kd;
  switch (k & 3) { /* quadrant = k mod 4 (two's complement gives the math mod) */
    case 0: return sin_poly(r);
    case 1: return cos_poly(r);
    case 2: return -sin_poly(r);
    default: return -cos_poly(r);
  }
}

/* ------------------------------------------------------------------------ */
/* Chaotic maps (Sec. 3).                                                    */
/* ------------------------------------------------------------------------ */

/* Eq. 5, PLCM: x/p on [0,p); (x-p)/(1/2-p) on [p,1/2]; F(1-x) on (1/2,1]. */
double orc_plcm_step(double x, double p) {
  double half_minus_p = 0.5 - p;
  if (x > 0.5) x = 1.0 - x;
  if (x < p) return x / p;
  return (x - p) / half_minus_p;
}

/* Eq. 6, 2DLASM: x' = sin(pi*mu*(y+3)*x*(1-x)); y' = sin(pi*mu*(x'+3)*y*(1-y)),
 * products evaluated left to right. */
void orc_lasm_step(double* x, double* y, double mu) {
  double pm = ORC_PI * mu;
  double xn = orc_csin(((pm * (*y + 3.0)) * *x) * (1.0 - *x));
  double yn = orc_csin(((pm * (xn + 3.0)) * *y) * (1.0 - *y));
  *x = xn;
  *y = yn;
}

/* "6 bytes from the mantissa": the low 48 bits of the binary64 pattern,
 * least significant byte first. */
void orc_mantissa_bytes(double v, uint8_t out[6]) {
  uint64_t bits;
  int k;
  memcpy(&bits, &v, 8);
  for (k = 0; k < 6; k++) out[k] = (uint8_t)((bits >> (8 * k)) & 0xffu);
}

/* A third map for the same strategy (Sec. 7, advantage iii: the strategy works
 * with other chaotic maps): the logistic map x' = r x (1 - x), r in [3.9, 4],
 * evaluated left to right, (r * x) * (1 - x).  Its PRBG is built like the
 * PLCM's: a pair of maps, 6 mantissa bytes per iterate, XORed. */
double orc_logistic_step(double x, double r) { return (r * x) * (1.0 - x); }

/* ------------------------------------------------------------------------ */
/* PRBGs (Sec. 3): continuous byte streams.                                  */
/* ------------------------------------------------------------------------ */

static void prbg_refill(orc_prbg* g) {
  uint8_t a[6], b[6];
  int k;
  if (g->kind == ORC_PRBG_PLCM_PAIR) {
    /* iterate both PLCMs, XOR their 6-byte groups */
    g->s[0] = orc_plcm_step(g->s[0], g->s[1]);
    g->s[2] = orc_plcm_step(g->s[2], g->s[3]);
    orc_mantissa_bytes(g->s[0], a);
    orc_mantissa_bytes(g->s[2], b);
    for (k = 0; k < 6; k++) g->buf[k] = a[k] ^ b[k];
    g->len = 6;
  } else if (g->kind == ORC_PRBG_LOGI_PAIR) {
    /* iterate both logistic maps, XOR their 6-byte groups */
    g->s[0] = orc_logistic_step(g->s[0], g->s[1]);
    g->s[2] = orc_logistic_step(g->s[2], g->s[3]);
    orc_mantissa_bytes(g->s[0], a);
    orc_mantissa_bytes(g->s[2], b);
    for (k = 0; k < 6; k++) g->buf[k] = a[k] ^ b[k];
    g->len = 6;
  } else if (g->kind == ORC_PRBG_LASM_PAIR) {
    /* iterate both 2DLASMs; emit x-groups XORed, then y-groups XORed */
    orc_lasm_step(&g->s[0], &g->s[1], g->s[2]);
    orc_lasm_step(&g->s[3], &g->s[4], g->s[5]);
    orc_mantissa_bytes(g->s[0], a);
    orc_mantissa_bytes(g->s[3], b);
    for (k = 0; k < 6; k++) g->buf[k] = a[k] ^ b[k];
    orc_mantissa_bytes(g->s[1], a);
    orc_mantissa_bytes(g->s[4], b);
    for (k = 0; k < 6; k++) g->buf[6 + k] = a[k] ^ b[k];
    g->len = 12;
  } else { /* ORC_PRBG_LASM_SINGLE: main PRBG of the 2DLASM cryptosystem */
    orc_lasm_step(&g->s[0], &g->s[1], g->s[2]);
    orc_mantissa_bytes(g->s[0], a);
    orc_mantissa_bytes(g->s[1], b);
    for (k = 0; k < 6; k++) { g->buf[k] = a[k]; g->buf[6 + k] = b[k]; }
    g->len = 12;
  }
  g->pos = 0;
}

void orc_prbg_init(orc_prbg* g, int kind, const double* params) {
  int k;
  memset(g, 0, sizeof(*g));
  g->kind = kind;
  for (k = 0; k < 6; k++) g->s[k] = params[k];
  g->len = 0; /* no iterate yet: the first output byte comes from x_1 */
  g->pos = 0;
}

void orc_prbg_bytes(orc_prbg* g, uint8_t* out, uint64_t nbytes) {
  uint64_t i;
  for (i = 0; i < nbytes; i++) {
    if (g->pos >= g->len) prbg_refill(g);
    out[i] = g->buf[g->pos++];
  }
}

/* One 6-byte group of PRBG_m as the 48-bit integer U (LSB first) and
 * u = (U + 1/2) * 2^-48 in (0,1) -- exact in binary64. */
static uint64_t next_group(orc_prbg* g) {
  uint8_t b[6];
  uint64_t U = 0;
  int k;
  orc_prbg_bytes(g, b, 6);
  for (k = 0; k < 6; k++) U |= (uint64_t)b[k] << (8 * k);
  return U;
}
static double group_to_unit(uint64_t U) { return (double)(2 * U + 1) * 0x1p-49; }

/* ------------------------------------------------------------------------ */
/* Cipher context (Alg. 1 main thread + Alg. 2 assistant threads, serial).   */
/* ------------------------------------------------------------------------ */

static int64_t pi_at(const orc_ctx* c, int64_t i) { /* first pixel of subframe i */
  return (i * c->P) / c->n;
}

int orc_key_valid(int kind, const double* k) {
  int i;
  for (i = 0; i < 4; i++) if (k[i] != k[i]) return 0; /* NaN */
  if (kind == ORC_PLCM) {
    /* Eq. 5: x0 in [0,1] (0 and 1 are absorbing, so rejected), p in (0,1/2) */
    return k[0] > 0.0 && k[0] < 1.0 && k[1] > 0.0 && k[1] < 0.5 &&
           k[2] > 0.0 && k[2] < 1.0 && k[3] > 0.0 && k[3] < 0.5;
  }
  if (kind == ORC_2DLASM) {
    /* Eq. 6: x0, y0 in (0,1); mu in [.37,.38] u [.4,.42] u [.44,.93] u {1} */
    double mu = k[1];
    int mu_ok = (mu >= 0.37 && mu <= 0.38) || (mu >= 0.4 && mu <= 0.42) ||
                (mu >= 0.44 && mu <= 0.93) || mu == 1.0;
    return k[0] > 0.0 && k[0] < 1.0 && k[2] > 0.0 && k[2] < 1.0 && mu_ok;
  }
  if (kind == ORC_LOGISTIC) {
    /* x0 in (0,1) (0 and 1 are absorbing); r in [3.9, 4] */
    return k[0] > 0.0 && k[0] < 1.0 && k[1] >= 3.9 && k[1] <= 4.0 &&
           k[2] > 0.0 && k[2] < 1.0 && k[3] >= 3.9 && k[3] <= 4.0;
  }
  return 0;
}

int orc_layout_valid(int H, int W, int C, int n, int rounds) {
  int64_t P;
  if (H < 1 || W < 1 || n < 1 || rounds < 1) return 0;
  if (!(C == 1 || C == 3 || C == 4)) return 0;
  P = (int64_t)H * W;
  if (n > P) return 0;
  /* every subframe must hold at least 2 bytes (decryption seed order) */
  if ((int64_t)C * (P / n) < 2) return 0;
  return 1;
}

size_t orc_ctx_size(int n) { return sizeof(orc_ctx) + (size_t)n * sizeof(orc_prbg); }

int orc_ctx_init(orc_ctx* c, int kind, const double* key, int H, int W, int C, int n, int rounds) {
  double mparams[6] = {0, 0, 0, 0, 0, 0};
  int i;
  if (!orc_key_valid(kind, key)) return 1;
  if (!orc_layout_valid(H, W, C, n, rounds)) return 2;
  c->kind = kind; c->H = H; c->W = W; c->C = C; c->n = n; c->rounds = rounds; c->chains = 0;
  c->P = (int64_t)H * W; c->N = c->P * C; c->frame = 0;
  if (kind == ORC_PLCM) {
    /* K = (x0^1, p^1, x0^2, p^2): PRBG_m is a PLCM pair */
    mparams[0] = key[0]; mparams[1] = key[1]; mparams[2] = key[2]; mparams[3] = key[3];
    orc_prbg_init(&c->main, ORC_PRBG_PLCM_PAIR, mparams);
  } else if (kind == ORC_LOGISTIC) {
    /* K = (x0^1, r^1, x0^2, r^2): PRBG_m is a logistic pair */
    mparams[0] = key[0]; mparams[1] = key[1]; mparams[2] = key[2]; mparams[3] = key[3];
    orc_prbg_init(&c->main, ORC_PRBG_LOGI_PAIR, mparams);
  } else {
    /* K = (x0, mu, y0): PRBG_m is a single 2DLASM, emitting x then y */
    mparams[0] = key[0]; mparams[1] = key[2]; mparams[2] = key[1];
    orc_prbg_init(&c->main, ORC_PRBG_LASM_SINGLE, mparams);
  }
  /* Alg. 1: iterate PRBG_m and convert the results into P_m, subframe by subframe */
  for (i = 0; i < n; i++) {
    double prm[6] = {0, 0, 0, 0, 0, 0};
    if (kind == ORC_PLCM) {
      double u1 = group_to_unit(next_group(&c->main));
      double u2 = group_to_unit(next_group(&c->main));
      double u3 = group_to_unit(next_group(&c->main));
      double u4 = group_to_unit(next_group(&c->main));
      prm[0] = u1; prm[1] = 0.05 + 0.4 * u2;
      prm[2] = u3; prm[3] = 0.05 + 0.4 * u4;
      orc_prbg_init(&c->sub[i], ORC_PRBG_PLCM_PAIR, prm);
    } else if (kind == ORC_LOGISTIC) {
      /* as the PLCM's: x0 = u, r = 3.9 + 0.1 u, each from its own group */
      double u1 = group_to_unit(next_group(&c->main));
      double u2 = group_to_unit(next_group(&c->main));
      double u3 = group_to_unit(next_group(&c->main));
      double u4 = group_to_unit(next_group(&c->main));
      prm[0] = u1; prm[1] = 3.9 + 0.1 * u2;
      prm[2] = u3; prm[3] = 3.9 + 0.1 * u4;
      orc_prbg_init(&c->sub[i], ORC_PRBG_LOGI_PAIR, prm);
    } else {
      double u1 = group_to_unit(next_group(&c->main));
      double u2 = group_to_unit(next_group(&c->main));
      double u3 = group_to_unit(next_group(&c->main));
      double u4 = group_to_unit(next_group(&c->main));
      double u5 = group_to_unit(next_group(&c->main));
      double u6 = group_to_unit(next_group(&c->main));
      /* (x0, y0, mu) per instance; state layout (x, y, mu) */
      prm[0] = u1; prm[1] = u2; prm[2] = 0.44 + 0.49 * u3;
      prm[3] = u4; prm[4] = u5; prm[5] = 0.44 + 0.49 * u6;
      orc_prbg_init(&c->sub[i], ORC_PRBG_LASM_PAIR, prm);
    }
  }
  return 0;
}

void orc_sub_params(const orc_ctx* c, int i, double* out6) {
  /* state of PRBG_a^i; equals its parameters before the first frame */
  memcpy(out6, c->sub[i].s, 6 * sizeof(double));
}

/* Test hook: restart PRBG_a^i of Alg. 2 from the given map parameters (its
 * next output byte comes from x_1 of the new orbit).  Lets a test put every
 * subframe on an orbit it can compute exactly by other means (the PLCM at
 * p = 1/4 on dyadic x0), so a whole frame follows from closed forms. */
void orc_set_sub_params(orc_ctx* c, int i, const double* params6) {
  orc_prbg_init(&c->sub[i], c->sub[i].kind, params6);
}

/* Alg. 1: one confusion seed per frame, a positive integer */
int64_t orc_next_sc(orc_ctx* c) { return 1 + (int64_t)(next_group(&c->main) % 65536u); }

/* Confusion table of Eq. 1: k(alpha) = floor(s_c * sin(2*pi*alpha/H)). */
void orc_ktable(int H, int64_t sc, int64_t* k) {
  int a;
  for (a = 0; a < H; a++) {
    double t = (ORC_TWO_PI * (double)a) / (double)H;
    k[a] = (int64_t)floor((double)sc * orc_csin(t));
  }
}

static int64_t mod_pos(int64_t v, int64_t m) { int64_t r = v % m; return r < 0 ? r + m : r; }

/* Eq. 1 over the whole frame: Y[alpha, beta] = X[a, o],
 * alpha = (a + o) mod H, beta = (o + k(alpha)) mod W (a = row, o = column). */
void orc_confuse(int H, int W, int C, const int64_t* k, const uint8_t* X, uint8_t* Y) {
  int a, o, ch;
  for (a = 0; a < H; a++)
    for (o = 0; o < W; o++) {
      int64_t alpha = mod_pos((int64_t)a + o, H);
      int64_t beta = mod_pos((int64_t)o + k[alpha], W);
      for (ch = 0; ch < C; ch++)
        Y[(alpha * W + beta) * C + ch] = X[((int64_t)a * W + o) * C + ch];
    }
}

/* Eq. 2: a = (alpha - beta + k(alpha)) mod H, o = (beta - k(alpha)) mod W. */
void orc_unconfuse(int H, int W, int C, const int64_t* k, const uint8_t* Y, uint8_t* X) {
  int alpha, beta, ch;
  for (alpha = 0; alpha < H; alpha++)
    for (beta = 0; beta < W; beta++) {
      int64_t o = mod_pos((int64_t)beta - k[alpha], W);
      int64_t a = mod_pos((int64_t)alpha - o, H);
      for (ch = 0; ch < C; ch++)
        X[(a * W + o) * C + ch] = Y[((int64_t)alpha * W + beta) * C + ch];
    }
}

/* Eq. 3 per subframe (Alg. 2): ks[i] holds subframe i's bytes for this round.
 * The first byte of subframe i is chained to s_d = the last byte of subframe
 * (i+1) mod n of the confused (pre-diffusion) frame Y. */
void orc_diffuse(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Y, uint8_t* Xo) {
  int64_t P = (int64_t)H * W;
  int i;
  for (i = 0; i < n; i++) {
    int64_t start = C * ((i * P) / n), end = C * (((i + 1) * P) / n);
    int64_t nxt = (i + 1) % n;
    int64_t seed_pos = C * (((nxt + 1) * P) / n) - 1;
    uint8_t sd = Y[seed_pos];
    int64_t q;
    for (q = start; q < end; q++) {
      uint8_t b = ks[i][q - start];
      uint8_t prev = (q == start) ? sd : Xo[q - 1];
      Xo[q] = (uint8_t)(b ^ (uint8_t)(Y[q] + b) ^ prev);
    }
  }
}

/* Eq. 4: F_p = (b xor F_c xor F_c[prev]) - b.  All non-first bytes first, then
 * each subframe's first byte with the seed recovered from subframe (i+1) mod n. */
void orc_undiffuse(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Xc, uint8_t* Y) {
  int64_t P = (int64_t)H * W;
  int i;
  for (i = 0; i < n; i++) {
    int64_t start = C * ((i * P) / n), end = C * (((i + 1) * P) / n);
    int64_t q;
    for (q = start + 1; q < end; q++) {
      uint8_t b = ks[i][q - start];
      Y[q] = (uint8_t)((uint8_t)(b ^ Xc[q] ^ Xc[q - 1]) - b);
    }
  }
  for (i = 0; i < n; i++) {
    int64_t start = C * ((i * P) / n);
    int64_t nxt = (i + 1) % n;
    int64_t seed_pos = C * (((nxt + 1) * P) / n) - 1;
    uint8_t b = ks[i][0];
    Y[start] = (uint8_t)((uint8_t)(b ^ Xc[start] ^ Y[seed_pos]) - b);
  }
}

/* Eq. 3 with one chain per channel (the alternative to the byte-chain
 * reading): byte ch of pixel p of subframe i follows byte ch of pixel p - 1;
 * the first pixel's byte ch follows byte ch of the last pixel of subframe
 * (i+1) mod n of the confused frame Y.  Keystream bytes as in orc_diffuse. */
void orc_diffuse_pc(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Y, uint8_t* Xo) {
  int64_t P = (int64_t)H * W;
  int i;
  for (i = 0; i < n; i++) {
    int64_t start = C * ((i * P) / n), end = C * (((i + 1) * P) / n);
    int64_t nxt = (i + 1) % n;
    int64_t seed_pixel = C * (((nxt + 1) * P) / n) - C; /* first byte of the last pixel of subframe nxt */
    int64_t q;
    for (q = start; q < end; q++) {
      int64_t ch = (q - start) % C;
      uint8_t b = ks[i][q - start];
      uint8_t prev = (q < start + C) ? Y[seed_pixel + ch] : Xo[q - C];
      Xo[q] = (uint8_t)(b ^ (uint8_t)(Y[q] + b) ^ prev);
    }
  }
}

/* Eq. 4 per channel: every pixel but the first from the ciphertext alone, then
 * each subframe's first pixel with the seed pixel recovered from subframe
 * (i+1) mod n (which must hold at least 2 pixels). */
void orc_undiffuse_pc(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Xc, uint8_t* Y) {
  int64_t P = (int64_t)H * W;
  int i;
  for (i = 0; i < n; i++) {
    int64_t start = C * ((i * P) / n), end = C * (((i + 1) * P) / n);
    int64_t q;
    for (q = start + C; q < end; q++) {
      uint8_t b = ks[i][q - start];
      Y[q] = (uint8_t)((uint8_t)(b ^ Xc[q] ^ Xc[q - C]) - b);
    }
  }
  for (i = 0; i < n; i++) {
    int64_t start = C * ((i * P) / n);
    int64_t nxt = (i + 1) % n;
    int64_t seed_pixel = C * (((nxt + 1) * P) / n) - C;
    int ch;
    for (ch = 0; ch < C; ch++) {
      uint8_t b = ks[i][ch];
      Y[start + ch] = (uint8_t)((uint8_t)(b ^ Xc[start + ch] ^ Y[seed_pixel + ch]) - b);
    }
  }
}

/* Select the diffusion chains of a context: 0 = bytes (R4, the default),
 * 1 = per channel, which needs every subframe to hold at least 2 pixels. */
int orc_ctx_set_chains(orc_ctx* c, int chains) {
  if (chains != 0 && chains != 1) return 1;
  if (chains == 1 && c->P / c->n < 2) return 2;
  c->chains = chains;
  return 0;
}

/* Per frame: s_c from PRBG_m, then r*S_i fresh bytes from each PRBG_a^i. */
static int frame_schedule(orc_ctx* c, int64_t* sc_out, int64_t* k, uint8_t** ks_all) {
  int i;
  int64_t sc = orc_next_sc(c);
  if (sc_out) *sc_out = sc;
  orc_ktable(c->H, sc, k);
  for (i = 0; i < c->n; i++) {
    int64_t Si = c->C * (pi_at(c, i + 1) - pi_at(c, i));
    ks_all[i] = (uint8_t*)malloc((size_t)(Si * c->rounds));
    if (!ks_all[i]) return 1;
    orc_prbg_bytes(&c->sub[i], ks_all[i], (uint64_t)(Si * c->rounds));
  }
  return 0;
}

static void free_ks(int n, uint8_t** ks_all) {
  int i;
  for (i = 0; i < n; i++) free(ks_all[i]);
}

int orc_encrypt_frame(orc_ctx* c, const uint8_t* in, uint8_t* out, int64_t* sc_out) {
  int64_t* k = (int64_t*)malloc(sizeof(int64_t) * c->H);
  uint8_t** ks_all = (uint8_t**)calloc((size_t)c->n, sizeof(uint8_t*));
  const uint8_t** ksr = (const uint8_t**)malloc(sizeof(uint8_t*) * (size_t)c->n);
  uint8_t* Y = (uint8_t*)malloc((size_t)c->N);
  int j, i, rc = 0;
  if (!k || !ks_all || !ksr || !Y) { rc = 3; goto done; }
  if (frame_schedule(c, sc_out, k, ks_all)) { rc = 3; goto done; }
  memmove(out, in, (size_t)c->N); /* F_c = F_p */
  for (j = 0; j < c->rounds; j++) {
    for (i = 0; i < c->n; i++) {
      int64_t Si = c->C * (pi_at(c, i + 1) - pi_at(c, i));
      ksr[i] = ks_all[i] + j * Si;
    }
    orc_confuse(c->H, c->W, c->C, k, out, Y);
    if (c->chains == 1)
      orc_diffuse_pc(c->H, c->W, c->C, c->n, ksr, Y, out);
    else
      orc_diffuse(c->H, c->W, c->C, c->n, ksr, Y, out);
  }
  c->frame++;
done:
  if (ks_all) free_ks(c->n, ks_all);
  free(k); free(ks_all); free(ksr); free(Y);
  return rc;
}

int orc_decrypt_frame(orc_ctx* c, const uint8_t* in, uint8_t* out, int64_t* sc_out) {
  int64_t* k = (int64_t*)malloc(sizeof(int64_t) * c->H);
  uint8_t** ks_all = (uint8_t**)calloc((size_t)c->n, sizeof(uint8_t*));
  const uint8_t** ksr = (const uint8_t**)malloc(sizeof(uint8_t*) * (size_t)c->n);
  uint8_t* Y = (uint8_t*)malloc((size_t)c->N);
  int j, i, rc = 0;
  if (!k || !ks_all || !ksr || !Y) { rc = 3; goto done; }
  if (frame_schedule(c, sc_out, k, ks_all)) { rc = 3; goto done; }
  memmove(out, in, (size_t)c->N);
  for (j = c->rounds - 1; j >= 0; j--) {
    for (i = 0; i < c->n; i++) {
      int64_t Si = c->C * (pi_at(c, i + 1) - pi_at(c, i));
      ksr[i] = ks_all[i] + j * Si;
    }
    if (c->chains == 1)
      orc_undiffuse_pc(c->H, c->W, c->C, c->n, ksr, out, Y);
    else
      orc_undiffuse(c->H, c->W, c->C, c->n, ksr, out, Y);
    orc_unconfuse(c->H, c->W, c->C, k, Y, out);
  }
  c->frame++;
done:
  if (ks_all) free_ks(c->n, ks_all);
  free(k); free(ks_all); free(ksr); free(Y);
  return rc;
}

/* The keystream of one frame for every subframe, concatenated in subframe
 * order (r*S_i bytes each), and the frame's s_c; advances the state exactly
 * like encrypt/decrypt of one frame. */
int orc_frame_keystream(orc_ctx* c, uint8_t* out, int64_t* sc_out) {
  int i;
  int64_t off = 0;
  int64_t sc = orc_next_sc(c);
  if (sc_out) *sc_out = sc;
  for (i = 0; i < c->n; i++) {
    int64_t Si = c->C * (pi_at(c, i + 1) - pi_at(c, i));
    orc_prbg_bytes(&c->sub[i], out + off, (uint64_t)(Si * c->rounds));
    off += Si * c->rounds;
  }
  c->frame++;
  return 0;
}

/* Checkpoint: the context holds no pointers, so its bytes are its state. */
void orc_save_state(const orc_ctx* c, void* buf) { memcpy(buf, c, orc_ctx_size(c->n)); }
void orc_load_state(orc_ctx* c, const void* buf) {
  const orc_ctx* s = (const orc_ctx*)buf;
  memcpy(c, buf, orc_ctx_size(s->n));
}
