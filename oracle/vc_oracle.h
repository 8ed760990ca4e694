/*
 * vc_oracle.h -- interface of the CPU oracle (test infrastructure only; see
 * vc_oracle.c).  Independent of the CUDA library's header.
 */
#ifndef VC_ORACLE_H
#define VC_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PLCM = 0, ORC_2DLASM = 1, ORC_LOGISTIC = 2 };
enum { ORC_PRBG_PLCM_PAIR = 0, ORC_PRBG_LASM_PAIR = 1, ORC_PRBG_LASM_SINGLE = 2, ORC_PRBG_LOGI_PAIR = 3 };

/* A PRBG: map state s[] plus the not yet consumed bytes of its last iterate.
 *  PLCM pair:     s = {x1, p1, x2, p2}
 *  2DLASM pair:   s = {x1, y1, mu1, x2, y2, mu2}
 *  2DLASM single: s = {x, y, mu}
 *  logistic pair: s = {x1, r1, x2, r2} */
typedef struct {
  int32_t kind;
  int32_t pos, len;
  uint8_t buf[12];
  double s[6];
} orc_prbg;

typedef struct {
  int32_t kind, H, W, C, n, rounds;
  int32_t chains; /* diffusion chains: 0 = one per subframe over its bytes (R4), 1 = one per channel */
  int64_t P, N, frame;
  orc_prbg main;  /* PRBG_m of Alg. 1 */
  orc_prbg sub[]; /* PRBG_a^i of Alg. 2, i = 0..n-1 */
} orc_ctx;

double orc_csin(double t);
double orc_sin_coef(int k);
double orc_cos_coef(int k);
void orc_constants(double* out5);
double orc_plcm_step(double x, double p);
void orc_lasm_step(double* x, double* y, double mu);
double orc_logistic_step(double x, double r);
void orc_mantissa_bytes(double v, uint8_t out[6]);

void orc_prbg_init(orc_prbg* g, int kind, const double* params);
void orc_prbg_bytes(orc_prbg* g, uint8_t* out, uint64_t nbytes);

int orc_key_valid(int kind, const double* key);
int orc_layout_valid(int H, int W, int C, int n, int rounds);
size_t orc_ctx_size(int n);
int orc_ctx_init(orc_ctx* c, int kind, const double* key, int H, int W, int C, int n, int rounds);
void orc_sub_params(const orc_ctx* c, int i, double* out6);
void orc_set_sub_params(orc_ctx* c, int i, const double* params6);
int64_t orc_next_sc(orc_ctx* c);
void orc_ktable(int H, int64_t sc, int64_t* k);
void orc_confuse(int H, int W, int C, const int64_t* k, const uint8_t* X, uint8_t* Y);
void orc_unconfuse(int H, int W, int C, const int64_t* k, const uint8_t* Y, uint8_t* X);
void orc_diffuse(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Y, uint8_t* Xo);
void orc_undiffuse(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Xc, uint8_t* Y);
void orc_diffuse_pc(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Y, uint8_t* Xo);
void orc_undiffuse_pc(int H, int W, int C, int n, const uint8_t* const* ks, const uint8_t* Xc, uint8_t* Y);
int orc_ctx_set_chains(orc_ctx* c, int chains);
int orc_encrypt_frame(orc_ctx* c, const uint8_t* in, uint8_t* out, int64_t* sc_out);
int orc_decrypt_frame(orc_ctx* c, const uint8_t* in, uint8_t* out, int64_t* sc_out);
int orc_frame_keystream(orc_ctx* c, uint8_t* out, int64_t* sc_out);
void orc_save_state(const orc_ctx* c, void* buf);
void orc_load_state(orc_ctx* c, const void* buf);

#ifdef __cplusplus
}
#endif
#endif
