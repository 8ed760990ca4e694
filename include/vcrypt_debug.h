/*
 * vcrypt_debug.h -- diagnostic entry points of the CUDA library, used by the
 * tests to compare single stages with an independent CPU implementation.
 * Same conventions as vcrypt.h (device pointers, stream-ordered, status codes).
 */
#ifndef VCRYPT_DEBUG_H
#define VCRYPT_DEBUG_H

#include <stdint.h>

#include "vcrypt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* out[i] = the cipher's sine of t[i] (the reading of "sin" in Eq. 1 / Eq. 6:
 * Cody-Waite reduction by pi/2, Taylor polynomials by Horner), n doubles each;
 * variant 0 = every reduction step on the binary64 pipe, 1 = the rounding,
 * floor and t - k*PIO2_HI on the integer pipes (must give the same bits).
 * VC_ERR_ARG for n < 0, null pointers with n > 0, or another variant. */
int vc_dbg_csin(const double* d_t, double* d_out, int64_t n, int32_t variant, void* stream);

/* out[i] = one PLCM step F(x[i], p[i]) (Eq. 5); variant 0 = binary64 pipe,
 * 1 = integer-pipe evaluation (must give the same bits). */
int vc_dbg_plcm(const double* d_x, const double* d_p, double* d_out, int64_t n, int32_t variant, void* stream);

/* One 2DLASM step (Eq. 6): in = n triples (x, y, mu), out = n pairs (x', y'). */
int vc_dbg_lasm(const double* d_xymu, double* d_out, int64_t n, void* stream);

/* The keystream the next nframes frames of the stream would use, advancing the
 * stream exactly as encrypt_frames would: d_ks receives nframes*rounds*N bytes
 * laid out [frame][round][frame byte q] (the byte diffused into position q in
 * that round, Eq. 3), d_sc the frames' confusion seeds s_c (Alg. 1). */
int vc_dbg_keystream(vc_ctx* ctx, uint8_t* d_ks, int64_t* d_sc, int32_t nframes, void* stream);

/* The passes the next encrypt_frames / decrypt_frames call of nframes >= 1
 * frames on this context would run: plan[0 .. min(n, cap) - 1] receives their
 * frame counts in order, info4 = {n passes, 1 if the first pass takes frames
 * whose keystream the previous call generated ahead, frames of keystream the
 * call would generate ahead for the next one at its end (0: none), warps per
 * SM-holding keystream CTA (0: the keystream shares all SMs)}.  Reads the
 * context only.  Errors: VC_ERR_ARG. */
int vc_dbg_call_plan(const vc_ctx* ctx, int32_t nframes, int32_t* plan, int32_t cap, int32_t* info4);

/* Jobs of the batcher's last batch that ran in its long-chain lane
 * (VC_BOPT_SPLIT; 0: none), or -VC_ERR_ARG. */
int vc_dbg_batch_split(const vc_batcher* b);

/* Internal geometry, for tests: {rows per tile, tiles per frame, padded frame
 * stride, N, P, scratch frames allocated, frames per pass, round-kernel shared
 * memory bytes}. */
int vc_dbg_layout(const vc_ctx* ctx, int32_t* out8);

/* Measured denominators of the keystream roofline, timed with CUDA events on
 * the current device (synchronous; each call takes a few milliseconds and
 * allocates a small scratch buffer):
 *  vc_dbg_fp64_peak: binary64 fused multiply-adds per second over all SMs
 *    (independent chains; one FMA counted as one operation);
 *  vc_dbg_imad_peak: 32-bit integer multiply-adds per second over all SMs;
 *  vc_dbg_plcm_latency: clock64 cycles per PLCM step (Eq. 5, integer-pipe
 *    form) along one dependent chain of `iters` steps (rounded up to a multiple
 *    of 4, run four to a loop pass as the keystream kernel runs them) from x0
 *    with parameter p (x0 in (0, 1), p in (0, 1/2)).
 * Errors: VC_ERR_ARG, VC_ERR_OOM, VC_ERR_CUDA. */
int vc_dbg_fp64_peak(double* ops_per_s, void* stream);
int vc_dbg_imad_peak(double* ops_per_s, void* stream);
int vc_dbg_plcm_latency(double x0, double p, int32_t iters, double* cycles_per_step, void* stream);

/* Since the last read (then reset): host milliseconds a vc_server spent per
 * part of its ticks (ms6[0..3]: frame clocks, readiness and job building;
 * prefetch of starved streams; the submission; the completion event), the
 * summed device milliseconds from each drained tick's first enqueued work to
 * its completion (ms6[4]) over ms6[5] ticks, and the ticks (*ticks).
 * Errors: VC_ERR_ARG. */
int vc_dbg_server_stats(vc_server* s, double* ms6, int64_t* ticks);

/* Latency records of a vc_server, for splitting per-frame latency into the
 * wait before submission (frame clock, keystream readiness, tick cadence) and
 * the device time after it.  vc_dbg_server_record: enable != 0 starts keeping
 * a record per drained frame and per drained tick (0 stops and frees them).
 * vc_dbg_server_take: moves up to cap records into out, 4 doubles each, and
 * sets *n to their number: which = 0 frames (stream id, arrival, submission,
 * completion), which = 1 ticks (submission, device start, device end, frame
 * count); times in seconds on the server's clock (vc_server_tick's `now`;
 * device times by CUDA events against the creation event).
 * Errors: VC_ERR_ARG. */
int vc_dbg_server_record(vc_server* s, int32_t enable);
int vc_dbg_server_take(vc_server* s, int32_t which, int32_t cap, double* out, int32_t* n);

#ifdef __cplusplus
}
#endif
#endif /* VCRYPT_DEBUG_H */
