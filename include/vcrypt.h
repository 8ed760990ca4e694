/*
 * vcrypt.h -- C ABI of the GB300 (sm_103a) implementation of the chaotic video
 * cipher of "Real-time chaotic video encryption based on multithreaded
 * parallel confusion and diffusion" (arXiv 2302.07411).
 *
 * The cipher (Sec. 2, Alg. 1, Alg. 2): a key K seeds a main chaotic PRBG_m
 * whose output gives every subframe i its own PRBG_a^i (two PLCMs, Eq. 5, or
 * two 2DLASMs, Eq. 6; Sec. 3) and gives every frame a confusion seed s_c.  Each
 * frame then goes through r rounds of whole-frame confusion (Eq. 1) followed by
 * per-subframe diffusion with ciphertext feedback (Eq. 3); decryption applies
 * Eq. 4 and Eq. 2 in reverse round order.
 *
 * Conventions for every entry point:
 *  - Frames are H x W x C uint8 in HWC order (row-major, channel fastest),
 *    N = H*W*C bytes per frame, consecutive frames N bytes apart.
 *  - Device pointers are CUDA device memory of the current device; the caller
 *    owns them.  Host pointers are ordinary (preferably pinned) host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is stream-ordered; a call returns once its work is enqueued,
 *    except where stated.
 *  - Every function returns VC_OK (0) or a VC_ERR_* code; none throws, none
 *    aborts.  On error nothing of the call's frames has been consumed from the
 *    keystream unless stated.
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef VCRYPT_H
#define VCRYPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define VC_OK 0
#define VC_ERR_ARG 1        /* null pointer, negative count, bad enum */
#define VC_ERR_KEY_RANGE 2  /* key outside the valid ranges of its map (Eq. 5, Eq. 6, logistic), or no such map */
#define VC_ERR_LAYOUT 3     /* H, W < 1; C not in {1,3,4}; n < 1; a subframe below 2 bytes; sizes too large */
#define VC_ERR_CUDA 4       /* a CUDA runtime call failed (message: vc_last_error) */
#define VC_ERR_OOM 5        /* device or host allocation failed */
#define VC_ERR_TIMEOUT 6    /* a bounded device-side wait gave up */
#define VC_ERR_SEQUENCE 7   /* frame submitted out of the stream's order */
#define VC_ERR_STATE 8      /* malformed checkpoint blob */
#define VC_ERR_UNSUPPORTED 9

/* ---- chaotic map of the PRBGs (Sec. 3) ---- */
#define VC_PLCM 0   /* key k = {x0^1, p^1, x0^2, p^2}: x0 in (0,1), p in (0, 1/2)        (Eq. 5) */
#define VC_2DLASM 1 /* key k = {x0, mu, y0, unused}: x0, y0 in (0,1),
                       mu in [.37,.38] u [.4,.42] u [.44,.93] u {1}                       (Eq. 6) */
#define VC_LOGISTIC 2 /* key k = {x0^1, r^1, x0^2, r^2}: x0 in (0,1), r in [3.9, 4]; the
                         logistic map x' = (r x)(1 - x) in the PLCM's place, as the paper
                         allows other chaotic maps (Sec. 7, advantage iii); per subframe
                         x0 = u, r = 3.9 + 0.1 u from PRBG_m as for the PLCM */

typedef struct {
  int32_t kind;  /* VC_PLCM, VC_2DLASM or VC_LOGISTIC */
  double k[4];   /* the key K of Alg. 1 (Sec. 5.1: four or three doubles) */
} vc_key;

typedef struct {
  int32_t height;      /* H, rows (the paper's frames are square, w x w) */
  int32_t width;       /* W, columns */
  int32_t channels;    /* C: 1, 3 (RGB, the paper's case) or 4 */
  int32_t n_subframes; /* n of Alg. 1 / Alg. 2: subframe i is pixels [floor(iP/n), floor((i+1)P/n)) */
  int32_t rounds;      /* r of Alg. 1, 1..16 (the paper uses 5, Sec. 6) */
} vc_layout;

typedef struct vc_ctx vc_ctx;

/* Create a cipher context for one video stream on the current CUDA device.
 * Validates the key (the ranges of its map: Eq. 5, Eq. 6, or the logistic
 * map's) and the layout, allocates the
 * device-resident chaotic state, and runs the key schedule of Alg. 1 (PRBG_m
 * keyed by K -> the parameters P_m of every PRBG_a^i) on the device
 * (synchronously).  Limits: H, W <= 16384, N = H*W*C < 2^31, n <= H*W, every
 * subframe >= 2 bytes.  *out receives the context (owned by the caller; free
 * with enc_destroy).  The device memory of contexts and batchers comes from a
 * stream-ordered pool of the library's own on each device: memory given back
 * is kept for reuse by later contexts until the process exits, and neither
 * allocation nor release waits for other work on the device.
 * Errors: VC_ERR_ARG, VC_ERR_KEY_RANGE, VC_ERR_LAYOUT, VC_ERR_OOM,
 * VC_ERR_CUDA. */
int enc_init(const vc_key* key, const vc_layout* layout, vc_ctx** out);

/* Encrypt nframes >= 0 consecutive frames of the stream (Alg. 1: per frame
 * s_c from PRBG_m; Alg. 2: r rounds of Eq. 1 then Eq. 3, with the diffusion
 * chains VC_OPT_DIFFUSION selects).  d_in and d_out are
 * device buffers of nframes*N bytes; d_in == d_out (in place) is allowed,
 * other overlap is not.  Advances the stream by nframes frames.  Errors:
 * VC_ERR_ARG, VC_ERR_CUDA. */
int encrypt_frames(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, void* stream);

/* Decrypt nframes consecutive frames (Eq. 4 then Eq. 2, rounds r-1..0), same
 * buffers, ordering and errors as encrypt_frames.  A decrypting context made
 * from the same key and layout reproduces the encrypting context's keystream
 * frame for frame. */
int decrypt_frames(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, void* stream);

/* encrypt_frames / decrypt_frames on frames frame_pitch bytes apart (the
 * frame_pitch of the boundary the cipher's inputs suggest, Alg. 1: a video V
 * of frames; e.g. frames inside a larger per-frame record, or rows of a
 * buffer pool).  frame_pitch = 0 means N (packed, as encrypt_frames);
 * otherwise frame_pitch >= N, any alignment, and the same pitch applies to
 * d_in and d_out (d_in == d_out allowed).  Only the N bytes at the start of
 * each frame slot are read or written.  Errors: those of encrypt_frames,
 * VC_ERR_ARG for 0 < frame_pitch < N. */
int encrypt_frames_pitched(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, size_t frame_pitch,
                           void* stream);
int decrypt_frames_pitched(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, size_t frame_pitch,
                           void* stream);

/* encrypt_frames / decrypt_frames on HOST buffers: copies h_in to the device,
 * runs the cipher, copies the result to h_out, in chunks that overlap copies
 * with compute; returns after the result is in h_out (synchronous).  direction
 * 0 = encrypt, 1 = decrypt.  Errors as above plus VC_ERR_OOM. */
int crypt_frames_host(vc_ctx* ctx, int32_t direction, const uint8_t* h_in, uint8_t* h_out, int32_t nframes,
                      void* stream);

/* crypt_frames_host without waiting for the result: enqueues the uploads, the
 * passes (on `stream`) and the downloads, and returns.  done_event, if not
 * null, is a cudaEvent_t of the caller, recorded after the call's last
 * download: once it has completed, h_out holds the result.  Until then h_in
 * must stay unchanged and h_out unread (pinned host memory, so the copies run
 * asynchronously; pageable memory makes the copies wait on the host).
 * enc_sync_status also waits for every download issued.  Consecutive calls on
 * one context pipeline: a call's first uploads and keystream start while the
 * previous call's last passes and downloads run (three staging buffers in
 * turn, each uploaded again after its previous download).  `stream` is not
 * ordered after the downloads.  As for encrypt_frames, the calls on one
 * context follow one another in the order of the stream they are given; a
 * caller that changes streams orders them itself.  Errors as
 * crypt_frames_host. */
int crypt_frames_host_async(vc_ctx* ctx, int32_t direction, const uint8_t* h_in, uint8_t* h_out, int32_t nframes,
                            void* stream, void* done_event);

/* ---- encryption without allocation ----
 * The paper has no counterpart of this entry point.  It serves callers that
 * must not allocate device memory while they work: programs whose GPU memory
 * is handed out by a framework's own pool or by a fixed budget reserved at
 * start-up, and latency-critical threads for which cudaMalloc, which may
 * synchronise the whole device, would stall the video pipeline.
 *
 * encrypt_frames_static does what encrypt_frames does (same arguments, same
 * ciphertext, same stream order, advances the stream the same way) but calls
 * no allocator: its scratch is one static device array of 16 MiB that the
 * library holds on every GPU that loads it, until the process exits.  The
 * caller still passes the input and output buffers and a context from
 * enc_init.
 *  - Limit: one frame needs about (r + 2) * N bytes of scratch plus small
 *    tables; a layout whose single frame does not fit in 16 MiB (768x768x3
 *    with r = 5 fits, 1280x720x3 does not) gets VC_ERR_UNSUPPORTED before any
 *    GPU work.  Frames that fit are processed several per pass.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it; make
 *    that first call before any stream capture.
 *  - All calls on a device share the one array and it keeps the last call's
 *    contents: calls whose GPU work overlaps in time (other host threads, or
 *    other streams without ordering between them) race on it.  Keep them on
 *    one stream or synchronise between them.  No byte of the array needs to
 *    start at zero: a call writes everything it reads.
 *  - On a context whose previous encrypt_frames call generated keystream
 *    ahead (VC_OPT_RUNAHEAD_CALLS), the call first undoes that run-ahead,
 *    which waits on the host for the context's internal keystream stream.
 *    Callers that must never wait can turn VC_OPT_RUNAHEAD_CALLS off, or use
 *    this entry point alone on the context.
 * Errors: VC_ERR_ARG, VC_ERR_UNSUPPORTED (frame too large), VC_ERR_CUDA. */
int encrypt_frames_static(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, void* stream);

/* ---- ragged batches (many streams per launch) ----
 * A batcher runs the frames of many streams -- each with its own key, layout
 * (resolution, channels, subframes, rounds), map and direction -- with one
 * launch per phase for the whole batch: frame schedules, shift tables, one
 * keystream kernel over every subframe chain of every stream, then one
 * persistent kernel per round over every (frame, tile) of every stream.  The
 * sequence is captured once per batch shape as a CUDA graph and replayed with
 * one graph launch per batch.  The results are byte-identical to running
 * each job alone with encrypt_frames / decrypt_frames. */
typedef struct {
  vc_ctx* ctx;          /* the stream's context; at most one job per context per batch */
  int32_t direction;    /* 0 = encrypt, 1 = decrypt */
  const uint8_t* d_in;  /* nframes * N bytes, device */
  uint8_t* d_out;       /* nframes * N bytes, device; may equal d_in unless the context has 1 round */
  int32_t nframes;      /* >= 0; 0 leaves the job out */
} vc_job;

typedef struct vc_batcher vc_batcher;

/* Create a batcher on the current device (owns its scratch pool, descriptor
 * staging and graph cache).  Errors: VC_ERR_ARG, VC_ERR_OOM, VC_ERR_CUDA. */
int vc_batcher_create(vc_batcher** out);

/* Enqueue one batch on `stream`: equivalent to the jobs' encrypt_frames /
 * decrypt_frames calls, advancing each context by its job's frames.  Returns
 * once enqueued; the host-side job array may be reused at once.  Later calls
 * on a context are ordered after the batch.  Errors: VC_ERR_ARG (null or
 * repeated context, bad direction, in-place job of a 1-round context),
 * VC_ERR_OOM, VC_ERR_CUDA. */
int vc_batch_submit(vc_batcher* b, const vc_job* jobs, int32_t njobs, void* stream);

/* Batcher options.
 * VC_BOPT_GRAPH:       1 (default) replay a captured CUDA graph per batch
 *                      shape; 0 plain kernel launches.
 * VC_BOPT_CTAS_PER_SM: CTAs per SM of the persistent round kernels; 0
 *                      (default) = the occupancy maximum.
 * VC_BOPT_RUNAHEAD:    A > 0 keeps every stream's keystream (which does not
 *                      depend on the frames) A frames ahead: each submit also
 *                      launches, on an internal stream, the keystream of the
 *                      stream's next frames into a device ring of 2A + 1
 *                      frame slots, so a later batch only runs the rounds.
 *                      A job may then ask for at most A frames, and a stream
 *                      with keystream produced ahead accepts no single-stream
 *                      calls or checkpoint (VC_ERR_SEQUENCE).  0 (default): off.
 * VC_BOPT_SINE:        the sine reduction of 2DLASM chains whose keystream a
 *                      batch generates (Eq. 6, both forms give the same bits):
 *                      1 all on the binary64 pipe (the shorter dependency
 *                      chain), 0 with the rounding, floor and t - k pi/2 on the
 *                      integer pipes (fewer binary64 operations), -1 (default)
 *                      chooses per batch: 1 while the batch's 2DLASM chains
 *                      fill at most about 3.5 warps per SM, else 0.
 * VC_BOPT_SPLIT:       batches with the keystream inside (run-ahead off):
 *                      jobs whose serial chains take much longer than the
 *                      others' go to a second lane on an internal stream --
 *                      their keystream in CTAs that each hold a whole SM,
 *                      their rounds behind it -- while the other jobs run
 *                      beside them (the results are the same).  -1 (default)
 *                      automatic: the jobs whose chains take at least half
 *                      the longest, when that one is long (about 2 ms) and
 *                      they are at most three quarters of the jobs; 1 split
 *                      whenever the jobs' chains differ; 0 never.
 * VC_BOPT_KS_PLACE:    where the keystream produced ahead (VC_BOPT_RUNAHEAD)
 *                      runs: 0 (default) one-warp CTAs sharing the SMs with
 *                      other work; 1 as the context's own calls place it
 *                      (VC_OPT_KS_SM_WARPS, -1 automatic: CTAs that hold
 *                      whole SMs when they leave enough SMs free).  A context
 *                      with VC_OPT_KS_SM_WARPS > 0 holds SMs in both.
 * VC_BOPT_KS_PRIORITY: the stream priority of the keystream produced ahead:
 *                      0 (default) the device's highest (a chain that starts
 *                      late delays every frame behind it), 1 its lowest (the
 *                      batches' round kernels, on a stream of higher priority,
 *                      take the SMs that free up first).  It applies to the
 *                      streams whose first production comes after it is set.
 * VC_BOPT_KS_URGENT:   1: a production for a stream that has no frame
 *                      produced ahead of its next one (it fell behind, or it
 *                      was just admitted) runs on a second production stream
 *                      of the device's highest priority, still after the
 *                      stream's earlier productions; 0 (default): all on one.
 * Errors: VC_ERR_ARG. */
#define VC_BOPT_GRAPH 1
#define VC_BOPT_CTAS_PER_SM 2
#define VC_BOPT_RUNAHEAD 3
#define VC_BOPT_SINE 4
#define VC_BOPT_SPLIT 5
#define VC_BOPT_KS_PLACE 6
#define VC_BOPT_KS_PRIORITY 7
#define VC_BOPT_KS_URGENT 8
int vc_batcher_set_option(vc_batcher* b, int32_t option, int64_t value);

/* With run-ahead on: start producing the keystream of each context's next
 * A frames now (e.g. right after a stream is admitted), on the context's
 * production stream: the next frame alone first, the rest queued behind it.
 * A call for a context whose production is still in flight adds nothing.
 * Productions after a submit are queued behind the ones still running (at
 * most four in flight per context); a production overwriting a ring slot
 * waits, on the device, for the batch that read the slot.
 * Errors: VC_ERR_ARG (run-ahead off, null or repeated context), VC_ERR_OOM,
 * VC_ERR_CUDA. */
int vc_batch_prefetch(vc_batcher* b, vc_ctx* const* ctxs, int32_t n);

/* 1 if the keystream of the context's next nframes frames has been produced
 * on the device (a batch using them will not wait for the producer), 0 if not
 * yet, -code on error.  Never blocks. */
int vc_batch_ready(vc_batcher* b, const vc_ctx* ctx, int32_t nframes);

/* Synchronise and free the batcher. */
void vc_batcher_destroy(vc_batcher* b);

/* ---- serving: the per-tick work of a continuous-batching loop ----
 * Real time (Sec. 6): every frame of a stream must be done within its frame
 * time (41.7 ms at 24 FPS).  A server holds many streams; each tick it takes,
 * for every stream, the frames that have arrived by the stream's clock
 * (frame k arrives at t_arrival + k / fps seconds after the server's
 * creation) and, in batch mode, whose keystream run-ahead is on the device,
 * and submits them as one ragged batch (mode 0) or as one encrypt_frames /
 * decrypt_frames call per frame (mode 1, for comparison: each stream's calls
 * on its own CUDA stream, created by vc_server_add, so that different
 * streams' calls run concurrently; a frame completes when its stream's calls
 * of the tick do).  Per-frame latency =
 * device completion time (CUDA event) - arrival time.  All calls are on the
 * host thread that drives the loop.
 *
 * vc_server_create: max_frames_per_tick 1..64 (also the keystream run-ahead of
 *   mode 0); stream = the CUDA stream the work is enqueued on.  Records the
 *   time origin (synchronises it).  Errors: VC_ERR_ARG, VC_ERR_OOM, VC_ERR_CUDA.
 * vc_server_add: registers a stream (the context stays owned by the caller and
 *   must outlive its registration).  Frame k is read from frame k mod src_period
 *   of d_src, which holds src_period + max_frames_per_tick - 1 frames of
 *   frame_bytes bytes (so a tick's frames are contiguous), and written to frame
 *   k mod ring_frames of d_ring.  *id receives the stream's handle.  Mode 0
 *   starts producing its keystream.  Errors: VC_ERR_ARG (and those of
 *   vc_batch_prefetch).
 * vc_server_tick: now = seconds since creation (host clock); *frames_submitted
 *   receives the number of frames submitted (may be 0).  Errors: those of
 *   vc_batch_submit / encrypt_frames / decrypt_frames, VC_ERR_CUDA.
 * vc_server_drain: returns up to cap completed frames (stream id, frame index,
 *   arrival time in s, latency in ms), oldest first; block = 1 waits for the
 *   oldest tick in flight.  Errors: VC_ERR_ARG, VC_ERR_CUDA.
 * vc_server_stream_done: 1 when all frames_total frames of the stream have
 *   completed, 0 otherwise, -VC_ERR_ARG for a bad handle.
 * vc_server_remove: unregisters a stream (waits for its frames in flight);
 *   the caller may then destroy its context.  Errors: VC_ERR_ARG.
 * vc_server_destroy: waits for the server's work; the contexts of streams
 *   still registered must still exist (the server detaches its internal
 *   streams from them), so remove a stream before destroying its context.
 * vc_server_inflight: ticks submitted and not yet drained. */
typedef struct vc_server vc_server;
int vc_server_create(int32_t mode, int32_t max_frames_per_tick, void* stream, vc_server** out);
int vc_server_add(vc_server* s, vc_ctx* ctx, int32_t direction, int64_t frame_bytes, const uint8_t* d_src,
                  int32_t src_period, uint8_t* d_ring, int32_t ring_frames, double fps, double t_arrival,
                  int64_t frames_total, int32_t* id);
int vc_server_tick(vc_server* s, double now, int32_t* frames_submitted);
int vc_server_drain(vc_server* s, int32_t block, int32_t cap, int32_t* ids, int64_t* frames, double* arrival_s,
                    double* latency_ms, int32_t* n);
int vc_server_stream_done(const vc_server* s, int32_t id);
int vc_server_remove(vc_server* s, int32_t id);
int32_t vc_server_inflight(const vc_server* s);
/* vc_server_set_option: an option of a batching server (mode 0): a batcher
 * option (VC_BOPT_*; the run-ahead is the server's max_frames_per_tick and
 * cannot be set), or VC_SOPT_QUEUED_TICKS: q > 0 submits a tick only while
 * fewer than q earlier ticks wait for the device to start them (a tick that
 * would queue deeper submits nothing, and its frames join the next, larger
 * batch); 0 (default) submits every tick.  VC_SOPT_LANES: k in 1..8 batching
 * lanes, set before the first stream and after the batcher options: tick i
 * goes to lane i mod k, each lane with its own batcher and a stream of the
 * server stream's priority (lane 0 is the server's stream), so that a tick
 * whose kernels wait for SMs does not hold up the next ticks; 1 (default).
 * Errors: VC_ERR_ARG (mode 1, VC_BOPT_RUNAHEAD, bad option or value, options
 * in the wrong order), VC_ERR_CUDA. */
#define VC_SOPT_QUEUED_TICKS 100
#define VC_SOPT_LANES 101
int vc_server_set_option(vc_server* s, int32_t option, int64_t value);
void vc_server_destroy(vc_server* s);

/* Size in bytes of a checkpoint of the context's stream state (chaotic map
 * values, pending keystream bytes, PRBG_m, frame counter). */
size_t enc_state_size(const vc_ctx* ctx);

/* Write the checkpoint into buf (host, *len >= enc_state_size); synchronises
 * the context's last stream.  *len receives the size.  Errors: VC_ERR_ARG,
 * VC_ERR_CUDA. */
int enc_save_state(vc_ctx* ctx, void* buf, size_t* len);

/* Restore a checkpoint taken from a context with the same key kind and layout.
 * Errors: VC_ERR_ARG, VC_ERR_STATE (size/layout mismatch), VC_ERR_CUDA. */
int enc_load_state(vc_ctx* ctx, const void* buf, size_t len);

/* Frames consumed so far by this context. */
int64_t enc_frame_index(const vc_ctx* ctx);

/* Synchronise the context's last stream and return the first error recorded
 * by its device code or its asynchronous CUDA work (VC_OK if none); clears it. */
int enc_sync_status(vc_ctx* ctx);

/* Make `stream` wait, on the device (the host does not block), for all work
 * the context has enqueued so far on its internal streams: the keystream
 * generated ahead for the next call (VC_OPT_RUNAHEAD_CALLS), a batcher's
 * productions, the copies of host-buffer calls.  An event recorded on
 * `stream` afterwards therefore marks the end of everything the context's
 * calls so far have set going (e.g. to time a run of calls).
 * Errors: VC_ERR_ARG, VC_ERR_CUDA. */
int enc_join(vc_ctx* ctx, void* stream);

/* ---- tuning options (enc_set_option / enc_get_option) ----
 * VC_OPT_CHUNK:    frames per internal pass (same as enc_set_chunk), 1..65535.
 * VC_OPT_PLCM_INT: 1 (default) evaluates the PLCM division and subtraction of
 *                  Eq. 5 exactly on the integer pipes, 0 uses the binary64
 *                  pipe; both give identical bits (IEEE-754 round to nearest).
 *                  2 and 3 are test modes: the integer form computes each
 *                  range and then rewrites it through its exact fallback, for
 *                  every subframe (2) or the odd-numbered ones only (3, lanes
 *                  of one warp take different paths), so the fallback
 *                  (normally taken about once in 2^30 iterates) is exercised;
 *                  the bytes are again identical.
 * VC_OPT_KS_LANES: lanes per subframe chain pair in the keystream kernel:
 *                  2 (default, one lane per chaotic map) or 1 (one thread runs
 *                  both maps of the pair).
 * VC_OPT_OVERLAP:  1 (default) generates the keystream of the next pass on an
 *                  internal stream while the rounds of the current pass run on
 *                  the caller's stream (the keystream does not depend on the
 *                  frames); 0 runs everything on the caller's stream.
 * VC_OPT_TILE_ROWS: frame rows per tile of the round kernels, a power of two
 *                  1..32 (capped so that a tile's shared memory -- one 32-bit
 *                  slot per pixel for C = 3 and 4, a byte for C = 1, plus the
 *                  tile's keystream when rows are whole 16-byte pieces -- stays
 *                  within 192 KB); 0 (default) takes the largest whose tile
 *                  stays within 110 KB.  Reading it back gives the rows in use.
 * VC_OPT_KS_SM_WARPS: -1..4.  k > 0 runs the keystream of each pass in CTAs
 *                  of k warps that each occupy a whole SM (they claim all of
 *                  its shared memory), on an internal stream of the device's
 *                  highest priority, so that the round kernels of the previous
 *                  pass run on the other SMs instead of taking issue slots from
 *                  the latency-bound chains; 0 lets both share every SM on a
 *                  normal-priority stream; -1 (default) chooses when
 *                  overlapping: PLCM 4 warps (one per SM sub-partition) if
 *                  those CTAs fill at most half of the SMs; 2DLASM (bound by
 *                  the SM's binary64 pipe) 2 warps if at least an eighth of
 *                  the SMs stay free, else as PLCM; otherwise 0.  The
 *                  keystream a batcher produces ahead (VC_BOPT_RUNAHEAD) for
 *                  this context holds SMs only when k > 0 is set explicitly
 *                  (else one-warp CTAs share the SMs: many streams' chains
 *                  pack the pipes better).
 * VC_OPT_RUNAHEAD_CALLS: 1 (default) with overlap: at the end of a call the
 *                  keystream of the next call's first pass is generated on the
 *                  internal stream, so it overlaps this call's last rounds; the
 *                  chain state from before it is kept on the device, and a
 *                  checkpoint, a batch, or an option that reallocates scratch
 *                  first undoes it exactly (nothing is observable but time);
 *                  0 turns it off (and undoes one that is pending).
 * VC_OPT_DIFFUSION: 0 (default) diffuses each subframe as one chain over its
 *                  bytes in memory order (the cipher of Eq. 3 / Eq. 4 as read
 *                  here); 1 runs one chain per colour channel over the
 *                  subframe's pixels, seeded by the same channel of the last
 *                  pixel of the next subframe (a variant: a plaintext change
 *                  in one channel then never reaches the others).  1 needs at
 *                  least 2 pixels in every subframe (else VC_ERR_LAYOUT) and
 *                  the round kernels' shared memory for word carries (a
 *                  layout whose needs exceed the device's: VC_ERR_LAYOUT);
 *                  it runs through encrypt_frames, decrypt_frames,
 *                  crypt_frames_host and batches (encrypt_frames_static
 *                  returns VC_ERR_UNSUPPORTED).  The
 *                  decrypting context must use the value the encrypting one
 *                  used; checkpoints do not record it.
 * VC_OPT_CHUNK = 0 selects frames per pass automatically (default). */
#define VC_OPT_CHUNK 1
#define VC_OPT_PLCM_INT 2
#define VC_OPT_KS_LANES 3
#define VC_OPT_OVERLAP 4
#define VC_OPT_TILE_ROWS 5
#define VC_OPT_KS_SM_WARPS 6
#define VC_OPT_RUNAHEAD_CALLS 7
#define VC_OPT_DIFFUSION 8

/* Set / read a tuning option.  Options never change the ciphertext.
 * Errors: VC_ERR_ARG (unknown option or value out of range). */
int enc_set_option(vc_ctx* ctx, int32_t option, int64_t value);
int enc_get_option(const vc_ctx* ctx, int32_t option, int64_t* value);

/* Upper bound on frames processed per internal pass (scratch memory grows with
 * it: about 2 (r + 2) N bytes per frame).  Default: automatic (about a sixth of
 * the call's frames, at most 64). */
int enc_set_chunk(vc_ctx* ctx, int32_t frames_per_pass);

/* Stage timing for profiling.  While enabled, every pass brackets its stages
 * with CUDA events recorded on the pass's stream: 0 = frame schedule (s_c and
 * the Eq. 1 shift table), 1 = keystream kernel, 2 = round kernels (all r rounds
 * and the diffusion fix-up).  Errors: VC_ERR_ARG. */
int enc_profile_enable(vc_ctx* ctx, int32_t enable);

/* Device milliseconds and kernel launches per stage accumulated since the last
 * read (ms3[3], launches3[3]); synchronises the recorded events and resets
 * the counters.  Errors: VC_ERR_ARG, VC_ERR_CUDA. */
int enc_profile_read(vc_ctx* ctx, double* ms3, int64_t* launches3);

/* ---- statistical and security measures (Sec. 4, Sec. 5) on the device ----
 * Frames are nframes x height x width x channels uint8 (HWC, frames
 * contiguous), device pointers; results are per frame and channel, in that
 * order, in caller-owned device arrays.  Stream-ordered.  Errors: VC_ERR_ARG
 * (shapes, null pointers), VC_ERR_CUDA.
 *
 * vc_stats_histogram: counts z[f][c][0..255] (uint32, 256 per frame and
 *   channel), and from them (each may be NULL) chi^2 = sum (z - e)^2 / e with
 *   e = pixels / 256 (Sec. 4.1), the histogram variance
 *   1/256^2 sum_i sum_j (z_i - z_j)^2 / 2 (Sec. 4.1) and the Shannon entropy
 *   sum p log2(1/p) (Sec. 4.3).
 * vc_stats_correlation: correlation coefficient cov(x, y) / sqrt(D(x) D(y))
 *   (1/N moments) of adjacent pixel pairs (Sec. 4.2): direction 0 horizontal
 *   (right neighbour), 1 vertical (lower), 2 diagonal (lower right).  d_pairs
 *   holds npairs pixel indices (row * width + column) of the pairs' first
 *   pixels (the paper samples them at random; indices whose pair leaves the
 *   frame are skipped), or is NULL for all pairs of the frame (npairs ignored).
 *   d_sums: scratch of 6 uint64 per frame and channel (exact moment sums, and
 *   the pairs used).
 * vc_stats_local_entropy: the (k, T_B) local entropy (Sec. 4.3) of one channel:
 *   the mean over nblocks blocks of side x side pixels, top-left corners
 *   d_blocks[2b], d_blocks[2b + 1] (row, column; chosen at random by the
 *   caller), of each block's entropy; d_block_ent receives nframes x nblocks
 *   block entropies (NaN for a block outside the frame), d_mean the means.
 * vc_stats_npcr_uaci: NPCR = #{a != b} / pixels x 100 and UACI =
 *   sum |a - b| / (pixels x 255) x 100 (Sec. 5.2) between frames of a and b;
 *   d_sums: scratch of 2 uint64 per frame and channel. */
int vc_stats_histogram(const uint8_t* d_frames, int32_t nframes, int32_t height, int32_t width, int32_t channels,
                       uint32_t* d_hist, double* d_chi2, double* d_var, double* d_entropy, void* stream);
int vc_stats_correlation(const uint8_t* d_frames, int32_t nframes, int32_t height, int32_t width, int32_t channels,
                         int32_t direction, const int32_t* d_pairs, int64_t npairs, uint64_t* d_sums, double* d_r,
                         void* stream);
int vc_stats_local_entropy(const uint8_t* d_frames, int32_t nframes, int32_t height, int32_t width, int32_t channels,
                           int32_t channel, const int32_t* d_blocks, int32_t nblocks, int32_t side,
                           double* d_block_ent, double* d_mean, void* stream);
int vc_stats_npcr_uaci(const uint8_t* d_a, const uint8_t* d_b, int32_t nframes, int32_t height, int32_t width,
                       int32_t channels, uint64_t* d_sums, double* d_npcr, double* d_uaci, void* stream);

/* Release the context and its device memory.  enc_destroy first waits for
 * the context's work (its internal streams and the stream of its last call);
 * when it returns, nothing of the context runs any more.
 * enc_destroy_async does not wait: the device memory goes back to the
 * library's stream-ordered pool after the work enqueued so far, and the host
 * object is freed at once.  The caller keeps the buffers that this work reads
 * or writes (its frames) alive until that work is complete (e.g. an event on
 * the stream of the last call).  A context whose keystream was generated
 * ahead (run-ahead) may still be running that keystream when this returns; it
 * touches only the context's own memory.  Both accept NULL. */
void enc_destroy(vc_ctx* ctx);
void enc_destroy_async(vc_ctx* ctx);

/* Human-readable text of a status code; last CUDA error text of this thread. */
const char* vc_strerror(int code);
const char* vc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VCRYPT_H */
