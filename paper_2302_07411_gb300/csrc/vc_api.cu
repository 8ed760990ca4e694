// vc_api.cu -- the C ABI of include/vcrypt.h and include/vcrypt_debug.h:
// argument checks, device memory of a stream context, and the order of the
// kernel launches of one pass (Alg. 1 / Alg. 2 on the GPU).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <unordered_set>
#include <vector>

#include "vc_internal.h"
#include "vcrypt.h"
#include "vcrypt_debug.h"

using vc::Layout;

namespace {

thread_local char g_err[512] = "";

void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

#define VC_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return VC_ERR_CUDA;                                                                  \
    }                                                                                      \
  } while (0)

// bytes of one row-band tile in shared memory (its pixel slots and, when staged,
// its keystream): two CTAs share an SM (deeper tiles measured faster than four
// shallower CTAs per SM, and they contend less with a concurrent keystream)
constexpr size_t kTileBudget = 110 * 1024;
constexpr size_t kTileHardCap = 192 * 1024;  // rows asked for explicitly (VC_OPT_TILE_ROWS) may use up to this
constexpr uint32_t kStateMagic = 0x56435354u;  // "VCST"
constexpr uint32_t kStateVersion = 1;

// ---- device memory: a stream-ordered pool of the library's own per device.
// A buffer is taken from it at once (its allocation stream carries nothing
// else) and given back in stream order after the work that used it, so that
// releasing a context's or a batcher's memory never waits for the device (a
// plain cudaFree waits for all of it, e.g. for other streams' long keystream
// chains).  The pool keeps its memory mapped between uses and never makes an
// allocation wait for another stream's work.
constexpr int kMaxPoolDevices = 64;
struct DevPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t st = nullptr;
};
std::mutex g_pool_mu;
DevPool g_pool[kMaxPoolDevices];

cudaError_t dev_pool(DevPool** out) {  // under g_pool_mu
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  DevPool& d = g_pool[dev];
  if (!d.pool) {
    cudaMemPoolProps pr{};
    pr.allocType = cudaMemAllocationTypePinned;
    pr.handleTypes = cudaMemHandleTypeNone;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &pr);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ull;
    int no = 0;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
    cudaStream_t st = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    d.pool = p;
    d.st = st;
  }
  *out = &d;
  return cudaSuccess;
}

// bytes of device memory, usable on every stream when this returns
template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  *p = nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  DevPool* d = nullptr;
  cudaError_t e = dev_pool(&d);
  void* v = nullptr;
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&v, bytes ? bytes : 1, d->pool, d->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->st);
  if (e == cudaSuccess) *p = static_cast<T*>(v);
  return e;
}

// p (may be null) back to the pool once the work enqueued on `after` so far is
// complete (after == nullptr: at once, for memory no work has used)
void dev_free(void* p, cudaStream_t after) {
  if (!p) return;
  if (!after) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    DevPool* d = nullptr;
    if (dev_pool(&d) == cudaSuccess) after = d->st;
  }
  cudaFreeAsync(p, after);
}

bool key_valid(const vc_key& k) {
  if (k.kind == VC_PLCM) {
    for (int i = 0; i < 4; i += 2)
      if (!(k.k[i] > 0.0 && k.k[i] < 1.0 && k.k[i + 1] > 0.0 && k.k[i + 1] < 0.5)) return false;
    return true;
  }
  if (k.kind == VC_2DLASM) {
    const double mu = k.k[1];
    const bool mu_ok = (mu >= 0.37 && mu <= 0.38) || (mu >= 0.4 && mu <= 0.42) || (mu >= 0.44 && mu <= 0.93) ||
                       mu == 1.0;
    return k.k[0] > 0.0 && k.k[0] < 1.0 && k.k[2] > 0.0 && k.k[2] < 1.0 && mu_ok;
  }
  if (k.kind == VC_LOGISTIC) {
    for (int i = 0; i < 4; i += 2)
      if (!(k.k[i] > 0.0 && k.k[i] < 1.0 && k.k[i + 1] >= 3.9 && k.k[i + 1] <= 4.0)) return false;
    return true;
  }
  return false;
}

// Geometry checks and the tile shape of the round kernels (tile_rows_max: 0 =
// as many rows, up to 32, as fit the shared-memory budget).
int make_layout(const vc_layout& l, Layout* L, int tile_rows_max = 0) {
  if (l.height < 1 || l.width < 1 || l.height > 16384 || l.width > 16384) return VC_ERR_LAYOUT;
  if (!(l.channels == 1 || l.channels == 3 || l.channels == 4)) return VC_ERR_LAYOUT;
  if (l.rounds < 1 || l.rounds > 16 || l.n_subframes < 1) return VC_ERR_LAYOUT;
  const long long P = (long long)l.height * l.width;
  const long long N = P * l.channels;
  if (N >= (1LL << 31) - 4096) return VC_ERR_LAYOUT;
  if (l.n_subframes > P) return VC_ERR_LAYOUT;
  if ((long long)l.channels * (P / l.n_subframes) < 2) return VC_ERR_LAYOUT;  // every subframe >= 2 bytes
  const long long rowb = (long long)l.width * l.channels;
  if (rowb > vc::kMaxRowBytes) return VC_ERR_LAYOUT;
  // a tile row in shared memory: its pixel slots, and its keystream when rows are whole 16-byte pieces
  const long long zrow = vc::tile_row_bytes(l.width, l.channels) + ((rowb & 15) == 0 ? rowb : 0);
  const size_t cap = tile_rows_max > 0 ? kTileHardCap : kTileBudget;
  int T = tile_rows_max > 0 ? tile_rows_max : 32;
  while (T > 1 && (size_t)T * zrow > cap) T >>= 1;
  if ((size_t)T * zrow > kTileHardCap) return VC_ERR_LAYOUT;
  const int NT = (l.height + T - 1) / T;
  if (NT > vc::kMaxTiles) return VC_ERR_LAYOUT;
  const int R = T >= 8 ? T / 8 : 1;
  L->H = l.height;
  L->W = l.width;
  L->C = l.channels;
  L->n = l.n_subframes;
  L->rounds = l.rounds;
  L->P = (int)P;
  L->N = (int)N;
  L->Npad = (N + 255) & ~255LL;
  L->T = T;
  L->NT = NT;
  L->R = R;
  L->lgR = R == 1 ? 0 : (R == 2 ? 1 : (R == 4 ? 2 : 3));
  L->NS = (l.height + R - 1) / R;
  L->ZS = vc::tile_row_stride(l.width, l.channels);
  // a window of m pixels holds at most floor(m n / P) + 1 subframe starts
  const long long tile_starts = (long long)T * l.width * l.n_subframes / P + 2;
  L->SC = tile_starts <= vc::kMaxSeedSlots ? (int)((tile_starts + 15) & ~15LL) : 0;
  return VC_OK;
}

}  // namespace

struct vc_ctx {
  int kind = 0;
  Layout L{};
  vc_layout user_layout{};
  int tile_rows = 0;  // 0 = automatic
  int dev = 0;
  // partition tables
  int* d_pi = nullptr;
  uint32_t* d_sbits = nullptr;
  int* d_srank = nullptr;
  int* d_fixlim = nullptr;
  // stream state
  vc::MainPrbg* d_main = nullptr;
  double* d_st = nullptr;
  double* d_par = nullptr;
  uint64_t* d_carry = nullptr;
  int* d_carry_len = nullptr;
  // per-pass scratch, sized for `cap` frames.  The keystream side (keystream,
  // s_c, shift tables) is double-buffered so that pass k+1's keystream can be
  // generated on ks_stream while pass k's rounds run on the caller's stream.
  int chunk = 0;  // frames per pass; 0 = automatic
  int cap = 0;
  uint8_t* d_ks[2] = {nullptr, nullptr};
  long long* d_sc[2] = {nullptr, nullptr};
  int* d_kmod[2] = {nullptr, nullptr};
  uint8_t* d_buf[2] = {nullptr, nullptr};
  uint8_t* d_agg[2] = {nullptr, nullptr};
  bool overlap = true;
  // > 0: the pass keystream runs in CTAs of this many warps that each hold a
  // whole SM, on a ks_stream of the device's highest priority; -1: 4 warps
  // (one per SM sub-partition) when those CTAs fill at most half the SMs
  int ks_sm_warps = -1;
  int num_sms = 0;
  cudaStream_t ks_stream = nullptr;
  // the frame schedule (s_c, shift tables) of a pass runs here, beside the
  // pass's keystream kernel; ev_sc_in / ev_sc_out order it after what the
  // keystream side held before and the keystream side after it
  cudaStream_t sc_stream = nullptr;
  cudaEvent_t ev_sc_in = nullptr, ev_sc_out = nullptr;
  cudaEvent_t ev_ks[2] = {};   // keystream buffer b written
  cudaEvent_t ev_rd[2] = {};   // rounds reading buffer b done
  cudaEvent_t ev_entry = nullptr;
  cudaEvent_t ev_batch = nullptr;  // recorded after a batch that used this context
  cudaEvent_t ev_free = nullptr;   // joins the other streams into ks_stream before a free
  bool batch_pending = false;
  // keystream run-ahead ring of the batcher: frame f's keystream, s_c and shift
  // table live in slot f mod ring_cap; `produced` frames exist (the chaotic
  // state has advanced that far), `frame` have been consumed.
  uint8_t* ring_ks = nullptr;
  long long* ring_sc = nullptr;
  int* ring_kmod = nullptr;
  int ring_cap = 0;
  // per ring slot: recorded after the batch that read it, so that a production
  // overwriting the slot waits for that batch and for no later one
  std::vector<cudaEvent_t> ev_slot;
  // the productions' stream (created with the ring, at the priority the
  // batcher asks for: VC_BOPT_KS_PRIORITY)
  cudaStream_t prod_stream = nullptr;
  // a second production stream of the device's highest priority, for the
  // productions of a stream with no frame produced ahead (VC_BOPT_KS_URGENT);
  // last_prod: the stream of the last production (chain order across the two)
  cudaStream_t prod_urgent = nullptr;
  cudaStream_t last_prod = nullptr;
  int64_t produced = 0;
  // productions of the ring run on ks_stream; the last eight are tracked so
  // that readiness can be polled without blocking
  static constexpr int kProdEv = 8;
  cudaEvent_t ev_prod[kProdEv] = {};
  int64_t prod_upto[kProdEv] = {};
  int64_t nprod = 0;
  int64_t produced_done = 0;  // frames known complete on the device
  int64_t passes = 0;
  // keystream run-ahead across calls: at the end of a call the first pass of
  // the next one (spec_frames frames) is generated into buffer spec_b; the next
  // call's rounds take its frames (spec_used so far).  d_snap holds the chain
  // state from before it, so that it can be undone exactly.
  bool spec_enabled = true;
  int spec_b = -1, spec_frames = 0, spec_used = 0;
  uint8_t* d_snap = nullptr;
  // staging for host-buffer calls
  static constexpr int kIoBufs = 3;
  uint8_t* d_io[kIoBufs] = {nullptr, nullptr, nullptr};
  int io_cap = 0;
  long long io_uses = 0;  // staging passes issued so far (buffer io_uses % kIoBufs is the next one)
  cudaStream_t copy_stream = nullptr;  // uploads (and table builds)
  cudaStream_t d2h_stream = nullptr;   // downloads of host-buffer calls
  cudaEvent_t ev_io[3 * kIoBufs] = {};
  cudaEvent_t ev[6] = {};
  int64_t frame = 0;
  cudaStream_t last = nullptr;
  int plcm_int = 1;  // 0 binary64 pipe, 1 integer pipes, 2/3 integer pipes + forced exact fallback (tests)
  bool diff_pc = false;  // diffusion chains: false = over the subframe's bytes (R4), true = one per channel
  int ks_lanes = 2;
  // stage profiling: recorded (stage, start, end) event pairs and a free pool
  bool prof = false;
  struct Mark {
    int stage, launches;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;

  vc::Tables tables() const { return vc::Tables{d_pi, d_sbits, d_srank, d_fixlim}; }
  vc::Chains chains() const { return vc::Chains{d_st, d_par, d_carry, d_carry_len}; }
  // PLCM and logistic pairs: x per map, (p, 1/2 - p) or (r, 0) per map;
  // 2DLASM pairs: (x, y) per map, pi * mu per map
  int state_words() const { return kind == VC_2DLASM ? 4 : 2; }
  int par_words() const { return kind == VC_2DLASM ? 2 : 4; }
};

namespace {

void sync_all(vc_ctx* c) {
  if (c->last) cudaStreamSynchronize(c->last);
  if (c->ks_stream) cudaStreamSynchronize(c->ks_stream);
  if (c->prod_stream) cudaStreamSynchronize(c->prod_stream);
  if (c->prod_urgent) cudaStreamSynchronize(c->prod_urgent);
  if (c->sc_stream) cudaStreamSynchronize(c->sc_stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  if (c->d2h_stream) cudaStreamSynchronize(c->d2h_stream);
}

// The per-channel round CTA (word carries and seeds) fits the device's shared
// memory per block.
bool pc_smem_fits(const vc_ctx* c, const Layout* L2 = nullptr) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev) != cudaSuccess) {
    cudaGetLastError();
    optin = 48 * 1024;
  }
  return vc::round_smem_bytes(L2 ? *L2 : c->L, true) <= (size_t)optin;
}

// ks_stream after everything enqueued so far on the context's other streams
// (its buffers are given back to the pool there, in stream order).
cudaStream_t ctx_join(vc_ctx* c) {
  cudaStream_t ks = c->ks_stream;
  if (!ks || !c->ev_free) {  // a context whose creation failed part-way: nothing of it ran
    sync_all(c);
    return nullptr;
  }
  for (cudaStream_t o : {c->last, c->copy_stream, c->d2h_stream, c->prod_stream, c->prod_urgent, c->sc_stream})
    if (o && o != ks && cudaEventRecord(c->ev_free, o) == cudaSuccess) cudaStreamWaitEvent(ks, c->ev_free, 0);
  return ks;
}

}  // namespace

void vc::ctx_release_stream(vc_ctx* c, cudaStream_t s) {
  if (!c || !s || c->last != s) return;
  // later work orders itself after the internal keystream stream, which now
  // waits (on the device) for what was enqueued on s
  if (c->ks_stream && c->ev_free && cudaEventRecord(c->ev_free, s) == cudaSuccess &&
      cudaStreamWaitEvent(c->ks_stream, c->ev_free, 0) == cudaSuccess) {
    c->last = nullptr;
    return;
  }
  cudaGetLastError();
  cudaStreamSynchronize(s);
  c->last = nullptr;
}

namespace {

// the pass scratch back to the pool after the work enqueued on `after`
void free_scratch(vc_ctx* c, cudaStream_t after) {
  for (int b = 0; b < 2; b++) {
    dev_free(c->d_ks[b], after);
    dev_free(c->d_sc[b], after);
    dev_free(c->d_kmod[b], after);
    dev_free(c->d_buf[b], after);
    dev_free(c->d_agg[b], after);
    c->d_ks[b] = c->d_buf[b] = c->d_agg[b] = nullptr;
    c->d_sc[b] = nullptr;
    c->d_kmod[b] = nullptr;
  }
  c->cap = 0;
}

int spec_rollback(vc_ctx* c);

int ensure_scratch(vc_ctx* c, int frames) {
  if (frames <= c->cap) return VC_OK;
  int rc = spec_rollback(c);
  if (rc) return rc;
  free_scratch(c, ctx_join(c));  // after the passes that used it
  const Layout& L = c->L;
  const size_t F = (size_t)frames;
  bool ok = true;
  for (int b = 0; b < 2 && ok; b++) {
    ok = dev_alloc(&c->d_ks[b], F * L.rounds * L.Npad) == cudaSuccess &&
         dev_alloc(&c->d_sc[b], F * sizeof(long long)) == cudaSuccess &&
         dev_alloc(&c->d_kmod[b], F * L.H * sizeof(int)) == cudaSuccess &&
         dev_alloc(&c->d_buf[b], F * L.Npad) == cudaSuccess && dev_alloc(&c->d_agg[b], F * L.NS * 4 + 16) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_scratch(c, nullptr);
    set_err("cudaMalloc of %d frames of scratch failed", frames);
    return VC_ERR_OOM;
  }
  c->cap = frames;
  return VC_OK;
}

// Frames per pass for a call of nframes frames.
int pass_frames(const vc_ctx* c, int nframes) {
  if (c->chunk > 0) return nframes < c->chunk ? nframes : c->chunk;
  int f = c->overlap ? (nframes + 5) / 6 : nframes;  // about six passes, so keystream and rounds overlap
  if (f > 64) f = 64;
  if (f < 1) f = 1;
  return nframes < f ? nframes : f;
}

// Pass sizes of a call of nframes frames with passes of at most F frames.  With
// overlap and automatic sizing the last passes shrink by a factor of about
// 3/4 each, down to about F/4: the rounds of the last pass are the only ones
// that no keystream overlaps, while each shrinking pass's rounds still hide
// behind the (serial) keystream of the next one.
void pass_plan(const vc_ctx* c, int nframes, int F, std::vector<int>& plan) {
  plan.clear();
  std::vector<int> tail;  // ascending: tail[0] is the last pass
  if (c->chunk == 0 && c->overlap && F >= 4) {
    for (int t = (F + 3) / 4; t < F; t = (4 * t + 2) / 3) tail.push_back(t);
  }
  long long tsum = 0;
  for (int t : tail) tsum += t;
  while (!tail.empty() && nframes - tsum < F) {  // keep at least one full-size pass ahead of the tail
    tsum -= tail.back();
    tail.pop_back();
  }
  const int body = nframes - (int)tsum;
  const int np = (body + F - 1) / F;
  for (int k = 0; k < np; k++) plan.push_back(body / np + (k < body % np ? 1 : 0));
  for (int k = (int)tail.size() - 1; k >= 0; k--) plan.push_back(tail[k]);
}

cudaEvent_t pool_event(vc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one stage of a pass with events when profiling is on.
struct StageMark {
  vc_ctx* c;
  cudaStream_t st;
  int stage, launches;
  cudaEvent_t a = nullptr;
  StageMark(vc_ctx* c_, cudaStream_t st_, int stage_, int launches_) : c(c_), st(st_), stage(stage_), launches(launches_) {
    if (c->prof) {
      a = pool_event(c);
      cudaEventRecord(a, st);
    }
  }
  ~StageMark() {
    if (a) {
      cudaEvent_t b = pool_event(c);
      cudaEventRecord(b, st);
      c->marks.push_back(vc_ctx::Mark{stage, launches, a, b});
    }
  }
};

// Warps per SM-holding keystream CTA for this context (0: shared SMs).  PLCM
// chains are latency-bound: 4 warps (one per scheduler) per SM when those CTAs
// leave half the SMs to the rounds.  2DLASM chains are bound by the SM's
// binary64 pipe: 2 warps per SM when at least an eighth of the SMs stay free.
int ks_warps_in_use(const vc_ctx* c) {
  if (c->ks_sm_warps >= 0) return c->ks_sm_warps;
  if (!c->overlap) return 0;
  const int lanes = 2 * c->L.n;
  if (c->kind == VC_2DLASM) {  // ~60 binary64 operations per step: four warps per SM saturate the pipe
    const int ctas2 = (lanes + 63) / 64;
    if (ctas2 + (c->num_sms + 7) / 8 <= c->num_sms) return 2;
  }
  const int ctas4 = (lanes + 127) / 128;
  return 2 * ctas4 <= c->num_sms ? 4 : 0;
}

// Keystream side of a pass into buffer b: s_c and shift tables (Alg. 1), then
// r * S_i bytes per subframe and frame (Sec. 3).
int keystream_stage(vc_ctx* c, int b, int nf, cudaStream_t ks) {
  vc::NvtxRange range("vc.keystream");
  const Layout& L = c->L;
  // s_c and the shift tables (which need only PRBG_m) on their own stream,
  // beside the keystream kernel (which needs only the subframe chains): after
  // what `ks` holds so far (buffer reuse, state snapshots), and `ks` waits for
  // them at the end of the stage, so whoever waits for the stage sees both
  // and the next pass's keystream never queues behind a schedule
  cudaStream_t sc = c->sc_stream;
  VC_CUDA(cudaEventRecord(c->ev_sc_in, ks));
  VC_CUDA(cudaStreamWaitEvent(sc, c->ev_sc_in, 0));
  {
    StageMark m(c, sc, 0, 2);
    VC_CUDA(vc::launch_frame_schedule(L, c->d_main, nf, c->d_sc[b], c->d_kmod[b], sc));
  }
  VC_CUDA(cudaEventRecord(c->ev_sc_out, sc));
  {
    StageMark m(c, ks, 1, 1);
    VC_CUDA(c->ks_lanes == 2
                ? vc::launch_keystream(c->kind, L, c->tables(), c->chains(), nf, c->d_ks[b], c->plcm_int, ks, 0, 0,
                                       ks_warps_in_use(c))
                : vc::launch_keystream_thread(c->kind, L, c->tables(), c->chains(), nf, c->d_ks[b], c->plcm_int, ks));
  }
  VC_CUDA(cudaStreamWaitEvent(ks, c->ev_sc_out, 0));
  return VC_OK;
}

// Issues the keystream of the next pass (on ks_stream when overlapping) and
// makes `st` wait for it; returns the buffer index.
int begin_pass(vc_ctx* c, int nf, cudaStream_t st, int* rc) {
  const int b = (int)(c->passes & 1);
  c->passes++;
  if (c->overlap) {
    cudaStream_t ks = c->ks_stream;
    *rc = VC_OK;
    if (cudaStreamWaitEvent(ks, c->ev_rd[b], 0) != cudaSuccess) {
      set_err("cudaStreamWaitEvent failed");
      *rc = VC_ERR_CUDA;
      return b;
    }
    *rc = keystream_stage(c, b, nf, ks);
    if (*rc) return b;
    if (cudaEventRecord(c->ev_ks[b], ks) != cudaSuccess || cudaStreamWaitEvent(st, c->ev_ks[b], 0) != cudaSuccess) {
      set_err("event record/wait failed");
      *rc = VC_ERR_CUDA;
    }
  } else {
    *rc = keystream_stage(c, b, nf, st);
  }
  return b;
}

int end_pass(vc_ctx* c, int b, cudaStream_t st) {
  if (c->overlap) VC_CUDA(cudaEventRecord(c->ev_rd[b], st));
  return VC_OK;
}

// The rounds of one pass over nf frames whose keystream, s_c and shift tables
// are frames f_off .. f_off + nf - 1 of buffer b (encrypt when dir == 0).
// in/out strides in bytes.
int rounds_pass(vc_ctx* c, int dir, const uint8_t* in, long long in_stride, uint8_t* out, long long out_stride,
                int nf, cudaStream_t st, int b, int f_off) {
  vc::NvtxRange range("vc.rounds");
  const Layout& L = c->L;
  const vc::Tables tb = c->tables();
  const long long ks_stride = (long long)L.rounds * L.Npad;
  const uint8_t* ksb = c->d_ks[b] + (long long)f_off * ks_stride;
  const int* kmod = c->d_kmod[b] + (long long)f_off * L.H;
  const int r = L.rounds;
  const bool pc = c->diff_pc;  // per-channel chains (the same kernels, word carries)
  StageMark rounds_mark(c, st, 2, r + (dir == 0 ? 1 : 0));
  // with one round and in == out, the round cannot write its own input: go through a buffer
  const bool bounce = (r == 1) && (in == out);
  uint8_t* final_out = bounce ? c->d_buf[0] : out;
  const long long final_stride = bounce ? L.Npad : out_stride;
  for (int step = 0; step < r; step++) {
    const uint8_t* src = step == 0 ? in : c->d_buf[(step - 1) & 1];
    const long long ss = step == 0 ? in_stride : L.Npad;
    uint8_t* dst = step == r - 1 ? final_out : c->d_buf[step & 1];
    const long long ds = step == r - 1 ? final_stride : L.Npad;
    if (dir == 0) {
      const int j = step;
      VC_CUDA(vc::launch_enc_round(L, tb, src, ss, dst, ds, ksb + (long long)j * L.Npad, ks_stride, kmod,
                                   step == 0 ? nullptr : c->d_agg[(step - 1) & 1], c->d_agg[step & 1], nf, st, pc));
    } else {
      const int j = r - 1 - step;
      VC_CUDA(
          vc::launch_dec_round(L, tb, src, ss, dst, ds, ksb + (long long)j * L.Npad, ks_stride, kmod, nf, st, pc));
    }
  }
  if (dir == 0) VC_CUDA(vc::launch_enc_fixup(L, tb, final_out, final_stride, c->d_agg[(r - 1) & 1], nf, st, pc));
  if (bounce)
    VC_CUDA(cudaMemcpy2DAsync(out, (size_t)out_stride, c->d_buf[0], (size_t)L.Npad, (size_t)L.N, (size_t)nf,
                              cudaMemcpyDeviceToDevice, st));
  return VC_OK;
}

// One pass over nf <= cap frames (encrypt when dir == 0).  in/out strides in bytes.
int run_pass(vc_ctx* c, int dir, const uint8_t* in, long long in_stride, uint8_t* out, long long out_stride, int nf,
             cudaStream_t st) {
  int rc = VC_OK;
  const int b = begin_pass(c, nf, st, &rc);
  if (rc) return rc;
  rc = rounds_pass(c, dir, in, in_stride, out, out_stride, nf, st, b, 0);
  if (rc) return rc;
  return end_pass(c, b, st);
}

// ---- keystream run-ahead across calls ----

// [MainPrbg][chain state][carries][carry lengths], each 256-byte aligned
size_t snap_part(size_t v) { return (v + 255) & ~(size_t)255; }
size_t snap_bytes(const vc_ctx* c) {
  const size_t n = (size_t)c->L.n;
  return snap_part(sizeof(vc::MainPrbg)) + snap_part(n * sizeof(double) * c->state_words()) +
         snap_part(n * 2 * sizeof(uint64_t)) + snap_part(n * sizeof(int));
}

// Copy the chain state to (save) or from (!save) the snapshot, on stream s.
int snap_copy(vc_ctx* c, bool save, cudaStream_t s) {
  const size_t n = (size_t)c->L.n;
  void* live[4] = {c->d_main, c->d_st, c->d_carry, c->d_carry_len};
  const size_t sz[4] = {sizeof(vc::MainPrbg), n * sizeof(double) * c->state_words(), n * 2 * sizeof(uint64_t),
                        n * sizeof(int)};
  uint8_t* p = c->d_snap;
  for (int k = 0; k < 4; k++) {
    VC_CUDA(cudaMemcpyAsync(save ? (void*)p : live[k], save ? live[k] : (const void*)p, sz[k],
                            cudaMemcpyDeviceToDevice, s));
    p += snap_part(sz[k]);
  }
  return VC_OK;
}

// At the end of a call: generate the keystream of the next call's first pass
// (nf frames) on ks_stream, keeping the state from before it.
int spec_issue(vc_ctx* c, int nf) {
  if (!c->overlap || !c->spec_enabled || c->spec_frames > 0 || nf <= 0 || nf > c->cap ||
      c->produced != c->frame)
    return VC_OK;
  if (!c->d_snap) {
    if (dev_alloc(&c->d_snap, snap_bytes(c)) != cudaSuccess) {
      cudaGetLastError();
      c->d_snap = nullptr;
      return VC_OK;  // no run-ahead without room for the snapshot
    }
  }
  const int b = (int)(c->passes & 1);
  cudaStream_t ks = c->ks_stream;
  VC_CUDA(cudaStreamWaitEvent(ks, c->ev_rd[b], 0));
  int rc = snap_copy(c, true, ks);
  if (rc) return rc;
  rc = keystream_stage(c, b, nf, ks);
  if (rc) return rc;
  VC_CUDA(cudaEventRecord(c->ev_ks[b], ks));
  c->passes++;
  c->spec_b = b;
  c->spec_frames = nf;
  c->spec_used = 0;
  return VC_OK;
}

// Rounds of nf (<= the frames left) run-ahead frames.
int spec_pass(vc_ctx* c, int dir, const uint8_t* in, long long in_stride, uint8_t* out, long long out_stride,
              int nf, cudaStream_t st) {
  const int b = c->spec_b;
  VC_CUDA(cudaStreamWaitEvent(st, c->ev_ks[b], 0));
  int rc = rounds_pass(c, dir, in, in_stride, out, out_stride, nf, st, b, c->spec_used);
  if (rc) return rc;
  rc = end_pass(c, b, st);
  if (rc) return rc;
  c->spec_used += nf;
  if (c->spec_used == c->spec_frames) {
    c->spec_frames = c->spec_used = 0;
    c->spec_b = -1;
  }
  return VC_OK;
}

// Undo the run-ahead: the state returns to frame c->frame (the snapshot, then
// the keystream of the frames already taken once more).
int spec_rollback(vc_ctx* c) {
  if (c->spec_frames == 0) return VC_OK;
  cudaStream_t ks = c->ks_stream;
  int rc = snap_copy(c, false, ks);
  if (rc) return rc;
  if (c->spec_used > 0) {
    VC_CUDA(cudaStreamWaitEvent(ks, c->ev_rd[c->spec_b], 0));
    rc = keystream_stage(c, c->spec_b, c->spec_used, ks);
    if (rc) return rc;
  }
  VC_CUDA(cudaStreamSynchronize(ks));
  c->spec_frames = c->spec_used = 0;
  c->spec_b = -1;
  return VC_OK;
}

// Drop the run-ahead whose state is about to be overwritten.
void spec_discard(vc_ctx* c) {
  if (c->spec_frames == 0) return;
  cudaStreamSynchronize(c->ks_stream);
  c->spec_frames = c->spec_used = 0;
  c->spec_b = -1;
}

// Pass sizes of a call: first the run-ahead frames still held (first_spec),
// then the plan of the rest.  *next_first: the first pass of a call of the same
// size, the run-ahead to issue at its end.
void call_plan(const vc_ctx* c, int nframes, int F, std::vector<int>& plan, bool* first_spec, int* next_first) {
  plan.clear();
  *first_spec = false;
  int rest = nframes;
  if (c->spec_frames > c->spec_used) {
    const int k = std::min(c->spec_frames - c->spec_used, nframes);
    plan.push_back(k);
    *first_spec = true;
    rest -= k;
  }
  std::vector<int> tail;
  if (rest > 0) {
    pass_plan(c, rest, F, tail);
    plan.insert(plan.end(), tail.begin(), tail.end());
  }
  std::vector<int> full;
  pass_plan(c, nframes, F, full);
  *next_first = full.empty() ? 0 : full[0];
}

// Single-stream calls generate the keystream inline: not while a batcher holds
// keystream produced ahead for this context.
int check_no_runahead(vc_ctx* c) {
  if (c->produced != c->frame) {
    set_err("a batcher holds %lld frames of keystream produced ahead for this stream; keep using the batcher",
            (long long)(c->produced - c->frame));
    return VC_ERR_SEQUENCE;
  }
  return VC_OK;
}

int enter(vc_ctx* c, cudaStream_t st) {
  int rg = check_no_runahead(c);
  if (rg) return rg;
  if (c->batch_pending) {  // a batch on another stream advanced this context last
    VC_CUDA(cudaStreamWaitEvent(st, c->ev_batch, 0));
    c->batch_pending = false;
  }
  c->last = st;
  if (c->overlap) {
    // the keystream side starts after what the caller enqueued before this call
    VC_CUDA(cudaEventRecord(c->ev_entry, st));
    VC_CUDA(cudaStreamWaitEvent(c->ks_stream, c->ev_entry, 0));
  }
  return VC_OK;
}

// pitch: bytes from one frame to the next in d_in and d_out (>= N).
int crypt_device(vc_ctx* c, int dir, const uint8_t* d_in, uint8_t* d_out, int nframes, void* stream,
                 long long pitch) {
  if (!c || nframes < 0 || (nframes > 0 && (!d_in || !d_out)) || pitch < c->L.N) {
    set_err("invalid argument");
    return VC_ERR_ARG;
  }
  if (nframes == 0) return VC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int F = pass_frames(c, nframes);
  int rc = ensure_scratch(c, F);
  if (rc) return rc;
  rc = enter(c, st);
  if (rc) return rc;
  const long long N = pitch;
  std::vector<int> plan;
  bool first_spec = false;
  int next_first = 0;
  call_plan(c, nframes, F, plan, &first_spec, &next_first);
  long long f0 = 0;
  for (size_t k = 0; k < plan.size(); k++) {
    const int nf = plan[k];
    rc = (k == 0 && first_spec) ? spec_pass(c, dir, d_in + f0 * N, N, d_out + f0 * N, N, nf, st)
                                : run_pass(c, dir, d_in + f0 * N, N, d_out + f0 * N, N, nf, st);
    if (rc) return rc;
    f0 += nf;
  }
  c->frame += nframes;
  c->produced = c->frame;
  c->produced_done = c->frame;
  return spec_issue(c, next_first);
}

}  // namespace

extern "C" {

const char* vc_strerror(int code) {
  switch (code) {
    case VC_OK: return "ok";
    case VC_ERR_ARG: return "invalid argument";
    case VC_ERR_KEY_RANGE: return "key outside the valid ranges of the chaotic map";
    case VC_ERR_LAYOUT: return "invalid frame layout or subframe count";
    case VC_ERR_CUDA: return "CUDA error";
    case VC_ERR_OOM: return "out of memory";
    case VC_ERR_TIMEOUT: return "device wait timed out";
    case VC_ERR_SEQUENCE: return "frame out of sequence";
    case VC_ERR_STATE: return "malformed state checkpoint";
    case VC_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* vc_last_error(void) { return g_err; }

int enc_init(const vc_key* key, const vc_layout* layout, vc_ctx** out) {
  if (!key || !layout || !out) {
    set_err("null argument");
    return VC_ERR_ARG;
  }
  *out = nullptr;
  if (!key_valid(*key)) {
    set_err("key outside the valid ranges");
    return VC_ERR_KEY_RANGE;
  }
  Layout L{};
  int rc = make_layout(*layout, &L);
  if (rc) {
    set_err("invalid layout");
    return rc;
  }
  vc_ctx* c = new (std::nothrow) vc_ctx();
  if (!c) return VC_ERR_OOM;
  c->kind = key->kind;
  c->L = L;
  c->user_layout = *layout;
  cudaGetDevice(&c->dev);
  const int n = L.n;
  const int nwords = L.P / 32 + 2;
  bool ok = dev_alloc(&c->d_pi, sizeof(int) * (n + 1)) == cudaSuccess &&
            dev_alloc(&c->d_sbits, sizeof(uint32_t) * nwords) == cudaSuccess &&
            dev_alloc(&c->d_srank, sizeof(int) * nwords) == cudaSuccess &&
            dev_alloc(&c->d_fixlim, sizeof(int) * L.NS) == cudaSuccess &&
            dev_alloc(&c->d_main, sizeof(vc::MainPrbg)) == cudaSuccess &&
            dev_alloc(&c->d_st, sizeof(double) * c->state_words() * n) == cudaSuccess &&
            dev_alloc(&c->d_par, sizeof(double) * c->par_words() * n) == cudaSuccess &&
            dev_alloc(&c->d_carry, sizeof(uint64_t) * 2 * n) == cudaSuccess &&
            dev_alloc(&c->d_carry_len, sizeof(int) * n) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    enc_destroy(c);
    set_err("device allocation failed");
    return VC_ERR_OOM;
  }
  if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->d2h_stream, cudaStreamNonBlocking) != cudaSuccess) {
    enc_destroy(c);
    set_err("stream creation failed");
    return VC_ERR_CUDA;
  }
  for (auto& e : c->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  for (auto& e : c->ev_io) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev);
  if (cudaStreamCreateWithPriority(&c->ks_stream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->sc_stream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_sc_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_sc_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_ks[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_ks[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_rd[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_rd[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_entry, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_batch, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_free, cudaEventDisableTiming) != cudaSuccess ||
      !std::all_of(std::begin(c->ev_prod), std::end(c->ev_prod), [](cudaEvent_t& e) {
        return cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
      })) {
    enc_destroy(c);
    set_err("stream/event creation failed");
    return VC_ERR_CUDA;
  }
  vc::MainPrbg m{};
  m.kind = key->kind;
  if (key->kind == VC_PLCM || key->kind == VC_LOGISTIC) {
    for (int i = 0; i < 4; i++) m.s[i] = key->k[i];
  } else {  // K = (x0, mu, y0) -> state (x, y, mu)
    m.s[0] = key->k[0];
    m.s[1] = key->k[2];
    m.s[2] = key->k[1];
  }
  cudaStream_t st = c->copy_stream;
  cudaError_t e = cudaMemcpyAsync(c->d_main, &m, sizeof(m), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = vc::launch_build_tables(L, c->d_pi, c->d_sbits, c->d_srank, c->d_fixlim, st);
  if (e == cudaSuccess) e = vc::launch_key_schedule(c->kind, c->d_main, c->chains(), n, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_err("key schedule failed: %s", cudaGetErrorString(e));
    enc_destroy(c);
    return VC_ERR_CUDA;
  }
  *out = c;
  return VC_OK;
}

int encrypt_frames(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, void* stream) {
  return crypt_device(ctx, 0, d_in, d_out, nframes, stream, ctx ? ctx->L.N : 0);
}

int decrypt_frames(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, void* stream) {
  return crypt_device(ctx, 1, d_in, d_out, nframes, stream, ctx ? ctx->L.N : 0);
}

int encrypt_frames_pitched(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, size_t frame_pitch,
                           void* stream) {
  if (!ctx) return VC_ERR_ARG;
  const long long pitch = frame_pitch == 0 ? ctx->L.N : (frame_pitch > ((size_t)1 << 40) ? -1 : (long long)frame_pitch);
  return crypt_device(ctx, 0, d_in, d_out, nframes, stream, pitch);
}

int decrypt_frames_pitched(vc_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, size_t frame_pitch,
                           void* stream) {
  if (!ctx) return VC_ERR_ARG;
  const long long pitch = frame_pitch == 0 ? ctx->L.N : (frame_pitch > ((size_t)1 << 40) ? -1 : (long long)frame_pitch);
  return crypt_device(ctx, 1, d_in, d_out, nframes, stream, pitch);
}

// Host staging buffers for passes of up to `frames` frames.
int ensure_io(vc_ctx* c, int frames) {
  if (c->io_cap >= frames) return VC_OK;
  cudaStream_t after = ctx_join(c);
  for (auto& b : c->d_io) {
    dev_free(b, after);
    b = nullptr;
  }
  c->io_cap = 0;
  const size_t N = (size_t)c->L.N;
  for (auto& b : c->d_io) {
    if (dev_alloc(&b, (size_t)frames * N) != cudaSuccess) {
      cudaGetLastError();
      set_err("staging allocation failed");
      return VC_ERR_OOM;
    }
  }
  c->io_cap = frames;
  return VC_OK;
}

namespace {

// The host-buffer path: wait = the call returns once h_out holds the result;
// otherwise `done` (if any) is recorded after the call's last download.
int crypt_host(vc_ctx* c, int32_t direction, const uint8_t* h_in, uint8_t* h_out, int32_t nframes, void* stream,
               bool wait, cudaEvent_t done_ev) {
  if (!c || nframes < 0 || (direction != 0 && direction != 1) || (nframes > 0 && (!h_in || !h_out))) {
    set_err("invalid argument");
    return VC_ERR_ARG;
  }
  if (nframes == 0) return VC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int F = pass_frames(c, nframes);
  int rc = ensure_scratch(c, F);
  if (rc) return rc;
  rc = enter(c, st);
  if (rc) return rc;
  const size_t N = (size_t)c->L.N;
  std::vector<int> plan;
  bool first_spec = false;
  int next_first = 0;
  call_plan(c, nframes, F, plan, &first_spec, &next_first);
  rc = ensure_io(c, std::max(F, plan[0]));  // a run-ahead pass can be larger than this call's passes
  if (rc) return rc;
  // Three streams and three staging buffers: uploads (copy_stream), passes
  // (st, in place in the buffer) and downloads (d2h_stream) of consecutive
  // passes overlap, also across calls; a buffer is uploaded again once its
  // previous download is done.
  constexpr int kIo = vc_ctx::kIoBufs;
  cudaEvent_t* up = c->ev_io;             // upload into buffer b done
  cudaEvent_t* done = c->ev_io + kIo;     // pass in buffer b done
  cudaEvent_t* down = c->ev_io + 2 * kIo; // download from buffer b done
  long long f0 = 0;
  int b = 0;
  for (int k = 0; k < (int)plan.size(); f0 += plan[k], k++) {
    const int nf = plan[k];
    b = (int)(c->io_uses % kIo);
    uint8_t* buf = c->d_io[b];
    if (c->io_uses >= kIo) VC_CUDA(cudaStreamWaitEvent(c->copy_stream, down[b], 0));
    c->io_uses++;
    VC_CUDA(cudaMemcpyAsync(buf, h_in + (size_t)f0 * N, nf * N, cudaMemcpyHostToDevice, c->copy_stream));
    VC_CUDA(cudaEventRecord(up[b], c->copy_stream));
    VC_CUDA(cudaStreamWaitEvent(st, up[b], 0));
    rc = (k == 0 && first_spec) ? spec_pass(c, direction, buf, (long long)N, buf, (long long)N, nf, st)
                                : run_pass(c, direction, buf, (long long)N, buf, (long long)N, nf, st);
    if (rc) return rc;
    VC_CUDA(cudaEventRecord(done[b], st));
    VC_CUDA(cudaStreamWaitEvent(c->d2h_stream, done[b], 0));
    VC_CUDA(cudaMemcpyAsync(h_out + (size_t)f0 * N, buf, nf * N, cudaMemcpyDeviceToHost, c->d2h_stream));
    VC_CUDA(cudaEventRecord(down[b], c->d2h_stream));
  }
  c->frame += nframes;
  c->produced = c->frame;
  c->produced_done = c->frame;
  rc = spec_issue(c, next_first);
  if (rc) return rc;
  if (!wait) {
    if (done_ev) VC_CUDA(cudaEventRecord(done_ev, c->d2h_stream));  // after the call's last download
    return VC_OK;
  }
  VC_CUDA(cudaStreamSynchronize(c->d2h_stream));
  VC_CUDA(cudaStreamSynchronize(c->copy_stream));
  VC_CUDA(cudaStreamSynchronize(st));
  return VC_OK;
}

}  // namespace

int crypt_frames_host(vc_ctx* c, int32_t direction, const uint8_t* h_in, uint8_t* h_out, int32_t nframes,
                      void* stream) {
  return crypt_host(c, direction, h_in, h_out, nframes, stream, true, nullptr);
}

int crypt_frames_host_async(vc_ctx* c, int32_t direction, const uint8_t* h_in, uint8_t* h_out, int32_t nframes,
                            void* stream, void* done_event) {
  return crypt_host(c, direction, h_in, h_out, nframes, stream, false, (cudaEvent_t)done_event);
}

namespace {
struct StateHeader {
  uint32_t magic, version;
  int32_t kind, H, W, C, n, rounds;
  int64_t frame;
};
}  // namespace

size_t enc_state_size(const vc_ctx* c) {
  if (!c) return 0;
  const size_t n = (size_t)c->L.n;
  return sizeof(StateHeader) + sizeof(vc::MainPrbg) + n * sizeof(double) * (c->state_words() + c->par_words()) +
         n * 2 * sizeof(uint64_t) + n * sizeof(int);
}

int enc_save_state(vc_ctx* c, void* buf, size_t* len) {
  if (!c || !buf || !len || *len < enc_state_size(c)) {
    set_err("invalid argument");
    return VC_ERR_ARG;
  }
  if (int rg = check_no_runahead(c)) return rg;
  if (int rs = spec_rollback(c)) return rs;
  sync_all(c);
  VC_CUDA(cudaGetLastError());
  const size_t n = (size_t)c->L.n;
  uint8_t* p = static_cast<uint8_t*>(buf);
  StateHeader h{kStateMagic, kStateVersion, c->kind, c->L.H, c->L.W, c->L.C, c->L.n, c->L.rounds, c->frame};
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  VC_CUDA(cudaMemcpy(p, c->d_main, sizeof(vc::MainPrbg), cudaMemcpyDeviceToHost));
  p += sizeof(vc::MainPrbg);
  VC_CUDA(cudaMemcpy(p, c->d_st, n * sizeof(double) * c->state_words(), cudaMemcpyDeviceToHost));
  p += n * sizeof(double) * c->state_words();
  VC_CUDA(cudaMemcpy(p, c->d_par, n * sizeof(double) * c->par_words(), cudaMemcpyDeviceToHost));
  p += n * sizeof(double) * c->par_words();
  VC_CUDA(cudaMemcpy(p, c->d_carry, n * 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  p += n * 2 * sizeof(uint64_t);
  VC_CUDA(cudaMemcpy(p, c->d_carry_len, n * sizeof(int), cudaMemcpyDeviceToHost));
  *len = enc_state_size(c);
  return VC_OK;
}

int enc_load_state(vc_ctx* c, const void* buf, size_t len) {
  if (!c || !buf) {
    set_err("invalid argument");
    return VC_ERR_ARG;
  }
  if (len != enc_state_size(c)) {
    set_err("checkpoint size %zu does not match %zu", len, enc_state_size(c));
    return VC_ERR_STATE;
  }
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.version != kStateVersion || h.kind != c->kind || h.H != c->L.H ||
      h.W != c->L.W || h.C != c->L.C || h.n != c->L.n || h.rounds != c->L.rounds || h.frame < 0) {
    set_err("checkpoint header does not match this context");
    return VC_ERR_STATE;
  }
  sync_all(c);
  spec_discard(c);
  const size_t n = (size_t)c->L.n;
  const uint8_t* p = static_cast<const uint8_t*>(buf) + sizeof(h);
  VC_CUDA(cudaMemcpy(c->d_main, p, sizeof(vc::MainPrbg), cudaMemcpyHostToDevice));
  p += sizeof(vc::MainPrbg);
  VC_CUDA(cudaMemcpy(c->d_st, p, n * sizeof(double) * c->state_words(), cudaMemcpyHostToDevice));
  p += n * sizeof(double) * c->state_words();
  VC_CUDA(cudaMemcpy(c->d_par, p, n * sizeof(double) * c->par_words(), cudaMemcpyHostToDevice));
  p += n * sizeof(double) * c->par_words();
  VC_CUDA(cudaMemcpy(c->d_carry, p, n * 2 * sizeof(uint64_t), cudaMemcpyHostToDevice));
  p += n * 2 * sizeof(uint64_t);
  VC_CUDA(cudaMemcpy(c->d_carry_len, p, n * sizeof(int), cudaMemcpyHostToDevice));
  c->frame = h.frame;
  c->produced = h.frame;
  c->produced_done = h.frame;
  return VC_OK;
}

int64_t enc_frame_index(const vc_ctx* c) { return c ? c->frame : -1; }

int enc_sync_status(vc_ctx* c) {
  if (!c) return VC_ERR_ARG;
  cudaError_t e = c->last ? cudaStreamSynchronize(c->last) : cudaSuccess;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy_stream);
  if (e == cudaSuccess && c->d2h_stream) e = cudaStreamSynchronize(c->d2h_stream);
  if (e == cudaSuccess && c->ks_stream) e = cudaStreamSynchronize(c->ks_stream);
  if (e == cudaSuccess && c->prod_stream) e = cudaStreamSynchronize(c->prod_stream);
  if (e == cudaSuccess && c->prod_urgent) e = cudaStreamSynchronize(c->prod_urgent);
  if (e == cudaSuccess && c->sc_stream) e = cudaStreamSynchronize(c->sc_stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err("asynchronous CUDA error: %s", cudaGetErrorString(e));
    return VC_ERR_CUDA;
  }
  return VC_OK;
}

int enc_join(vc_ctx* c, void* stream) {
  if (!c) return VC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  for (cudaStream_t o : {c->ks_stream, c->prod_stream, c->prod_urgent, c->sc_stream, c->copy_stream, c->d2h_stream})
    if (o && o != st) {
      VC_CUDA(cudaEventRecord(c->ev_free, o));
      VC_CUDA(cudaStreamWaitEvent(st, c->ev_free, 0));
    }
  return VC_OK;
}

int enc_set_chunk(vc_ctx* c, int32_t frames_per_pass) {
  if (!c || frames_per_pass < 1 || frames_per_pass > 65535) return VC_ERR_ARG;
  c->chunk = frames_per_pass;
  return VC_OK;
}

int enc_profile_enable(vc_ctx* c, int32_t enable) {
  if (!c) return VC_ERR_ARG;
  c->prof = enable != 0;
  return VC_OK;
}

int enc_profile_read(vc_ctx* c, double* ms3, int64_t* launches3) {
  if (!c || !ms3 || !launches3) return VC_ERR_ARG;
  for (int i = 0; i < 3; i++) {
    ms3[i] = 0.0;
    launches3[i] = 0;
  }
  for (auto& m : c->marks) {
    VC_CUDA(cudaEventSynchronize(m.b));
    float ms = 0.f;
    VC_CUDA(cudaEventElapsedTime(&ms, m.a, m.b));
    ms3[m.stage] += ms;
    launches3[m.stage] += m.launches;
    c->pool.push_back(m.a);
    c->pool.push_back(m.b);
  }
  c->marks.clear();
  return VC_OK;
}

int enc_set_option(vc_ctx* c, int32_t option, int64_t value) {
  if (!c) return VC_ERR_ARG;
  switch (option) {
    case VC_OPT_CHUNK:
      if (value == 0) {
        c->chunk = 0;
        return VC_OK;
      }
      return enc_set_chunk(c, value < 1 || value > 65535 ? -1 : (int32_t)value);
    case VC_OPT_PLCM_INT:
      if (value < 0 || value > 3) return VC_ERR_ARG;
      c->plcm_int = (int)value;
      return VC_OK;
    case VC_OPT_KS_LANES:
      if (value != 1 && value != 2) return VC_ERR_ARG;
      c->ks_lanes = (int)value;
      return VC_OK;
    case VC_OPT_OVERLAP: {
      if (value != 0 && value != 1) return VC_ERR_ARG;
      int rs = spec_rollback(c);
      if (rs) return rs;
      sync_all(c);
      c->overlap = value != 0;
      return VC_OK;
    }
    case VC_OPT_DIFFUSION:
      if (value != 0 && value != 1) return VC_ERR_ARG;
      if (value == 1 && c->L.P / c->L.n < 2) {
        set_err("per-channel diffusion needs at least 2 pixels in every subframe");
        return VC_ERR_LAYOUT;
      }
      if (value == 1 && !pc_smem_fits(c)) {
        set_err("per-channel diffusion of this layout needs %zu bytes of shared memory per round CTA",
                vc::round_smem_bytes(c->L, true));
        return VC_ERR_LAYOUT;
      }
      c->diff_pc = value == 1;
      return VC_OK;
    case VC_OPT_RUNAHEAD_CALLS: {
      if (value != 0 && value != 1) return VC_ERR_ARG;
      if (value == 0) {
        int rs = spec_rollback(c);
        if (rs) return rs;
      }
      c->spec_enabled = value != 0;
      return VC_OK;
    }
    case VC_OPT_KS_SM_WARPS: {
      if (value < -1 || value > 4) return VC_ERR_ARG;
      sync_all(c);
      int least = 0, greatest = 0;
      VC_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      cudaStream_t s2 = nullptr;
      VC_CUDA(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, value != 0 ? greatest : least));
      cudaStreamDestroy(c->ks_stream);
      c->ks_stream = s2;
      c->ks_sm_warps = (int)value;
      return VC_OK;
    }
    case VC_OPT_TILE_ROWS: {
      if (value != 0 && (value < 1 || value > 32 || (value & (value - 1)))) return VC_ERR_ARG;
      Layout L2{};
      if (make_layout(c->user_layout, &L2, (int)value) != VC_OK) return VC_ERR_ARG;
      if (c->diff_pc && !pc_smem_fits(c, &L2)) {
        set_err("per-channel diffusion with %d tile rows needs %zu bytes of shared memory per round CTA", (int)value,
                vc::round_smem_bytes(L2, true));
        return VC_ERR_LAYOUT;
      }
      int rs = spec_rollback(c);
      if (rs) return rs;
      sync_all(c);
      int* fl = nullptr;
      if (dev_alloc(&fl, sizeof(int) * L2.NS) != cudaSuccess) {
        cudaGetLastError();
        set_err("tile table allocation failed");
        return VC_ERR_OOM;
      }
      // the partition tables other than the tile limits do not depend on the tile shape
      VC_CUDA(vc::launch_build_tables(L2, c->d_pi, c->d_sbits, c->d_srank, fl, c->copy_stream));
      VC_CUDA(cudaStreamSynchronize(c->copy_stream));
      dev_free(c->d_fixlim, nullptr);  // the context's streams are idle
      c->d_fixlim = fl;
      free_scratch(c, nullptr);
      c->L = L2;
      c->tile_rows = (int)value;
      return VC_OK;
    }
  }
  set_err("unknown option %d", option);
  return VC_ERR_ARG;
}

int enc_get_option(const vc_ctx* c, int32_t option, int64_t* value) {
  if (!c || !value) return VC_ERR_ARG;
  switch (option) {
    case VC_OPT_CHUNK: *value = c->chunk; return VC_OK;
    case VC_OPT_PLCM_INT: *value = c->plcm_int; return VC_OK;
    case VC_OPT_KS_LANES: *value = c->ks_lanes; return VC_OK;
    case VC_OPT_OVERLAP: *value = c->overlap ? 1 : 0; return VC_OK;
    case VC_OPT_TILE_ROWS: *value = c->L.T; return VC_OK;
    case VC_OPT_KS_SM_WARPS: *value = c->ks_sm_warps; return VC_OK;
    case VC_OPT_RUNAHEAD_CALLS: *value = c->spec_enabled ? 1 : 0; return VC_OK;
    case VC_OPT_DIFFUSION: *value = c->diff_pc ? 1 : 0; return VC_OK;
  }
  return VC_ERR_ARG;
}

namespace {

// Releases the context; wait: first wait for its work (enc_destroy), else
// give its memory back in stream order after that work (enc_destroy_async).
void destroy_ctx(vc_ctx* c, bool wait) {
  if (!c) return;
  if (wait) sync_all(c);
  cudaStream_t after = ctx_join(c);
  if (wait) after = nullptr;
  free_scratch(c, after);
  for (auto b : c->d_io) dev_free(b, after);
  for (void* b : {(void*)c->d_pi, (void*)c->d_sbits, (void*)c->d_srank, (void*)c->d_fixlim, (void*)c->d_main,
                  (void*)c->d_st, (void*)c->d_par, (void*)c->d_carry, (void*)c->d_carry_len, (void*)c->ring_ks,
                  (void*)c->ring_sc, (void*)c->ring_kmod, (void*)c->d_snap})
    dev_free(b, after);
  // events and streams: their resources are released once pending work is done
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->ev_io)
    if (e) cudaEventDestroy(e);
  for (auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->d2h_stream) cudaStreamDestroy(c->d2h_stream);
  if (c->ks_stream) cudaStreamDestroy(c->ks_stream);
  if (c->prod_stream) cudaStreamDestroy(c->prod_stream);
  if (c->prod_urgent) cudaStreamDestroy(c->prod_urgent);
  if (c->sc_stream) cudaStreamDestroy(c->sc_stream);
  for (int b = 0; b < 2; b++) {
    if (c->ev_ks[b]) cudaEventDestroy(c->ev_ks[b]);
    if (c->ev_rd[b]) cudaEventDestroy(c->ev_rd[b]);
  }
  for (cudaEvent_t e : {c->ev_entry, c->ev_batch, c->ev_free, c->ev_sc_in, c->ev_sc_out})
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_slot) cudaEventDestroy(e);
  for (int i = 0; i < vc_ctx::kProdEv; i++)
    if (c->ev_prod[i]) cudaEventDestroy(c->ev_prod[i]);
  delete c;
}

}  // namespace

void enc_destroy(vc_ctx* c) { destroy_ctx(c, true); }

void enc_destroy_async(vc_ctx* c) { destroy_ctx(c, false); }

// ---- diagnostics (include/vcrypt_debug.h) ----

int vc_dbg_csin(const double* d_t, double* d_out, int64_t n, int32_t variant, void* stream) {
  if (n < 0 || (n > 0 && (!d_t || !d_out)) || variant < 0 || variant > 1) return VC_ERR_ARG;
  VC_CUDA(vc::launch_dbg_csin(d_t, d_out, n, variant, (cudaStream_t)stream));
  return VC_OK;
}

int vc_dbg_plcm(const double* d_x, const double* d_p, double* d_out, int64_t n, int32_t variant, void* stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_p || !d_out)) || variant < 0 || variant > 1) return VC_ERR_ARG;
  VC_CUDA(vc::launch_dbg_plcm(d_x, d_p, d_out, n, variant, (cudaStream_t)stream));
  return VC_OK;
}

int vc_dbg_lasm(const double* d_xymu, double* d_out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!d_xymu || !d_out))) return VC_ERR_ARG;
  VC_CUDA(vc::launch_dbg_lasm(d_xymu, d_out, n, (cudaStream_t)stream));
  return VC_OK;
}

int vc_dbg_keystream(vc_ctx* c, uint8_t* d_ks, int64_t* d_sc, int32_t nframes, void* stream) {
  if (!c || nframes < 0 || (nframes > 0 && (!d_ks || !d_sc))) return VC_ERR_ARG;
  if (nframes == 0) return VC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout& L = c->L;
  const int F = pass_frames(c, nframes);
  int rc = spec_rollback(c);
  if (rc) return rc;
  rc = ensure_scratch(c, F);
  if (rc) return rc;
  rc = enter(c, st);
  if (rc) return rc;
  for (int f0 = 0; f0 < nframes; f0 += F) {
    const int nf = (nframes - f0) < F ? (nframes - f0) : F;
    const int b = begin_pass(c, nf, st, &rc);
    if (rc) return rc;
    VC_CUDA(cudaMemcpy2DAsync(d_ks + (size_t)f0 * L.rounds * L.N, (size_t)L.N, c->d_ks[b], (size_t)L.Npad,
                              (size_t)L.N, (size_t)nf * L.rounds, cudaMemcpyDeviceToDevice, st));
    VC_CUDA(cudaMemcpyAsync(d_sc + f0, c->d_sc[b], nf * sizeof(long long), cudaMemcpyDeviceToDevice, st));
    rc = end_pass(c, b, st);
    if (rc) return rc;
  }
  c->frame += nframes;
  c->produced = c->frame;
  c->produced_done = c->frame;
  return VC_OK;
}

int vc_dbg_call_plan(const vc_ctx* c, int32_t nframes, int32_t* plan, int32_t cap, int32_t* info4) {
  if (!c || nframes < 1 || !info4 || cap < 0 || (cap > 0 && !plan)) return VC_ERR_ARG;
  std::vector<int> p;
  bool first_spec = false;
  int next_first = 0;
  call_plan(c, nframes, pass_frames(c, nframes), p, &first_spec, &next_first);
  for (int k = 0; k < (int)p.size() && k < cap; k++) plan[k] = p[k];
  info4[0] = (int32_t)p.size();
  info4[1] = first_spec ? 1 : 0;
  info4[2] = (c->overlap && c->spec_enabled) ? next_first : 0;
  info4[3] = ks_warps_in_use(c);
  return VC_OK;
}

int vc_dbg_layout(const vc_ctx* c, int32_t* out8) {
  if (!c || !out8) return VC_ERR_ARG;
  out8[0] = c->L.T;
  out8[1] = c->L.NT;
  out8[2] = (int32_t)c->L.Npad;
  out8[3] = c->L.N;
  out8[4] = c->L.P;
  out8[5] = c->cap;
  out8[6] = c->chunk > 0 ? c->chunk : pass_frames(c, 1 << 20);
  out8[7] = (int32_t)vc::round_smem_bytes(c->L, c->diff_pc);
  return VC_OK;
}

}  // extern "C"

// =============================================================================
// encrypt_frames_static: encryption without any device allocation in the call.
//
// The per-pass scratch (keystream, shift tables, s_c, the two round buffers
// and the tile aggregates) comes from one file-scope device array instead of
// cudaMalloc.  Host code cannot use the array's name as a device address, so
// the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
// =============================================================================

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB, held by every device that loads the library
constexpr int kStaticMaxDevices = 64;

}  // namespace

static __device__ __align__(256) uint8_t g_vc_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};

int static_scratch_address(void** out) {
  int dev = 0;
  VC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) {
    set_err("device %d beyond the %d devices the static scratch supports", dev, kStaticMaxDevices);
    return VC_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vc_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_err("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      return VC_ERR_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return VC_OK;
}

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// Static-scratch bytes one frame of a pass needs.
size_t static_bytes_per_frame(const Layout& L) {
  return round256((size_t)L.rounds * L.Npad) + 2 * round256((size_t)L.Npad) + round256((size_t)L.H * sizeof(int)) +
         round256(sizeof(long long)) + 2 * round256((size_t)L.NS);
}

}  // namespace

extern "C" int encrypt_frames_static(vc_ctx* c, const uint8_t* d_in, uint8_t* d_out, int32_t nframes, void* stream) {
  if (!c || nframes < 0 || (nframes > 0 && (!d_in || !d_out))) {
    set_err("invalid argument");
    return VC_ERR_ARG;
  }
  if (c->diff_pc) {
    set_err("per-channel diffusion runs through encrypt_frames / decrypt_frames only");
    return VC_ERR_UNSUPPORTED;
  }
  const Layout& L = c->L;
  const size_t per_frame = static_bytes_per_frame(L);
  if (per_frame > kStaticScratchBytes) {
    set_err("encrypt_frames_static: one %dx%dx%d frame with %d rounds needs %zu bytes of scratch, the static "
            "scratch holds %zu",
            L.H, L.W, L.C, L.rounds, per_frame, kStaticScratchBytes);
    return VC_ERR_UNSUPPORTED;
  }
  if (nframes == 0) return VC_OK;
  int rc = check_no_runahead(c);
  if (rc) return rc;
  rc = spec_rollback(c);  // keystream this context generated ahead for its next call
  if (rc) return rc;
  void* base = nullptr;
  rc = static_scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->batch_pending) {
    VC_CUDA(cudaStreamWaitEvent(st, c->ev_batch, 0));
    c->batch_pending = false;
  }
  // keystream work of earlier overlapped calls (internal stream) comes first
  VC_CUDA(cudaEventRecord(c->ev_entry, c->ks_stream));
  VC_CUDA(cudaStreamWaitEvent(st, c->ev_entry, 0));
  c->last = st;

  const int F = (int)(kStaticScratchBytes / per_frame);
  const vc::Tables tb = c->tables();
  const long long ks_stride = (long long)L.rounds * L.Npad;
  const int r = L.rounds;
  const long long N = L.N;
  for (int f0 = 0; f0 < nframes; f0 += F) {
    const int nf = (nframes - f0) < F ? (nframes - f0) : F;
    uint8_t* p = static_cast<uint8_t*>(base);
    uint8_t* ks = p;
    p += round256((size_t)nf * L.rounds * L.Npad);
    uint8_t* buf[2];
    buf[0] = p;
    p += round256((size_t)nf * L.Npad);
    buf[1] = p;
    p += round256((size_t)nf * L.Npad);
    int* kmod = reinterpret_cast<int*>(p);
    p += round256((size_t)nf * L.H * sizeof(int));
    long long* sc = reinterpret_cast<long long*>(p);
    p += round256((size_t)nf * sizeof(long long));
    uint8_t* agg[2];
    agg[0] = p;
    p += round256((size_t)nf * L.NS);
    agg[1] = p;

    const uint8_t* in = d_in + f0 * N;
    uint8_t* out = d_out + f0 * N;
    VC_CUDA(vc::launch_frame_schedule(L, c->d_main, nf, sc, kmod, st));
    VC_CUDA(c->ks_lanes == 2 ? vc::launch_keystream(c->kind, L, tb, c->chains(), nf, ks, c->plcm_int, st)
                             : vc::launch_keystream_thread(c->kind, L, tb, c->chains(), nf, ks, c->plcm_int, st));
    const bool bounce = (r == 1) && (in == out);
    uint8_t* final_out = bounce ? buf[0] : out;
    const long long final_stride = bounce ? L.Npad : N;
    for (int j = 0; j < r; j++) {
      const uint8_t* src = j == 0 ? in : buf[(j - 1) & 1];
      const long long ss = j == 0 ? N : L.Npad;
      uint8_t* dst = j == r - 1 ? final_out : buf[j & 1];
      const long long ds = j == r - 1 ? final_stride : L.Npad;
      VC_CUDA(vc::launch_enc_round(L, tb, src, ss, dst, ds, ks + (long long)j * L.Npad, ks_stride, kmod,
                                   j == 0 ? nullptr : agg[(j - 1) & 1], agg[j & 1], nf, st));
    }
    VC_CUDA(vc::launch_enc_fixup(L, tb, final_out, final_stride, agg[(r - 1) & 1], nf, st));
    if (bounce)
      VC_CUDA(cudaMemcpy2DAsync(out, (size_t)N, buf[0], (size_t)L.Npad, (size_t)L.N, (size_t)nf,
                                cudaMemcpyDeviceToDevice, st));
  }
  // later overlapped calls start their keystream after this call's
  VC_CUDA(cudaEventRecord(c->ev_entry, st));
  VC_CUDA(cudaStreamWaitEvent(c->ks_stream, c->ev_entry, 0));
  c->frame += nframes;
  c->produced = c->frame;
  c->produced_done = c->frame;
  return VC_OK;
}

// =============================================================================
// Ragged batches
// =============================================================================

namespace {

// The launch lane of a batcher: device descriptors, pinned staging (two
// alternating buffers) and the graphs captured for it.
struct BatchLane {
  vc::JobDesc* d_jobs = nullptr;
  vc::BatchHdr* d_hdr = nullptr;
  int jobs_cap = 0;
  vc::JobDesc* h_jobs[2] = {nullptr, nullptr};
  vc::BatchHdr* h_hdr[2] = {nullptr, nullptr};
  cudaEvent_t staged[2] = {nullptr, nullptr};
  int cur = 0;
  std::map<std::tuple<int, int, int, int, int, size_t, int, int>, cudaGraphExec_t> graphs;
  std::vector<void*> retired_host;  // outgrown pinned staging, freed with the lane (its copies may be in flight)
};

}  // namespace

struct vc_batcher {
  int dev = 0, sms = 0;
  BatchLane cons;
  uint8_t* d_pool = nullptr;
  size_t pool_cap = 0;
  bool use_graph = true;
  int ctas_per_sm = 0;
  int runahead = 0;  // frames of keystream kept ahead per stream (0 = off)
  int sine = -1;     // 2DLASM sine reduction in the batch keystream: -1 by load, 0 integer-assisted, 1 binary64
  int split = -1;    // long-chain lane: -1 automatic, 0 never, 1 whenever the jobs differ
  int last_split = 0;  // jobs the last batch ran in the long-chain lane
  int ks_place = 0;    // run-ahead productions: 0 shared SMs, 1 as the context's own calls place them
  bool ks_urgent = false;  // productions for a stream with no frame produced ahead go to its urgent stream
  bool ks_low = false;  // run-ahead productions at the device's lowest stream priority (else its highest)
  BatchLane cons_long;  // the long-chain lane (its own staging and graphs)
  cudaStream_t side = nullptr;  // the long-chain lane's stream
  cudaEvent_t fork = nullptr, join = nullptr, long_up = nullptr;
  cudaEvent_t done = nullptr;  // the end of the last batch, on its stream
  cudaStream_t cap_stream = nullptr;
  std::map<size_t, int> ctas_for_smem;  // round-kernel CTAs per SM by shared-memory size (queried once)
};

namespace {

int bucket(int v, int lo) {
  int b = lo;
  while (b < v) b <<= 1;
  return b;
}

void drop_graphs(BatchLane& l) {
  for (auto& kv : l.graphs) cudaGraphExecDestroy(kv.second);
  l.graphs.clear();
}

void free_lane(BatchLane& l) {  // the device is idle
  drop_graphs(l);
  dev_free(l.d_jobs, nullptr);
  dev_free(l.d_hdr, nullptr);
  for (int i = 0; i < 2; i++) {
    cudaFreeHost(l.h_jobs[i]);
    cudaFreeHost(l.h_hdr[i]);
    if (l.staged[i]) cudaEventDestroy(l.staged[i]);
  }
  for (void* h : l.retired_host) cudaFreeHost(h);
  l = BatchLane();
}

int init_lane(BatchLane& l) {
  bool ok = dev_alloc(&l.d_hdr, sizeof(vc::BatchHdr)) == cudaSuccess &&
            cudaMallocHost(&l.h_hdr[0], sizeof(vc::BatchHdr)) == cudaSuccess &&
            cudaMallocHost(&l.h_hdr[1], sizeof(vc::BatchHdr)) == cudaSuccess &&
            cudaEventCreateWithFlags(&l.staged[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&l.staged[1], cudaEventDisableTiming) == cudaSuccess;
  return ok ? VC_OK : VC_ERR_OOM;
}

// Descriptors for `need` jobs.  The old device array goes back to the pool
// after the work enqueued on `after` (the batches that read it); the old
// pinned staging is kept until the lane is freed.
int grow_lane(BatchLane& l, int need, cudaStream_t after) {
  if (need <= l.jobs_cap) return VC_OK;
  const int cap = bucket(need, 64);
  drop_graphs(l);  // the descriptor address is a kernel argument of the captured graphs (in flight: freed when done)
  dev_free(l.d_jobs, after);
  for (int i = 0; i < 2; i++)
    if (l.h_jobs[i]) l.retired_host.push_back(l.h_jobs[i]);
  l.d_jobs = nullptr;
  l.h_jobs[0] = l.h_jobs[1] = nullptr;
  l.jobs_cap = 0;
  if (dev_alloc(&l.d_jobs, sizeof(vc::JobDesc) * cap) != cudaSuccess ||
      cudaMallocHost(&l.h_jobs[0], sizeof(vc::JobDesc) * cap) != cudaSuccess ||
      cudaMallocHost(&l.h_jobs[1], sizeof(vc::JobDesc) * cap) != cudaSuccess) {
    cudaGetLastError();
    set_err("batch descriptor allocation failed");
    return VC_ERR_OOM;
  }
  l.jobs_cap = cap;
  return VC_OK;
}

// aggw: bytes per sub-tile aggregate (4 for per-channel chains)
size_t job_scratch_bytes(const Layout& L, int nf, bool with_keystream, int aggw = 1) {
  size_t b = 2 * round256((size_t)nf * L.Npad) + 2 * round256((size_t)nf * L.NS * aggw);
  if (with_keystream)
    b += round256((size_t)nf * L.rounds * L.Npad) + round256((size_t)nf * L.H * sizeof(int)) +
         round256((size_t)nf * sizeof(long long));
  return b;
}

// A keystream ring of `cap` frame slots; the first one also makes the
// productions' stream (low_priority: the device's lowest, else its highest).
int ensure_ring(vc_ctx* c, int cap, bool low_priority) {
  if (!c->prod_stream) {
    int least = 0, greatest = 0;
    VC_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    VC_CUDA(cudaStreamCreateWithPriority(&c->prod_stream, cudaStreamNonBlocking, low_priority ? least : greatest));
    VC_CUDA(cudaStreamCreateWithPriority(&c->prod_urgent, cudaStreamNonBlocking, greatest));
  }
  if (c->ring_cap >= cap) return VC_OK;
  if (c->ring_cap > 0 && c->produced != c->frame) {
    set_err("cannot grow a keystream ring that holds frames");
    return VC_ERR_SEQUENCE;
  }
  cudaStream_t after = ctx_join(c);  // after the productions and batches that used it
  dev_free(c->ring_ks, after);
  dev_free(c->ring_sc, after);
  dev_free(c->ring_kmod, after);
  c->ring_ks = nullptr;
  c->ring_sc = nullptr;
  c->ring_kmod = nullptr;
  c->ring_cap = 0;
  const Layout& L = c->L;
  if (dev_alloc(&c->ring_ks, (size_t)cap * L.rounds * L.Npad) != cudaSuccess ||
      dev_alloc(&c->ring_sc, (size_t)cap * sizeof(long long)) != cudaSuccess ||
      dev_alloc(&c->ring_kmod, (size_t)cap * L.H * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    set_err("keystream ring allocation failed");
    return VC_ERR_OOM;
  }
  for (cudaEvent_t e : c->ev_slot) cudaEventDestroy(e);
  c->ev_slot.assign((size_t)cap, nullptr);
  for (auto& e : c->ev_slot)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      set_err("ring event creation failed");
      return VC_ERR_CUDA;
    }
  c->ring_cap = cap;
  return VC_OK;
}

// Non-blocking: advance produced_done over the completed productions.
int poll_production(vc_ctx* c) {
  for (int64_t k = c->nprod - vc_ctx::kProdEv; k < c->nprod; k++) {
    if (k < 0) continue;
    const int i = (int)(k % vc_ctx::kProdEv);
    if (c->prod_upto[i] <= c->produced_done) continue;
    const cudaError_t e = cudaEventQuery(c->ev_prod[i]);
    if (e == cudaErrorNotReady) break;  // later ones are not done either
    if (e != cudaSuccess) {
      set_err("cudaEventQuery: %s", cudaGetErrorString(e));
      return VC_ERR_CUDA;
    }
    c->produced_done = c->prod_upto[i];
  }
  return VC_OK;
}

bool production_busy(vc_ctx* c) {
  if (c->nprod == 0) return false;
  return cudaEventQuery(c->ev_prod[(c->nprod - 1) % vc_ctx::kProdEv]) == cudaErrorNotReady;
}

// Productions not known complete (after a non-blocking poll).
int productions_in_flight(vc_ctx* c) {
  if (poll_production(c) != VC_OK) return vc_ctx::kProdEv;
  int n = 0;
  for (int64_t k = std::max<int64_t>(0, c->nprod - vc_ctx::kProdEv); k < c->nprod; k++)
    if (c->prod_upto[k % vc_ctx::kProdEv] > c->produced_done) n++;
  return n;
}

// Produce frames [produced, target) of the stream's keystream into its ring on
// its own internal stream, after the batch that last read the ring's slots.
// place: 0 one-warp CTAs sharing the SMs, 1 the placement of the context's own
// calls (VC_OPT_KS_SM_WARPS); an explicit VC_OPT_KS_SM_WARPS > 0 holds SMs in
// both.
// urgent: on the high-priority production stream (the stream has no frame
// produced ahead of its next one), after the last production wherever it ran.
int produce(vc_ctx* c, int64_t target, int place, bool urgent = false) {
  if (c->produced >= target) return VC_OK;
  vc::NvtxRange range("vc.keystream");
  cudaStream_t ks = (urgent && c->prod_urgent) ? c->prod_urgent : c->prod_stream;
  if (c->last_prod && c->last_prod != ks && c->nprod > 0)  // the chains continue from the last production
    VC_CUDA(cudaStreamWaitEvent(ks, c->ev_prod[(c->nprod - 1) % vc_ctx::kProdEv], 0));
  c->last_prod = ks;
  if (c->produced == c->frame && !c->batch_pending) {  // single-stream work on this context first
    for (cudaStream_t o : {c->last, c->ks_stream})
      if (o) {
        VC_CUDA(cudaEventRecord(c->ev_entry, o));
        VC_CUDA(cudaStreamWaitEvent(ks, c->ev_entry, 0));
      }
  }
  // the slots about to be overwritten: after the batches that read them (a slot
  // no batch has read yet has an event never recorded: no wait)
  for (int64_t f = c->produced; f < target; f++) VC_CUDA(cudaStreamWaitEvent(ks, c->ev_slot[f % c->ring_cap], 0));
  // at most kProdEv productions in flight (their events are tracked); the
  // oldest is normally long done, this only blocks if it is not
  if (c->nprod >= vc_ctx::kProdEv) {
    const int i = (int)(c->nprod % vc_ctx::kProdEv);
    if (c->prod_upto[i] > c->produced_done) {
      VC_CUDA(cudaEventSynchronize(c->ev_prod[i]));
      c->produced_done = c->prod_upto[i];
    }
  }
  const int nf = (int)(target - c->produced);
  const int slot0 = (int)(c->produced % c->ring_cap);
  VC_CUDA(vc::launch_frame_schedule(c->L, c->d_main, nf, c->ring_sc, c->ring_kmod, ks, c->ring_cap, slot0));
  // one-warp CTAs sharing the SMs (many streams' chains pack the pipes),
  // unless VC_OPT_KS_SM_WARPS was set explicitly: then CTAs of that many warps
  // that hold whole SMs (for a stream whose serial chains would otherwise
  // miss its frame period)
  VC_CUDA(vc::launch_keystream(c->kind, c->L, c->tables(), c->chains(), nf, c->ring_ks, c->plcm_int, ks, c->ring_cap,
                               slot0, c->ks_sm_warps > 0 ? c->ks_sm_warps : (place == 1 ? ks_warps_in_use(c) : 0)));
  const int i = (int)(c->nprod % vc_ctx::kProdEv);
  VC_CUDA(cudaEventRecord(c->ev_prod[i], ks));
  c->prod_upto[i] = target;
  c->nprod++;
  c->produced = target;
  return VC_OK;
}

vc::JobDesc base_desc(vc_ctx* c) {
  vc::JobDesc d{};
  d.L = c->L;
  d.tb = c->tables();
  d.ch = c->chains();
  d.main = c->d_main;
  d.kind = c->kind;
  return d;
}

// Stage `nj` descriptors (already in l.h_jobs[l.cur]) and launch them on st:
// a captured graph per shape, or plain launches.
// uploaded != nullptr: plain launches (no graph), with `uploaded` recorded on
// st between the descriptor upload and the kernels.
int launch_lane(vc_batcher* b, BatchLane& l, int nj, int warps, int tiles, int kmods, int rounds, size_t smem,
                cudaStream_t st, const int* vbeg, const int* vend, int variants, int ks_sm_warps,
                cudaEvent_t uploaded = nullptr) {
  vc::JobDesc* hj = l.h_jobs[l.cur];
  vc::BatchHdr* hh = l.h_hdr[l.cur];
  hh->njobs = nj;
  hh->total_warps = warps;
  hh->total_tiles = tiles;
  hh->total_kmod = kmods;
  for (int v = 0; v < vc::kBatchVariants; v++) {
    hh->vbeg[v] = vbeg[v];
    hh->vend[v] = vend[v];
  }
  vc::BatchShape sh;
  sh.variants = variants;
  sh.ks_sm_warps = ks_sm_warps;
  sh.jobs_cap = bucket(nj, 64);
  if (sh.jobs_cap > l.jobs_cap) sh.jobs_cap = l.jobs_cap;
  sh.warps_cap = bucket(warps, 64);
  sh.kmod_cap = bucket(kmods, 1024);
  sh.rounds = rounds;
  sh.smem = (smem + 16383) & ~(size_t)16383;
  sh.grid = 1;
  if (rounds > 0) {
    int ctas = 0;
    auto hit = b->ctas_for_smem.find(sh.smem);
    if (hit != b->ctas_for_smem.end()) {
      ctas = hit->second;
    } else {
      VC_CUDA(vc::prepare_batch_kernels(sh.smem));
      VC_CUDA(vc::batch_ctas_per_sm(sh.smem, &ctas));
      b->ctas_for_smem[sh.smem] = ctas;
    }
    if (ctas < 1) {
      set_err("round kernel does not fit with %zu bytes of shared memory", sh.smem);
      return VC_ERR_UNSUPPORTED;
    }
    if (b->ctas_per_sm > 0 && b->ctas_per_sm < ctas) ctas = b->ctas_per_sm;
    sh.grid = b->sms * ctas;
  }
  const size_t jobs_bytes = sizeof(vc::JobDesc) * (size_t)sh.jobs_cap;
  if (b->use_graph && !uploaded) {
    const auto key = std::make_tuple(sh.jobs_cap, sh.warps_cap, sh.kmod_cap, sh.rounds, sh.grid, sh.smem, l.cur,
                                     sh.variants * 8 + sh.ks_sm_warps);
    auto it = l.graphs.find(key);
    if (it == l.graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      VC_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaMemcpyAsync(l.d_hdr, hh, sizeof(vc::BatchHdr), cudaMemcpyHostToDevice, b->cap_stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(l.d_jobs, hj, jobs_bytes, cudaMemcpyHostToDevice, b->cap_stream);
      if (e == cudaSuccess) e = vc::launch_batch(l.d_jobs, l.d_hdr, sh, b->cap_stream);
      const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        set_err("batch graph capture failed: %s", cudaGetErrorString(e));
        return VC_ERR_CUDA;
      }
      it = l.graphs.emplace(key, ge).first;
    }
    VC_CUDA(cudaGraphLaunch(it->second, st));
  } else {
    VC_CUDA(cudaMemcpyAsync(l.d_hdr, hh, sizeof(vc::BatchHdr), cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaMemcpyAsync(l.d_jobs, hj, jobs_bytes, cudaMemcpyHostToDevice, st));
    if (uploaded) VC_CUDA(cudaEventRecord(uploaded, st));
    VC_CUDA(vc::launch_batch(l.d_jobs, l.d_hdr, sh, st));
  }
  VC_CUDA(cudaEventRecord(l.staged[l.cur], st));
  l.cur ^= 1;
  return VC_OK;
}

}  // namespace

extern "C" {

int vc_batcher_create(vc_batcher** out) {
  if (!out) return VC_ERR_ARG;
  *out = nullptr;
  vc_batcher* b = new (std::nothrow) vc_batcher();
  if (!b) return VC_ERR_OOM;
  cudaGetDevice(&b->dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  bool ok = init_lane(b->cons) == VC_OK && grow_lane(b->cons, 64, nullptr) == VC_OK &&
            init_lane(b->cons_long) == VC_OK && grow_lane(b->cons_long, 64, nullptr) == VC_OK &&
            cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, prio_greatest) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->long_up, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    vc_batcher_destroy(b);
    set_err("batcher creation failed");
    return VC_ERR_OOM;
  }
  *out = b;
  return VC_OK;
}

int vc_batcher_set_option(vc_batcher* b, int32_t option, int64_t value) {
  if (!b) return VC_ERR_ARG;
  switch (option) {
    case VC_BOPT_GRAPH:
      if (value != 0 && value != 1) return VC_ERR_ARG;
      b->use_graph = value != 0;
      return VC_OK;
    case VC_BOPT_CTAS_PER_SM:
      if (value < 0 || value > 32) return VC_ERR_ARG;
      b->ctas_per_sm = (int)value;
      drop_graphs(b->cons);
      drop_graphs(b->cons_long);
      return VC_OK;
    case VC_BOPT_RUNAHEAD:
      if (value < 0 || value > 64) return VC_ERR_ARG;
      b->runahead = (int)value;
      return VC_OK;
    case VC_BOPT_SINE:
      if (value < -1 || value > 1) return VC_ERR_ARG;
      b->sine = (int)value;
      return VC_OK;
    case VC_BOPT_SPLIT:
      if (value < -1 || value > 1) return VC_ERR_ARG;
      b->split = (int)value;
      return VC_OK;
    case VC_BOPT_KS_PLACE:
      if (value != 0 && value != 1) return VC_ERR_ARG;
      b->ks_place = (int)value;
      return VC_OK;
    case VC_BOPT_KS_PRIORITY:
      if (value != 0 && value != 1) return VC_ERR_ARG;
      b->ks_low = value == 1;
      return VC_OK;
    case VC_BOPT_KS_URGENT:
      if (value != 0 && value != 1) return VC_ERR_ARG;
      b->ks_urgent = value == 1;
      return VC_OK;
  }
  return VC_ERR_ARG;
}

}  // extern "C"

namespace {

// Descriptors of one lane of a batch and its launch geometry.
struct LaneFill {
  int nj = 0, warps = 0, tiles = 0, kmods = 0, rounds = 0, variants = 0;
  size_t smem = 4096;  // at least the fix-up's carries
  int vbeg[vc::kBatchVariants] = {}, vend[vc::kBatchVariants] = {};
};

// Serial steps of one map chain of a job (its longest subframe) times the
// cycles of one step, for choosing which jobs bound a batch with the
// keystream inline (PLCM and logistic: one iterate per 6 bytes of a map;
// 2DLASM: one step per 12 bytes of a pair).
double job_chain_cycles(const vc_job& J) {
  const Layout& L = J.ctx->L;
  const double smax = (double)L.C * (double)((L.P + L.n - 1) / L.n);
  const double bytes = (double)J.nframes * L.rounds * smax;
  const int kind = J.ctx->kind;
  const double steps = kind == VC_2DLASM ? bytes / 12.0 : bytes / 6.0;
  const double cyc = kind == VC_2DLASM ? 3400.0 : (kind == VC_LOGISTIC ? 370.0 : 290.0);
  return steps * cyc;
}

// lane_of[k] = 1 for the jobs that go to the long-chain lane.  Automatic
// (VC_BOPT_SPLIT -1): the jobs whose chains take at least half the longest,
// when the longest takes over 2 ms at 2 GHz, the others are at least a
// quarter of the batch's jobs, and the long jobs' warps fit on half the SMs
// in two-warp CTAs; 1: the same without the size conditions.
bool split_long_jobs(const vc_batcher* b, const vc_job* jobs, const std::vector<int>& live, std::vector<int>& lane_of) {
  const int nj = (int)live.size();
  if (b->split == 0 || nj < 2) return false;
  double tmax = 0;
  std::vector<double> t((size_t)nj);
  for (int k = 0; k < nj; k++) {
    t[k] = job_chain_cycles(jobs[live[k]]);
    tmax = std::max(tmax, t[k]);
  }
  int nlong = 0, lwarps = 0;
  for (int k = 0; k < nj; k++) {
    lane_of[k] = t[k] >= 0.5 * tmax ? 1 : 0;
    if (lane_of[k]) {
      nlong++;
      lwarps += (jobs[live[k]].ctx->L.n + 15) / 16;
    }
  }
  if (nlong == nj) {  // all alike: nothing bounds the batch alone
    for (int k = 0; k < nj; k++) lane_of[k] = 0;
    if (b->split != 1) return false;
    int kmax = 0;
    for (int k = 1; k < nj; k++)
      if (t[k] > t[kmax]) kmax = k;
    lane_of[kmax] = 1;
    return true;
  }
  if (b->split == 1) return true;
  const bool ok = tmax > 4e6 && 4 * (nj - nlong) >= nj && lwarps <= b->sms;
  if (!ok) std::fill(lane_of.begin(), lane_of.end(), 0);
  return ok;
}

// Descriptors of the jobs live[k] with lane_of[k] == which into lane l's
// staging, their scratch taken from the pool at *pp.
void fill_lane(vc_batcher* b, BatchLane& l, const vc_job* jobs, const std::vector<int>& live,
               const std::vector<int>& lane_of, int which, int A, uint8_t** pp, LaneFill& F) {
  vc::JobDesc* hj = l.h_jobs[l.cur];
  uint8_t* p = *pp;
  for (int k = 0; k < (int)live.size(); k++) {
    if (lane_of[k] != which) continue;
    const vc_job& J = jobs[live[k]];
    vc_ctx* c = J.ctx;
    const Layout& L = c->L;
    const int nf = J.nframes;
    const bool pc = c->diff_pc && L.C > 1;
    const int v = vc::batch_variant(J.direction, L.C, pc);
    if (!(F.variants & (1 << v))) F.vbeg[v] = F.tiles;
    F.variants |= 1 << v;
    F.vend[v] = F.tiles + nf * L.NT;
    vc::JobDesc d = base_desc(c);
    d.dir = J.direction;
    d.nframes = nf;
    d.in = J.d_in;
    d.out = J.d_out;
    if (A > 0) {
      d.mode = 1;
      d.ks = c->ring_ks;
      d.sc = c->ring_sc;
      d.kmod = c->ring_kmod;
      d.ring_cap = c->ring_cap;
      d.ring_slot0 = (int)(c->frame % c->ring_cap);
    } else {
      d.mode = 0;
      d.ks = p;
      p += round256((size_t)nf * L.rounds * L.Npad);
      d.kmod = reinterpret_cast<int*>(p);
      p += round256((size_t)nf * L.H * sizeof(int));
      d.sc = reinterpret_cast<long long*>(p);
      p += round256((size_t)nf * sizeof(long long));
    }
    d.buf[0] = p;
    p += round256((size_t)nf * L.Npad);
    d.buf[1] = p;
    p += round256((size_t)nf * L.Npad);
    d.pc = pc ? 1 : 0;
    d.agg[0] = p;
    p += round256((size_t)nf * L.NS * (pc ? 4 : 1));
    d.agg[1] = p;
    p += round256((size_t)nf * L.NS * (pc ? 4 : 1));
    d.warp_base = F.warps;
    d.tile_base = F.tiles;
    d.kmod_base = F.kmods;
    if (d.mode == 0) {
      F.warps += (L.n + 15) / 16;
      F.kmods += nf * L.H;
    }
    F.tiles += nf * L.NT;
    if (L.rounds > F.rounds) F.rounds = L.rounds;
    const size_t sm = vc::round_smem_bytes(L, pc);
    if (sm > F.smem) F.smem = sm;
    hj[F.nj++] = d;
  }
  // 2DLASM chains of the lane's keystream: the all-binary64 sine reduction
  // (the shorter dependency chain) on SMs they hold, and while their warps
  // leave the SMs' binary64 pipes unsaturated -- about 3.5 warps of 2DLASM
  // chains fill one SM's pipe -- else the integer-assisted one (fewer
  // binary64 operations); both give the same bits
  int lasm_warps = 0;
  for (int k = 0; k < F.nj; k++)
    if (hj[k].mode == 0 && hj[k].kind == VC_2DLASM) lasm_warps += (hj[k].L.n + 15) / 16;
  const int b64 = b->sine >= 0 ? b->sine : ((which == 1 || 2 * lasm_warps <= 7 * b->sms) ? 1 : 0);
  for (int k = 0; k < F.nj; k++) hj[k].sine_b64 = (hj[k].kind == VC_2DLASM) ? b64 : 0;
  *pp = p;
}

}  // namespace

extern "C" {

int vc_batch_submit(vc_batcher* b, const vc_job* jobs, int32_t njobs, void* stream) {
  vc::NvtxRange range("vc.batch");
  if (!b || njobs < 0 || (njobs > 0 && !jobs)) {
    set_err("invalid argument");
    return VC_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int A = b->runahead;
  // validate and lay out the jobs
  std::vector<int> live;
  live.reserve(njobs);
  std::unordered_set<const vc_ctx*> seen;
  size_t pool_need = 0;
  for (int j = 0; j < njobs; j++) {
    const vc_job& J = jobs[j];
    if (!J.ctx || (J.direction != 0 && J.direction != 1) || J.nframes < 0 ||
        (J.nframes > 0 && (!J.d_in || !J.d_out))) {
      set_err("invalid job %d", j);
      return VC_ERR_ARG;
    }
    if (!seen.insert(J.ctx).second) {
      set_err("job %d repeats a context", j);
      return VC_ERR_ARG;
    }
    if (J.nframes == 0) continue;
    if (J.ctx->L.rounds == 1 && J.d_in == J.d_out) {
      set_err("job %d: in-place with one round is not supported in a batch", j);
      return VC_ERR_ARG;
    }
    if (A > 0 && J.nframes > A) {
      set_err("job %d asks for %d frames, more than the %d frames of keystream run-ahead", j, J.nframes, A);
      return VC_ERR_ARG;
    }
    if (A == 0 && J.ctx->produced != J.ctx->frame) {
      set_err("job %d: its stream holds keystream produced ahead; keep run-ahead on", j);
      return VC_ERR_SEQUENCE;
    }
    live.push_back(j);
    pool_need += job_scratch_bytes(J.ctx->L, J.nframes, A == 0, J.ctx->diff_pc ? 4 : 1);
  }
  const int nj = (int)live.size();
  if (nj == 0) return VC_OK;
  // jobs ordered by round-kernel variant (direction, channels): each variant's
  // tiles form one range
  std::stable_sort(live.begin(), live.end(), [&](int x, int y) {
    return vc::batch_variant(jobs[x].direction, jobs[x].ctx->L.C, jobs[x].ctx->diff_pc) <
           vc::batch_variant(jobs[y].direction, jobs[y].ctx->L.C, jobs[y].ctx->diff_pc);
  });
  int rc = VC_OK;
  for (int k = 0; k < nj; k++) {  // single-stream calls' keystream generated ahead: undone
    rc = spec_rollback(jobs[live[k]].ctx);
    if (rc) return rc;
  }
  // what the last batch used goes back to the pool after it (st waits for its end)
  if (nj > b->cons.jobs_cap || nj > b->cons_long.jobs_cap || pool_need > b->pool_cap)
    VC_CUDA(cudaStreamWaitEvent(st, b->done, 0));
  rc = grow_lane(b->cons, nj, st);
  if (rc) return rc;
  rc = grow_lane(b->cons_long, nj, st);
  if (rc) return rc;
  if (pool_need > b->pool_cap) {
    dev_free(b->d_pool, st);
    b->d_pool = nullptr;
    b->pool_cap = 0;
    const size_t cap = pool_need + pool_need / 4;
    if (dev_alloc(&b->d_pool, cap) != cudaSuccess) {
      cudaGetLastError();
      set_err("batch scratch pool of %zu bytes failed", cap);
      return VC_ERR_OOM;
    }
    b->pool_cap = cap;
  }
  for (int k = 0; k < nj; k++) {
    const vc_job& J = jobs[live[k]];
    vc_ctx* c = J.ctx;
    // the batch runs after what the context's single-stream calls enqueued on other streams
    if (c->last && c->last != st && !c->batch_pending) {
      VC_CUDA(cudaEventRecord(c->ev_entry, c->last));
      VC_CUDA(cudaStreamWaitEvent(st, c->ev_entry, 0));
    }
    if (A > 0) {
      // frames not produced yet are produced now (with the look-ahead); the
      // batch waits only if its frames are not known to be complete
      rc = ensure_ring(c, 2 * A + 1, b->ks_low);
      if (rc) return rc;
      if (c->produced < c->frame + J.nframes) {
        rc = produce(c, c->frame + J.nframes + A, b->ks_place, b->ks_urgent);
        if (rc) return rc;
      }
      rc = poll_production(c);
      if (rc) return rc;
      if (c->produced_done < c->frame + J.nframes)
        VC_CUDA(cudaStreamWaitEvent(st, c->ev_prod[(c->nprod - 1) % vc_ctx::kProdEv], 0));
    }
  }

  // ---- the batch: the rounds of every job (and the keystream when inline) ----
  // With the keystream inline, jobs whose chains are much longer than the
  // rest (they bound the batch) may go to a second lane on a side stream:
  // their keystream in CTAs that hold whole SMs, their rounds behind it,
  // while the other jobs' keystream and rounds run beside them.
  std::vector<int> lane_of((size_t)nj, 0);
  const bool split = A == 0 && split_long_jobs(b, jobs, live, lane_of);
  uint8_t* p = b->d_pool;
  LaneFill F0, F1;
  VC_CUDA(cudaEventSynchronize(b->cons.staged[b->cons.cur]));
  fill_lane(b, b->cons, jobs, live, lane_of, 0, A, &p, F0);
  if (split) {
    VC_CUDA(cudaEventSynchronize(b->cons_long.staged[b->cons_long.cur]));
    fill_lane(b, b->cons_long, jobs, live, lane_of, 1, A, &p, F1);
    // the long lane first, on a stream of the highest priority: its CTAs need
    // empty SMs, so they must reach the GPU before the short lane's CTAs
    // spread over every SM; the short lane waits for its descriptor upload
    VC_CUDA(cudaEventRecord(b->fork, st));
    VC_CUDA(cudaStreamWaitEvent(b->side, b->fork, 0));
    rc = launch_lane(b, b->cons_long, F1.nj, F1.warps, F1.tiles, F1.kmods, F1.rounds, F1.smem, b->side, F1.vbeg,
                     F1.vend, F1.variants, 2, b->long_up);
    if (rc) return rc;
    VC_CUDA(cudaEventRecord(b->join, b->side));
    VC_CUDA(cudaStreamWaitEvent(st, b->long_up, 0));
  }
  rc = launch_lane(b, b->cons, F0.nj, F0.warps, F0.tiles, F0.kmods, F0.rounds, F0.smem, st, F0.vbeg, F0.vend,
                   F0.variants, 0);
  if (rc) return rc;
  if (split) VC_CUDA(cudaStreamWaitEvent(st, b->join, 0));
  VC_CUDA(cudaEventRecord(b->done, st));
  b->last_split = split ? F1.nj : 0;
  for (int k = 0; k < nj; k++) {
    const vc_job& J = jobs[live[k]];
    vc_ctx* c = J.ctx;
    if (A > 0)
      for (int64_t f = c->frame; f < c->frame + J.nframes; f++)
        VC_CUDA(cudaEventRecord(c->ev_slot[f % c->ring_cap], st));
    c->frame += J.nframes;
    if (A == 0) {
      c->produced = c->frame;
      c->produced_done = c->frame;
    }
    c->last = st;
    VC_CUDA(cudaEventRecord(c->ev_batch, st));
    c->batch_pending = true;
  }
  // ---- top-ups: each stream's keystream back to A frames ahead, on its own
  // internal stream, queued behind the productions still running there (so
  // that a long chain never idles between frames), a few at most ----
  if (A > 0) {
    for (int k = 0; k < nj; k++) {
      vc_ctx* c = jobs[live[k]].ctx;
      if (c->produced >= c->frame + A || productions_in_flight(c) >= vc_ctx::kProdEv / 2) continue;
      rc = produce(c, c->frame + A, b->ks_place, b->ks_urgent && c->produced <= c->frame);
      if (rc) return rc;
    }
  }
  return VC_OK;
}

int vc_batch_prefetch(vc_batcher* b, vc_ctx* const* ctxs, int32_t n) {
  if (!b || n < 0 || (n > 0 && !ctxs)) return VC_ERR_ARG;
  const int A = b->runahead;
  if (A <= 0) {
    set_err("prefetch needs run-ahead (VC_BOPT_RUNAHEAD > 0)");
    return VC_ERR_ARG;
  }
  std::unordered_set<const vc_ctx*> seen;
  for (int k = 0; k < n; k++) {
    vc_ctx* c = ctxs[k];
    if (!c || !seen.insert(c).second) {
      set_err("prefetch: null or repeated context");
      return VC_ERR_ARG;
    }
    int rc = spec_rollback(c);
    if (rc) return rc;
    rc = ensure_ring(c, 2 * A + 1, b->ks_low);
    if (rc) return rc;
    // the next frame on its own (ready soonest), then the rest of the run-ahead
    // queued behind it; a repeated call while a production is in flight adds
    // nothing (coalesced, like the top-ups)
    bool issued = false;
    if (c->produced < c->frame + 1) {
      rc = produce(c, c->frame + 1, b->ks_place, b->ks_urgent);
      if (rc) return rc;
      issued = true;
    }
    if (c->produced < c->frame + A && (issued || !production_busy(c))) {
      rc = produce(c, c->frame + A, b->ks_place);
      if (rc) return rc;
    }
  }
  return VC_OK;
}

int vc_batch_ready(vc_batcher* b, const vc_ctx* c, int32_t nframes) {
  if (!b || !c || nframes < 0) return -VC_ERR_ARG;
  if (nframes == 0) return 1;
  vc_ctx* cc = const_cast<vc_ctx*>(c);
  const int rc = poll_production(cc);
  if (rc) return -rc;
  return cc->produced_done >= cc->frame + nframes ? 1 : 0;
}

int vc_dbg_batch_split(const vc_batcher* b) { return b ? b->last_split : -VC_ERR_ARG; }

void vc_batcher_destroy(vc_batcher* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_lane(b->cons);
  free_lane(b->cons_long);
  dev_free(b->d_pool, nullptr);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->long_up) cudaEventDestroy(b->long_up);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
}

}  // extern "C"
