// vc_server.cu -- the per-tick work of a continuous-batching serving loop in
// native code, on top of the library's public C ABI (vcrypt.h).
//
// The paper's target is real-time video (every frame of a 24 FPS stream within
// its 41.7 ms frame time, Sec. 6).  A server holds many independent streams;
// each tick it takes, for every stream, the frames that have arrived by its
// frame clock and whose keystream run-ahead is ready, and submits them as one
// ragged batch (vc_batch_submit: one launch per phase over all streams), or,
// for comparison, as one encrypt_frames / decrypt_frames call per frame, each
// stream on its own CUDA stream so that different streams' calls overlap.
// Completion is timed with CUDA events against an event recorded at creation,
// so per-frame latency = device completion time - arrival time.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdint>
#include <algorithm>
#include <deque>
#include <vector>

#include "vc_internal.h"
#include "vcrypt.h"
#include "vcrypt_debug.h"

namespace {

struct SrvStream {
  vc_ctx* ctx = nullptr;
  int dir = 0;
  long long N = 0;  // bytes per frame
  const uint8_t* src = nullptr;
  int src_period = 1;
  uint8_t* ring = nullptr;
  int ring_frames = 1;
  double fps = 24.0, t_arr = 0.0;
  int64_t total = 0, next = 0, done = 0;
  bool active = false;
  // one-call-per-frame mode: the stream's own CUDA stream, so that the calls
  // of different streams run concurrently, and the event that joins it back
  cudaStream_t cs = nullptr;
  cudaEvent_t join = nullptr;
};

struct SrvFrame {
  int32_t id;
  int64_t frame;
  double arrival;
  double submitted;  // host time of the tick that submitted it
};

struct SrvTick {
  cudaEvent_t ev0 = nullptr;  // before the submission
  cudaEvent_t ev = nullptr;   // after all of the tick's work
  std::vector<SrvFrame> frames;
  // one-call-per-frame mode: the completion event of each stream's calls and
  // the end of its frames in `frames` (each frame is timed by its own stream)
  std::vector<cudaEvent_t> job_ev;
  std::vector<size_t> job_end;
  size_t taken = 0;  // frames already returned by a partial drain
  double now = 0.0;  // host time of the submission
};

}  // namespace

struct vc_server {
  int mode = 0;  // 0 batch, 1 one call per frame
  int maxf = 4;
  cudaStream_t st = nullptr;
  vc_batcher* b = nullptr;
  cudaEvent_t t0 = nullptr;
  std::vector<SrvStream> streams;
  std::deque<SrvTick> inflight;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<vc_job> jobs;
  std::vector<int32_t> job_stream;  // stream index of each job
  std::vector<vc_ctx*> starved;
  double host_ms[4] = {0, 0, 0, 0};  // readiness and job building, prefetch, submission, completion event
  int64_t host_ticks = 0;
  double gpu_ms = 0;  // device time from a tick's first enqueued work to its completion, summed
  int64_t gpu_ticks = 0;
  // latency records (vc_dbg_server_record): per frame (stream, arrival,
  // submission, completion), per tick (submission, device start, device end,
  // frames), seconds since creation
  bool rec = false;
  std::vector<double> rec_frames, rec_ticks;
  // batching: a tick is submitted only while fewer than this many submitted
  // ticks wait for the device to start them (0: every tick); the frames of a
  // skipped tick go into the next, larger batch
  int max_queued = 0;
  int64_t skipped = 0;
  // batching lanes: tick i goes to lane i mod lanes (lane 0: b on st), each
  // with its own batcher (scratch, staging, graphs) and stream, so that a tick
  // whose kernels wait for SMs does not hold up the ticks of the other lanes
  std::vector<vc_batcher*> lane_b;
  std::vector<cudaStream_t> lane_st;
  int64_t next_lane = 0;
  std::vector<std::pair<int32_t, int64_t>> bopts;  // batcher options set so far (replayed on new lanes)
};

namespace {

double ms_since(std::chrono::steady_clock::time_point a) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
}

cudaEvent_t srv_event(vc_server* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

}  // namespace

extern "C" {

int vc_server_create(int32_t mode, int32_t max_frames_per_tick, void* stream, vc_server** out) {
  if (!out || (mode != 0 && mode != 1) || max_frames_per_tick < 1 || max_frames_per_tick > 64) return VC_ERR_ARG;
  *out = nullptr;
  vc_server* s = new vc_server;
  s->mode = mode;
  s->maxf = max_frames_per_tick;
  s->st = (cudaStream_t)stream;
  if (mode == 0) {
    int rc = vc_batcher_create(&s->b);
    if (rc == VC_OK) rc = vc_batcher_set_option(s->b, VC_BOPT_RUNAHEAD, max_frames_per_tick);
    if (rc != VC_OK) {
      vc_server_destroy(s);
      return rc;
    }
  }
  if (cudaEventCreate(&s->t0) != cudaSuccess || cudaEventRecord(s->t0, s->st) != cudaSuccess ||
      cudaEventSynchronize(s->t0) != cudaSuccess) {
    cudaGetLastError();
    vc_server_destroy(s);
    return VC_ERR_CUDA;
  }
  *out = s;
  return VC_OK;
}

int vc_server_add(vc_server* s, vc_ctx* ctx, int32_t direction, int64_t frame_bytes, const uint8_t* d_src,
                  int32_t src_period, uint8_t* d_ring, int32_t ring_frames, double fps, double t_arrival,
                  int64_t frames_total, int32_t* id) {
  if (!s || !ctx || !id || (direction != 0 && direction != 1) || frame_bytes < 1 || !d_src || src_period < 1 ||
      !d_ring || ring_frames < 1 || !(fps > 0.0) || frames_total < 1)
    return VC_ERR_ARG;
  SrvStream t;
  t.ctx = ctx;
  t.dir = direction;
  t.N = frame_bytes;
  t.src = d_src;
  t.src_period = src_period;
  t.ring = d_ring;
  t.ring_frames = ring_frames;
  t.fps = fps;
  t.t_arr = t_arrival;
  t.total = frames_total;
  t.active = true;
  if (s->mode == 0) {
    vc_ctx* c = ctx;
    int rc = vc_batch_prefetch(s->b, &c, 1);  // keystream of its first frames now
    if (rc) return rc;
  } else if (cudaStreamCreateWithFlags(&t.cs, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&t.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (t.cs) cudaStreamDestroy(t.cs);
    return VC_ERR_CUDA;
  }
  s->streams.push_back(t);
  *id = (int32_t)(s->streams.size() - 1);
  return VC_OK;
}

int vc_server_tick(vc_server* s, double now, int32_t* frames_submitted) {
  vc::NvtxRange range("vc.tick");
  if (!s) return VC_ERR_ARG;
  if (frames_submitted) *frames_submitted = 0;
  s->jobs.clear();
  s->job_stream.clear();
  s->starved.clear();
  auto t_start = std::chrono::steady_clock::now();
  s->host_ticks++;
  if (s->mode == 0 && s->max_queued > 0) {
    int queued = 0;
    for (auto it = s->inflight.rbegin(); it != s->inflight.rend() && queued < s->max_queued; ++it) {
      const cudaError_t e = cudaEventQuery(it->ev0);
      if (e == cudaErrorNotReady) {
        queued++;
        continue;
      }
      if (e != cudaSuccess) return VC_ERR_CUDA;
      break;  // earlier ticks started before this one
    }
    if (queued >= s->max_queued) {
      s->skipped++;
      return VC_OK;
    }
  }
  SrvTick tick;
  for (size_t i = 0; i < s->streams.size(); i++) {
    SrvStream& t = s->streams[i];
    if (!t.active || t.next >= t.total) continue;
    int64_t arrived = (int64_t)std::floor((now - t.t_arr) * t.fps) + 1;
    if (arrived > t.total) arrived = t.total;
    int64_t m = arrived - t.next;
    if (m <= 0) continue;
    const int slot = (int)(t.next % t.ring_frames);
    if (m > s->maxf) m = s->maxf;
    if (m > t.ring_frames - slot) m = t.ring_frames - slot;
    if (s->mode == 0) {
      // only frames whose keystream is on the device: a stream whose keystream
      // is still being produced does not hold up the others
      while (m > 0) {
        const int r = vc_batch_ready(s->b, t.ctx, (int32_t)m);
        if (r < 0) return -r;
        if (r == 1) break;
        m--;
      }
      if (m == 0) {
        s->starved.push_back(t.ctx);
        continue;
      }
    }
    const int k0 = (int)(t.next % t.src_period);
    vc_job j;
    j.ctx = t.ctx;
    j.direction = t.dir;
    j.d_in = t.src + (size_t)k0 * t.N;
    j.d_out = t.ring + (size_t)slot * t.N;
    j.nframes = (int32_t)m;
    s->jobs.push_back(j);
    s->job_stream.push_back((int32_t)i);
    for (int64_t k = 0; k < m; k++) tick.frames.push_back(SrvFrame{(int32_t)i, t.next + k, t.t_arr + (t.next + k) / t.fps, now});
    t.next += m;
  }
  s->host_ms[0] += ms_since(t_start);
  t_start = std::chrono::steady_clock::now();
  if (!s->starved.empty()) {  // no-op for a stream whose production is in flight
    int rc = vc_batch_prefetch(s->b, s->starved.data(), (int32_t)s->starved.size());
    if (rc) return rc;
  }
  s->host_ms[1] += ms_since(t_start);
  if (s->jobs.empty()) return VC_OK;
  t_start = std::chrono::steady_clock::now();
  tick.ev0 = srv_event(s);
  // the tick's lane
  vc_batcher* lb = s->b;
  cudaStream_t lst = s->st;
  if (s->mode == 0 && !s->lane_b.empty()) {
    const int k = (int)(s->next_lane++ % (int64_t)(s->lane_b.size() + 1));
    if (k > 0) {
      lb = s->lane_b[k - 1];
      lst = s->lane_st[k - 1];
    }
  }
  if (!tick.ev0 || cudaEventRecord(tick.ev0, lst) != cudaSuccess) {
    cudaGetLastError();
    return VC_ERR_CUDA;
  }
  if (s->mode == 0) {
    int rc = vc_batch_submit(lb, s->jobs.data(), (int32_t)s->jobs.size(), lst);
    if (rc) return rc;
  } else {
    // each stream's calls on its own CUDA stream (after the tick's start),
    // timed by an event there, then joined back into the server's stream
    size_t fend = 0;
    for (size_t q = 0; q < s->jobs.size(); q++) {
      const vc_job& j = s->jobs[q];
      SrvStream& t = s->streams[s->job_stream[q]];
      if (cudaStreamWaitEvent(t.cs, tick.ev0, 0) != cudaSuccess) {
        cudaGetLastError();
        return VC_ERR_CUDA;
      }
      for (int k = 0; k < j.nframes; k++) {
        const uint8_t* in = j.d_in + (size_t)k * t.N;
        uint8_t* out = j.d_out + (size_t)k * t.N;
        int rc = j.direction == 0 ? encrypt_frames(j.ctx, in, out, 1, t.cs) : decrypt_frames(j.ctx, in, out, 1, t.cs);
        if (rc) return rc;
      }
      cudaEvent_t e = srv_event(s);
      if (!e || cudaEventRecord(e, t.cs) != cudaSuccess || cudaEventRecord(t.join, t.cs) != cudaSuccess ||
          cudaStreamWaitEvent(s->st, t.join, 0) != cudaSuccess) {
        cudaGetLastError();
        return VC_ERR_CUDA;
      }
      fend += (size_t)j.nframes;
      tick.job_ev.push_back(e);
      tick.job_end.push_back(fend);
    }
  }
  s->host_ms[2] += ms_since(t_start);
  t_start = std::chrono::steady_clock::now();
  tick.ev = srv_event(s);
  if (!tick.ev || cudaEventRecord(tick.ev, lst) != cudaSuccess) {
    cudaGetLastError();
    return VC_ERR_CUDA;
  }
  s->host_ms[3] += ms_since(t_start);
  if (frames_submitted) *frames_submitted = (int32_t)tick.frames.size();
  tick.now = now;
  s->inflight.push_back(std::move(tick));
  return VC_OK;
}

int vc_server_drain(vc_server* s, int32_t block, int32_t cap, int32_t* ids, int64_t* frames, double* arrival_s,
                    double* latency_ms, int32_t* n_out) {
  if (!s || !n_out || cap < 0 || (cap > 0 && (!ids || !frames || !arrival_s || !latency_ms))) return VC_ERR_ARG;
  int32_t n = 0;
  while (!s->inflight.empty() && n < cap) {
    SrvTick& tk = s->inflight.front();
    cudaError_t e = block ? cudaEventSynchronize(tk.ev) : cudaEventQuery(tk.ev);
    if (e == cudaErrorNotReady) break;
    if (e != cudaSuccess) return VC_ERR_CUDA;
    float ms = 0.f, dur = 0.f;
    if (cudaEventElapsedTime(&ms, s->t0, tk.ev) != cudaSuccess) return VC_ERR_CUDA;
    if (tk.taken == 0 && tk.ev0 && cudaEventElapsedTime(&dur, tk.ev0, tk.ev) == cudaSuccess) {
      s->gpu_ms += dur;
      s->gpu_ticks++;
      if (s->rec) {
        const double t = tk.now, e = ms / 1e3;
        s->rec_ticks.insert(s->rec_ticks.end(), {t, e - dur / 1e3, e, (double)tk.frames.size()});
      }
    }
    const double done_s = ms / 1e3;
    size_t q = 0;  // the job (stream) of frame tk.taken in one-call-per-frame mode
    while (tk.taken < tk.frames.size() && n < cap) {
      double fdone = done_s;
      if (!tk.job_ev.empty()) {
        while (q + 1 < tk.job_end.size() && tk.job_end[q] <= tk.taken) q++;
        float jm = 0.f;
        if (cudaEventElapsedTime(&jm, s->t0, tk.job_ev[q]) != cudaSuccess) return VC_ERR_CUDA;
        fdone = jm / 1e3;
      }
      const SrvFrame& f = tk.frames[tk.taken++];
      ids[n] = f.id;
      frames[n] = f.frame;
      arrival_s[n] = f.arrival;
      latency_ms[n] = (fdone - f.arrival) * 1e3;
      if (s->rec) s->rec_frames.insert(s->rec_frames.end(), {(double)f.id, f.arrival, f.submitted, fdone});
      s->streams[f.id].done++;
      n++;
    }
    if (tk.taken == tk.frames.size()) {
      s->ev_pool.push_back(tk.ev);
      if (tk.ev0) s->ev_pool.push_back(tk.ev0);
      for (cudaEvent_t e : tk.job_ev) s->ev_pool.push_back(e);
      s->inflight.pop_front();
    }
  }
  *n_out = n;
  return VC_OK;
}

int vc_server_stream_done(const vc_server* s, int32_t id) {
  if (!s || id < 0 || id >= (int32_t)s->streams.size()) return -VC_ERR_ARG;
  const SrvStream& t = s->streams[id];
  return t.done >= t.total ? 1 : 0;
}

int vc_server_remove(vc_server* s, int32_t id) {
  if (!s || id < 0 || id >= (int32_t)s->streams.size()) return VC_ERR_ARG;
  SrvStream& t = s->streams[id];
  if (t.done < t.next) {  // its frames still in flight: wait for them
    for (const SrvTick& tk : s->inflight)
      for (size_t k = tk.taken; k < tk.frames.size(); k++)
        if (tk.frames[k].id == id) {
          cudaEventSynchronize(tk.ev);
          break;
        }
  }
  // the context must not keep a stream of this server as the one of its last
  // work (the server destroys them)
  for (cudaStream_t ls : s->lane_st) vc::ctx_release_stream(t.ctx, ls);
  if (t.cs) {
    vc::ctx_release_stream(t.ctx, t.cs);
    cudaStreamDestroy(t.cs);
    t.cs = nullptr;
  }
  t.active = false;
  t.ctx = nullptr;
  if (t.join) {
    cudaEventDestroy(t.join);
    t.join = nullptr;
  }
  return VC_OK;
}

int32_t vc_server_inflight(const vc_server* s) { return s ? (int32_t)s->inflight.size() : 0; }

int vc_server_set_option(vc_server* s, int32_t option, int64_t value) {
  if (!s || s->mode != 0 || !s->b || option == VC_BOPT_RUNAHEAD) return VC_ERR_ARG;
  if (option == VC_SOPT_QUEUED_TICKS) {
    if (value < 0 || value > 64) return VC_ERR_ARG;
    s->max_queued = (int)value;
    return VC_OK;
  }
  if (option == VC_SOPT_LANES) {
    if (value < 1 || value > 8 || !s->streams.empty() || !s->lane_b.empty()) return VC_ERR_ARG;
    int least = 0, greatest = 0, prio = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamGetPriority(s->st, &prio) != cudaSuccess) {
      cudaGetLastError();
      return VC_ERR_CUDA;
    }
    for (int k = 1; k < (int)value; k++) {
      vc_batcher* b = nullptr;
      cudaStream_t st = nullptr;
      int rc = vc_batcher_create(&b);
      if (rc == VC_OK) rc = vc_batcher_set_option(b, VC_BOPT_RUNAHEAD, s->maxf);
      for (const auto& o : s->bopts)
        if (rc == VC_OK) rc = vc_batcher_set_option(b, o.first, o.second);
      if (rc == VC_OK && cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess) {
        cudaGetLastError();
        rc = VC_ERR_CUDA;
      }
      if (rc != VC_OK) {
        if (b) vc_batcher_destroy(b);
        return rc;
      }
      s->lane_b.push_back(b);
      s->lane_st.push_back(st);
    }
    return VC_OK;
  }
  if (!s->lane_b.empty()) return VC_ERR_ARG;  // batcher options come before the lanes
  const int rc = vc_batcher_set_option(s->b, option, value);
  if (rc == VC_OK) s->bopts.emplace_back(option, value);
  return rc;
}

int vc_dbg_server_stats(vc_server* s, double* ms6, int64_t* ticks) {
  if (!s || !ms6 || !ticks) return VC_ERR_ARG;
  for (int k = 0; k < 4; k++) {
    ms6[k] = s->host_ms[k];
    s->host_ms[k] = 0;
  }
  ms6[4] = s->gpu_ms;
  ms6[5] = (double)s->gpu_ticks;
  s->gpu_ms = 0;
  s->gpu_ticks = 0;
  *ticks = s->host_ticks;
  s->host_ticks = 0;
  return VC_OK;
}

int vc_dbg_server_record(vc_server* s, int32_t enable) {
  if (!s) return VC_ERR_ARG;
  s->rec = enable != 0;
  if (!s->rec) {
    s->rec_frames.clear();
    s->rec_ticks.clear();
  }
  return VC_OK;
}

int vc_dbg_server_take(vc_server* s, int32_t which, int32_t cap, double* out, int32_t* n) {
  if (!s || !n || (which != 0 && which != 1) || cap < 0 || (cap > 0 && !out)) return VC_ERR_ARG;
  std::vector<double>& v = which == 0 ? s->rec_frames : s->rec_ticks;
  const size_t k = std::min<size_t>((size_t)cap, v.size() / 4);
  std::copy(v.begin(), v.begin() + 4 * k, out);
  v.erase(v.begin(), v.begin() + 4 * k);
  *n = (int32_t)k;
  return VC_OK;
}

void vc_server_destroy(vc_server* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  for (cudaStream_t st : s->lane_st) cudaStreamSynchronize(st);
  for (SrvTick& tk : s->inflight) {
    if (tk.ev) cudaEventDestroy(tk.ev);
    if (tk.ev0) cudaEventDestroy(tk.ev0);
    for (cudaEvent_t e : tk.job_ev) cudaEventDestroy(e);
  }
  for (SrvStream& t : s->streams) {  // streams still registered: their contexts are alive
    if (t.active && t.ctx) {
      for (cudaStream_t ls : s->lane_st) vc::ctx_release_stream(t.ctx, ls);
      if (t.cs) vc::ctx_release_stream(t.ctx, t.cs);
    }
    if (t.cs) cudaStreamDestroy(t.cs);
    if (t.join) cudaEventDestroy(t.join);
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->t0) cudaEventDestroy(s->t0);
  if (s->b) vc_batcher_destroy(s->b);
  for (vc_batcher* b : s->lane_b) vc_batcher_destroy(b);
  for (cudaStream_t st : s->lane_st) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
