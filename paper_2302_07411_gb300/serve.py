"""Continuous-batching serving loop for the chaotic video cipher.

Video streams arrive over time (each with its own key, resolution, frame rate
and direction).  The loop admits a stream when its device memory fits the HBM
budget, keeps its key and chaotic state resident on the GPU, and every tick
gathers the frames that have arrived on all admitted streams into ONE ragged
batch (vc_batch_submit: one CUDA-graph replay for every stream, resolution and
direction).  Frames that arrive while earlier batches run join the next tick;
GPU work of consecutive ticks overlaps with the host's next gathering.  A
frame's latency is the device completion time of its batch minus the frame's
arrival time (CUDA event timestamps, so host polling adds nothing).  The
per-tick work (frame clocks of all streams, keystream readiness, the
submission, completion events) runs in libvcrypt's vc_server; this module
admits, registers and retires streams.

mode="perframe" is the comparison: the same loop, but each ready frame is
encrypted by its own encrypt_frames / decrypt_frames call (one launch sequence
per frame).
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import binding as B


def subframes_for(H: int) -> int:
    """The subframe count the serving configuration uses: n = ceil(H / 4)."""
    return max(1, math.ceil(H / 4))


# warps per SM-holding keystream CTA by map: PLCM and logistic chains are
# latency-bound (one warp per scheduler), 2DLASM chains share the SM's
# binary64 pipe (two warps)
HOLD_WARPS = {0: 4, 1: 2, 2: 4}

# map iterates per keystream byte: a PLCM or logistic pair emits 6 bytes per
# iterate of each of its two maps (Sec. 3), a 2DLASM pair 12 bytes per step
# of its two maps (Eq. 6: x then y)
ITERS_PER_BYTE = {0: 2.0 / 6.0, 1: 2.0 / 12.0, 2: 2.0 / 6.0}


def calibrate(kinds=(0, 1), use_cache: bool = True) -> dict:
    """Device rates that compute-aware admission charges streams against,
    measured on this GPU (CUDA events) and cached per GPU name:

    * ks_iter_per_s[kind]: map iterates per second of the keystream under
      serving load -- many streams' productions at once, each on its own CUDA
      stream in the kernel productions use (one-warp CTAs sharing the SMs):
      128 PLCM or 48 2DLASM streams of 768x768x3 with n = 192, one frame each;
    * chain_s_per_iter[kind]: the seconds one chain needs per iterate under
      that load (the serial limit of a single stream's chains);
    * rounds_px_per_s: pixels per second of the five rounds (1920x1080x3,
      n = 270, 8 frames, keystream not overlapped)."""
    import torch

    from . import autotune

    key = f"serve-calibration-v3|{autotune._gpu_name()}|{','.join(map(str, kinds))}"
    cache = autotune._load() if use_cache else {}
    if key in cache:
        return cache[key]
    out = {"ks_iter_per_s": {}, "chain_s_per_iter": {}, "chain_s_per_iter_held": {},
           "sms": torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count}
    H, W, C = 768, 768, 3
    n = subframes_for(H)
    N = H * W * C
    keys = {0: [0.31, 0.21, 0.62, 0.37], 1: [0.31, 0.6, 0.62], 2: [0.31, 3.95, 0.62, 3.99]}
    main = torch.cuda.current_stream()
    for kind in kinds:
        K = 48 if kind == 1 else 128
        ciphers, bufs, streams = [], [], []
        for i in range(K):
            c = B.Cipher(kind, keys[kind], H, W, C, n, 5)
            c.set_option(B.VC_OPT_OVERLAP, 0)
            c.set_option(B.VC_OPT_KS_SM_WARPS, 0)
            ciphers.append(c)
            bufs.append((torch.empty(5 * N, dtype=torch.uint8, device="cuda"),
                         torch.empty(1, dtype=torch.int64, device="cuda")))
            streams.append(torch.cuda.Stream())

        def produce_all():
            ev = torch.cuda.Event()
            ev.record(main)
            for c, (ks, sc), st in zip(ciphers, bufs, streams):
                st.wait_event(ev)
                B.vc_dbg_keystream(c.ctx, ks, sc, 1, stream=st)
            for st in streams:
                main.wait_stream(st)

        produce_all()  # warm-up (scratch allocation)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        produce_all()
        e1.record(main)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        for c in ciphers:
            c.close()
        per_chain = 5 * (N / n) * ITERS_PER_BYTE[kind] / 2  # iterates of one map chain per frame
        out["ks_iter_per_s"][str(kind)] = K * 2 * n * per_chain / sec
        out["chain_s_per_iter"][str(kind)] = sec / per_chain
        # one stream alone in CTAs that hold whole SMs (HOLD_WARPS warps each)
        c = B.Cipher(kind, keys[kind], H, W, C, n, 5)
        c.set_option(B.VC_OPT_KS_SM_WARPS, HOLD_WARPS[kind])
        ks, sc = bufs[0]
        B.vc_dbg_keystream(c.ctx, ks, sc, 1)
        torch.cuda.synchronize()
        B.enc_profile_enable(c.ctx, True)
        B.enc_profile_read(c.ctx)
        B.vc_dbg_keystream(c.ctx, ks, sc, 1)
        torch.cuda.synchronize()
        out["chain_s_per_iter_held"][str(kind)] = B.enc_profile_read(c.ctx)["keystream"]["ms"] * 1e-3 / per_chain
        c.close()
    Hr, Wr = 1080, 1920
    x = torch.zeros((8, Hr, Wr, 3), dtype=torch.uint8, device="cuda")
    c = B.Cipher(0, keys[0], Hr, Wr, 3, subframes_for(Hr), 5)
    c.set_option(B.VC_OPT_OVERLAP, 0)
    c.encrypt(x, x)
    torch.cuda.synchronize()
    B.enc_profile_enable(c.ctx, True)
    B.enc_profile_read(c.ctx)
    c.encrypt(x, x)
    torch.cuda.synchronize()
    prof = B.enc_profile_read(c.ctx)
    c.close()
    out["rounds_px_per_s"] = 8 * Hr * Wr / (prof["rounds"]["ms"] * 1e-3)
    cache = autotune._load()
    cache[key] = out
    autotune._store(cache)
    return out


class ComputeBudget:
    """Compute-aware admission and keystream placement.  A stream whose own
    chains, sharing the SMs under load, would be busy more than `hold_above`
    of its frame period gets its keystream in CTAs that hold whole SMs
    (VC_OPT_KS_SM_WARPS); it is refused when even there one chain's iterates
    per frame times the calibrated seconds per iterate, times the frame rate,
    exceed `chain_busy_max` (a chain is serial; its frames' keystream is
    produced ahead).  Each admitted stream is charged the fraction of the
    device it keeps busy -- its keystream iterates per second over the
    calibrated rate of its map (held: its SMs' share of the device), plus its
    pixels per second over the rounds' rate -- against `target`."""

    def __init__(self, rates: dict, target: float = 0.8, chain_busy_max: float = 0.6, hold_above: float = 0.5):
        self.rates, self.target = rates, target
        self.chain_busy_max, self.hold_above = chain_busy_max, hold_above
        self.used = 0.0

    def plan(self, spec: dict) -> dict:
        H, W, C, kind, fps = spec["H"], spec["W"], spec["C"], spec["kind"], float(spec["fps"])
        P = H * W
        n = subframes_for(H)
        S = P * C / n  # bytes per subframe
        it_chain = 5 * S * ITERS_PER_BYTE[kind] / 2  # iterates of one map chain per frame
        k = str(kind)
        busy = fps * it_chain * self.rates["chain_s_per_iter"][k]
        hold = 0
        ks_load = fps * 2 * n * it_chain / self.rates["ks_iter_per_s"][k]
        if busy > self.hold_above and "chain_s_per_iter_held" in self.rates:
            hold = HOLD_WARPS[kind]
            busy = fps * it_chain * self.rates["chain_s_per_iter_held"][k]
            ctas = -(-2 * n // (32 * hold))
            ks_load = ctas * busy / float(self.rates.get("sms", 152))
        return {"load": ks_load + fps * P / self.rates["rounds_px_per_s"], "busy": busy, "hold": hold}

    def cost(self, spec: dict) -> tuple[float, float]:
        p = self.plan(spec)
        return p["load"], p["busy"]

    def admit(self, spec: dict) -> tuple[bool, float, str]:
        p = self.plan(spec)
        if p["busy"] > self.chain_busy_max:
            return False, 0.0, "chain"
        if self.used + p["load"] > self.target:
            return False, 0.0, "load"
        self.used += p["load"]
        return True, p["load"], ""

    def release(self, load: float) -> None:
        self.used = max(0.0, self.used - load)


@dataclass
class Stream:
    spec: dict
    cipher: B.Cipher
    out: object                      # device ring of output frames
    bytes: int
    frames_total: int = 0
    sid: int = -1                    # handle in the native server
    load: float = 0.0                # device fraction charged by the compute budget


@dataclass
class ServeResult:
    mode: str
    latencies_ms: list = field(default_factory=list)
    arrivals_s: list = field(default_factory=list)   # frame arrival time of each latency sample
    first_frame_ms: list = field(default_factory=list)  # per stream: latency of its first frame
    frames: int = 0
    admitted: int = 0
    rejected: int = 0      # HBM budget
    rejected_load: int = 0   # compute budget: the device is full
    rejected_chain: int = 0  # compute budget: the stream's own chains cannot keep up
    failed: int = 0        # admitted streams whose context could not be created (error kept in `errors`)
    errors: list = field(default_factory=list)
    peak_streams: int = 0
    wall_s: float = 0.0
    ticks: int = 0
    tick_host_ms: list = field(default_factory=list)  # host time of each loop iteration that submitted work
    native_ms: dict = field(default_factory=dict)      # host ms per part of the native ticks
    frame_records: object = None  # [k, 4]: stream, arrival, submission, completion (s), when recorded
    stream_info: dict = field(default_factory=dict)  # when recorded: native stream id -> (kind, H, W, fps, direction, hold)
    tick_records: object = None   # [m, 4]: submission, device start, device end (s), frames

    def latency_split(self, steady_after_s: float = 0.0) -> dict:
        """Per-frame latency split at the submission (frames arriving after
        steady_after_s): the wait from arrival to the tick that submitted the
        frame (frame clock, keystream readiness, tick cadence) and the device
        time from that tick to completion; per tick, the device time and the
        delay from submission to the device starting it."""
        if self.frame_records is None or not len(self.frame_records):
            return {}
        fr = self.frame_records[self.frame_records[:, 1] >= steady_after_s]
        tk = self.tick_records
        q = lambda a, p: round(float(np.percentile(a, p)) * 1e3, 3) if len(a) else None
        wait, dev = fr[:, 2] - fr[:, 1], fr[:, 3] - fr[:, 2]
        out = {"frames": int(len(fr)), "wait_p50_ms": q(wait, 50), "wait_p99_ms": q(wait, 99),
               "device_p50_ms": q(dev, 50), "device_p99_ms": q(dev, 99)}
        if tk is not None and len(tk):
            tk = tk[tk[:, 0] >= steady_after_s]
            out.update({"ticks": int(len(tk)), "tick_device_p50_ms": q(tk[:, 2] - tk[:, 1], 50),
                        "tick_device_p99_ms": q(tk[:, 2] - tk[:, 1], 99),
                        "tick_queue_p99_ms": q(tk[:, 1] - tk[:, 0], 99)})
        return out

    def summary(self, steady_after_s: float | None = None) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        out = {"mode": self.mode, "frames": self.frames, "fps": round(self.frames / max(self.wall_s, 1e-9), 1),
               "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
               "max_ms": round(float(lat.max()), 3), "admitted": self.admitted, "rejected": self.rejected,
               "rejected_load": self.rejected_load, "rejected_chain": self.rejected_chain, "failed": self.failed, "peak_concurrent_streams": self.peak_streams, "ticks": self.ticks}
        if self.first_frame_ms:
            out["first_frame_p99_ms"] = round(float(np.percentile(self.first_frame_ms, 99)), 3)
        if self.tick_host_ms:
            out["tick_host_p50_ms"] = round(float(np.percentile(self.tick_host_ms, 50)), 3)
            out["tick_host_p99_ms"] = round(float(np.percentile(self.tick_host_ms, 99)), 3)
        if self.native_ms.get("ticks"):
            t = self.native_ms["ticks"]
            out["native_tick_ms"] = {k: round(v / t, 4) for k, v in self.native_ms.items()
                                     if k not in ("ticks", "gpu_ms_per_tick")}
            out["gpu_ms_per_tick"] = round(self.native_ms.get("gpu_ms_per_tick", 0.0), 4)
        if steady_after_s is not None:
            arr = np.array(self.arrivals_s)
            sel = lat[arr >= steady_after_s] if len(arr) == len(lat) else lat
            if sel.size:
                out["steady_after_s"] = steady_after_s
                out["steady_frames"] = int(sel.size)
                out["steady_p50_ms"] = round(float(np.percentile(sel, 50)), 3)
                out["steady_p99_ms"] = round(float(np.percentile(sel, 99)), 3)
        return out


def tune_shapes(requests) -> dict:
    """The autotuner's choice (rows per round-kernel tile, by the rounds'
    device time; cached per GPU) for every shape class (kind, H, W, C) of
    the requests, with n = ceil(H/4): {(kind, H, W, C): {"tile_rows": T}}."""
    from . import autotune

    out = {}
    for r in requests:
        k = (r["kind"], r["H"], r["W"], r["C"])
        if k not in out:
            out[k] = autotune.tune_rounds(r["kind"], r["H"], r["W"], r["C"], subframes_for(r["H"]))["options"]
    return out


class Server:
    """Runs a list of stream requests (synth.serving_workload) in real time."""

    def __init__(self, hbm_budget_bytes: int = 64 << 30, tick_ms: float = 4.0, mode: str = "batch",
                 max_frames_per_tick: int | None = None, ring: int = 8, keep_outputs: bool = False,
                 cipher_options: dict | None = None, compute: ComputeBudget | None = None,
                 setup_lead_s: float = 0.0, tuned: dict | None = None, record: bool = False,
                 server_options: dict | None = None, priority: int | None = None):
        """compute: admission also charges each stream's device load (None:
        HBM budget only).  setup_lead_s: a request is admitted this long
        before its first frame arrives (the session's setup), so its context
        and, when batching, its first frames' keystream exist by then.
        tuned: per shape class (kind, H, W, C) the options the autotuner
        chose (tune_shapes), applied to each stream's context.  record: keep
        per-frame and per-tick latency records (ServeResult.latency_split).
        max_frames_per_tick: frames of one stream per tick; when batching also
        the keystream run-ahead (default 2 batching, 4 per frame).
        server_options: options of a batching server (VC_BOPT_*,
        VC_SOPT_QUEUED_TICKS) over the defaults below.
        priority: of the server's CUDA stream (torch's convention: lower is
        more urgent).  Batching defaults: the server's stream above the
        default priority and the keystream productions at the device's lowest
        (VC_BOPT_KS_PRIORITY 1), so that the SMs a long production frees go
        to the ticks' round kernels first, whose frames are due; measured on
        the 768x768 capacity and mixed workloads, this halves the first-frame
        latency at equal steady-state latency.  Two tick lanes
        (VC_SOPT_LANES 2): consecutive ticks on two batchers and streams, so
        that a tick whose round kernels wait for SMs does not hold up the
        next one (320 streams of 768x768 at p99 12 ms with two lanes, 392 ms
        with one, in the same run).  Urgent productions (VC_BOPT_KS_URGENT
        1: a stream with no frame produced ahead gets its next production on
        a stream of the highest priority) are left off: in an A/B of three
        repeats both held 320 streams of 768x768 at p99 12 ms, and past the
        capacity (384) the urgent form collapsed further (p99 1.2-1.4 s
        against 0.4-0.9 s)."""
        import torch

        self.torch = torch
        self.compute = compute
        self.lead = setup_lead_s
        self.tuned = dict(tuned or {})
        self.cipher_options = dict(cipher_options or {})  # enc_set_option values for every stream
        self.budget = hbm_budget_bytes
        self.tick = tick_ms / 1e3
        self.mode = mode
        batching = mode == "batch"
        self.maxf = max_frames_per_tick if max_frames_per_tick is not None else (2 if batching else 4)
        self.ring = ring
        defaults = {B.VC_BOPT_KS_PRIORITY: 1, B.VC_SOPT_LANES: 2} if batching else {}
        self.server_options = defaults | dict(server_options or {})
        if priority is None:
            priority = -1 if batching else 0
        self.stream = torch.cuda.Stream(priority=priority)

        self.inputs = {}  # (H, W, C) -> device frames reused as input content
        from concurrent.futures import ThreadPoolExecutor

        self.pool = ThreadPoolExecutor(max_workers=2)
        self.keep = keep_outputs
        self.record = record
        self.finished: list[Stream] = []  # kept when keep_outputs (tests)

    def _open(self, spec: dict, fp: int) -> Stream:
        torch = self.torch
        H, W, C = spec["H"], spec["W"], spec["C"]
        ciph = B.Cipher(spec["kind"], spec["key"], H, W, C, subframes_for(H), 5)
        for opt, val in self.cipher_options.items():
            ciph.set_option(opt, val)
        tuned = self.tuned.get((spec["kind"], H, W, C))
        if tuned:
            ciph.set_option(B.VC_OPT_TILE_ROWS, int(tuned.get("tile_rows", 0)))
        if self.compute is not None:
            hold = self.compute.plan(spec)["hold"]
            if hold:
                ciph.set_option(B.VC_OPT_KS_SM_WARPS, hold)
        out = torch.empty((self.ring, H, W, C), dtype=torch.uint8, device="cuda")
        return Stream(spec, ciph, out, fp, frames_total=max(1, int(spec["duration"] * spec["fps"])))

    def input_frames(self, H, W, C):
        """Input content: frame k of a stream of this size is input_frames[k % maxf]
        (2 * maxf frames are kept so m <= maxf consecutive frames are contiguous)."""
        key = (H, W, C)
        if key not in self.inputs:
            rng = np.random.default_rng(H * 7 + W)
            base = rng.integers(0, 256, size=(self.maxf, H, W, C), dtype=np.uint8)
            self.inputs[key] = self.torch.from_numpy(np.concatenate([base, base])).cuda()
        return self.inputs[key]

    @staticmethod
    def footprint(spec: dict, ring: int, maxf: int) -> int:
        """Device bytes a stream holds while admitted: its output ring, its
        state, and its share of the batch scratch (keystream, buffers)."""
        N = spec["H"] * spec["W"] * spec["C"]
        n = subframes_for(spec["H"])
        state = n * (6 * 8 + 20) + (spec["H"] * spec["W"] // 32 + 2) * 8
        scratch = maxf * (5 + 2) * ((N + 255) // 256 * 256)
        return ring * N + state + scratch

    def run(self, requests: list[dict], horizon_s: float | None = None) -> ServeResult:
        """Real-time loop: admissions and retirements here, the per-tick work
        (frame clocks, keystream readiness, one submission per tick, completion
        events) in libvcrypt's vc_server."""
        torch = self.torch
        res = ServeResult(self.mode)
        pending = deque(sorted(requests, key=lambda r: r["arrival"]))
        lead = self.lead
        starting = deque()  # futures of streams whose context is being created
        active: dict[int, Stream] = {}
        used = 0
        torch.cuda.synchronize()
        srv = B.NativeServer(0 if self.mode == "batch" else 1, self.maxf, self.stream)
        if self.record:
            srv.record(True)
        if self.mode == "batch":  # the lanes last: they copy the batcher options set before them
            for opt, val in sorted(self.server_options.items(), key=lambda kv: kv[0] == B.VC_SOPT_LANES):
                srv.set_option(opt, val)
        t0 = time.perf_counter()  # the server's time origin was just recorded
        end_time = horizon_s if horizon_s is not None else max(
            (r["arrival"] + r["duration"] for r in requests), default=0.0)

        def drain(block: bool):
            ids, frames, arr, lat = srv.drain(block)
            res.latencies_ms.extend(lat.tolist())
            res.arrivals_s.extend(arr.tolist())
            res.frames += len(lat)
            first = frames == 0
            res.first_frame_ms.extend(lat[first].tolist())

        try:
            while True:
                t_iter = time.perf_counter()
                now = t_iter - t0
                # admissions (HBM budget, then the compute budget)
                while pending and pending[0]["arrival"] - lead <= now:
                    spec = pending.popleft()
                    fp = self.footprint(spec, self.ring, self.maxf)
                    if used + fp > self.budget:
                        res.rejected += 1
                        continue
                    load = 0.0
                    if self.compute is not None:
                        ok, load, why = self.compute.admit(spec)
                        if not ok:
                            if why == "chain":
                                res.rejected_chain += 1
                            else:
                                res.rejected_load += 1
                            continue
                    used += fp
                    res.admitted += 1
                    # context creation (key schedule on the GPU) off the loop's thread
                    starting.append((self.pool.submit(self._open, spec, fp), fp, load))
                while starting and starting[0][0].done():
                    fut, fp, load = starting.popleft()
                    try:
                        st = fut.result()
                    except Exception as e:  # e.g. a key outside the valid ranges: this stream only
                        res.failed += 1
                        res.errors.append(f"{type(e).__name__}: {e}")
                        used -= fp
                        if self.compute is not None:
                            self.compute.release(load)
                        continue
                    st.load = load
                    H, W, C = st.spec["H"], st.spec["W"], st.spec["C"]
                    st.sid = srv.add(st.cipher, st.spec["direction"], H * W * C, self.input_frames(H, W, C),
                                     self.maxf, st.out, self.ring, float(st.spec["fps"]), st.spec["arrival"],
                                     st.frames_total)
                    active[st.sid] = st
                    if self.record:
                        sp = st.spec
                        res.stream_info[st.sid] = (sp["kind"], H, W, sp["fps"], sp["direction"],
                                                   self.compute.plan(sp)["hold"] if self.compute else 0)
                res.peak_streams = max(res.peak_streams, len(active))
                if srv.tick(now) > 0:
                    res.ticks += 1
                    res.tick_host_ms.append((time.perf_counter() - t_iter) * 1e3)
                drain(block=False)
                # retire streams whose last frame is done
                for sid, st in list(active.items()):
                    last_arrival = st.spec["arrival"] + (st.frames_total - 1) / st.spec["fps"]
                    if now >= last_arrival and srv.stream_done(sid):
                        srv.remove(sid)
                        used -= st.bytes
                        if self.compute is not None:
                            self.compute.release(st.load)
                        del active[sid]
                        if self.keep:
                            self.finished.append(st)
                        else:
                            st.cipher.close(wait=False)  # its frames are done; run-ahead keystream may still run
                if not pending and not active and not starting and srv.inflight() == 0:
                    break
                if now > end_time + 5.0:  # safety: stop a run that cannot keep up
                    break
                nxt = self.tick - ((time.perf_counter() - t0) % self.tick)
                time.sleep(max(0.0, nxt))
            drain(block=True)
        finally:
            res.wall_s = time.perf_counter() - t0
            res.native_ms = srv.host_stats()
            if self.record:
                res.frame_records, res.tick_records = srv.take_records()
            for sid, st in active.items():
                srv.remove(sid)  # before its context goes: the server forgets it
                if self.keep:
                    self.finished.append(st)
                else:
                    st.cipher.close()
            srv.close()
        return res

    def close(self):
        self.pool.shutdown(wait=True)


def capacity(mode: str, H: int, W: int, fps: int = 24, budget_ms: float = 1000.0 / 24.0,
             counts=(16, 32, 64, 128, 256, 512), seconds: float = 4.0, seed: int = 21,
             hbm_budget_bytes: int = 200 << 30, tick_ms: float = 4.0, ramp_s: float = 0.5,
             warm_s: float = 1.0, cipher_options: dict | None = None, kinds=(0, 1)) -> dict:
    """Largest number of concurrent fps streams of H x W x 3 (half encrypt,
    half decrypt, maps cycling through `kinds`: PLCM 0, 2DLASM 1) whose
    steady-state per-frame p99 latency stays below budget_ms.  Streams arrive
    uniformly over ramp_s seconds and last `seconds`; "steady" counts the
    frames arriving after ramp_s + warm_s.  Time to first frame is reported
    separately."""
    import synth

    best, runs = 0, []
    steady_from = ramp_s + warm_s
    # one short untimed run first, as large as the first count: one-time
    # costs (module loading, the memory pool's growth, shared-memory
    # configuration) stay out of the search
    nw = counts[0] if counts else 1
    warm = synth.serving_workload(nw, seed=seed + 1, rate_per_s=nw / ramp_s, resolutions=((H, W),),
                                  fps_choices=(fps,), duration_s=(1.0, 1.0))
    srv = Server(hbm_budget_bytes=hbm_budget_bytes, tick_ms=tick_ms, mode=mode, cipher_options=cipher_options)
    srv.run(warm)
    srv.close()
    for n in counts:
        reqs = synth.serving_workload(n, seed=seed, rate_per_s=n / ramp_s, resolutions=((H, W),),
                                      fps_choices=(fps,), duration_s=(seconds, seconds))
        for k, r in enumerate(reqs):  # maps cycle through `kinds`, each stream keyed for its map
            kind = kinds[k % len(kinds)]
            if r["kind"] != kind:
                r["kind"] = kind
                r["key"] = synth.key_for_seed(kind, 1000 + r["sid"])
        srv = Server(hbm_budget_bytes=hbm_budget_bytes, tick_ms=tick_ms, mode=mode, cipher_options=cipher_options)
        res = srv.run(reqs)
        srv.close()
        s = res.summary(steady_after_s=steady_from)
        s["streams"] = n
        runs.append(s)
        p99 = s.get("steady_p99_ms", s["p99_ms"])
        if s["rejected"] == 0 and p99 < budget_ms:
            best = n
        else:
            break
    return {"mode": mode, "resolution": f"{H}x{W}x3", "fps": fps, "p99_budget_ms": round(budget_ms, 2),
            "criterion": f"p99 of frames arriving after {steady_from:g} s (admission ramp {ramp_s:g} s)",
            "max_streams": best, "runs": runs}


def serve_mixed(mode: str, nstreams: int = 256, rate_per_s: float = 64.0, seed: int = 5,
                targets=(1.0, 0.95, 0.9, 0.8, 0.7, 0.55, 0.4), budget_ms: float = 1000.0 / 24.0,
                hbm_budget_bytes: int = 160 << 30, setup_lead_s: float = 0.1, rates: dict | None = None,
                steady_after_s: float = 1.5, server_kw: dict | None = None) -> dict:
    """The mixed serving workload: nstreams requests arriving as a Poisson
    process (rate_per_s), resolutions 480^2 ... 3840x2160, 24 / 30 / 60 FPS,
    PLCM and 2DLASM alternating, half encrypt and half decrypt, n = ceil(H/4)
    (synth.serving_workload).  Served with compute-aware admission at the
    given load targets in turn, until the steady-state p99 per-frame latency of
    the admitted streams is under budget_ms; every run is reported (admitted,
    rejected by memory / device load / chain rate, p50 / p99, first-frame p99,
    frames/s).  Requests are admitted setup_lead_s before their first frame."""
    import synth

    rates = rates or calibrate()
    reqs = synth.serving_workload(nstreams, seed=seed, rate_per_s=rate_per_s)
    tuned = tune_shapes(reqs)
    runs, best = [], None
    for t in targets:
        srv = Server(hbm_budget_bytes=hbm_budget_bytes, mode=mode, compute=ComputeBudget(rates, target=t),
                     setup_lead_s=setup_lead_s, tuned=tuned, record=True, **(server_kw or {}))
        res = srv.run(reqs)
        srv.close()
        summ = res.summary(steady_after_s=steady_after_s)
        summ["load_target"] = t
        summ["split"] = res.latency_split(steady_after_s)
        runs.append(summ)
        if summ.get("steady_p99_ms", summ["p99_ms"]) < budget_ms:
            best = summ
            break
    return {"mode": mode, "requests": nstreams, "rate_per_s": rate_per_s, "p99_budget_ms": round(budget_ms, 2),
            "setup_lead_s": setup_lead_s,
            "tuned": {f"{k[0]}:{k[1]}x{k[2]}x{k[3]}": v for k, v in tuned.items()},
            "admitted_within_budget": best["admitted"] if best else 0,
            "load_target": best["load_target"] if best else None, "runs": runs}


def batch_mix(nstreams: int = 64, ticks: int = 8, warm: int = 3, split: int = -1, rates: dict | None = None) -> dict:
    """Ragged batches against one call per frame.  nstreams streams, each with
    its own key, resolutions cycling 480^2, 576^2, 768^2 and 1920x1080
    (n = ceil(H/4)), maps and directions alternating, one frame per stream per
    tick.  Four forms, each on its own contexts:

    * batched_inline: one vc_batch_submit per tick with the keystream inside
      it (one graph replay: schedule, keystream, rounds, fix-up of every
      stream; long chains in the second lane per `split`);
    * batched_runahead: one vc_batch_submit per tick of rounds only, each
      stream's keystream produced one frame ahead on its own internal stream
      (SM-holding CTAs for the streams whose chains the compute budget says
      need them at 24 FPS);
    * per_frame: encrypt_frames / decrypt_frames per stream, each on its own
      CUDA stream, the next call's keystream generated ahead (the default);
    * per_frame_inline: the same without that run-ahead.

    Time per tick = host wall time over `ticks` ticks between two device-wide
    synchronisations after `warm` ticks, so that keystream generated ahead on
    the contexts' internal streams is counted in the tick that issued it.  The
    outputs of the last tick are compared byte for byte across the forms."""
    import torch

    import synth

    res = [(480, 480), (576, 576), (768, 768), (1080, 1920)]
    specs = []
    for s_ in range(nstreams):
        H, W = res[s_ % len(res)]
        kind, direction = (s_ // 4) % 2, (s_ // 8) % 2
        specs.append((kind, direction, synth.key_for_seed(kind, 900 + s_), H, W, subframes_for(H)))
    frames = {}
    for (_, _, _, H, W, _) in specs:
        if (H, W) not in frames:
            frames[(H, W)] = torch.from_numpy(synth.uniform_frames(1, H, W, 3, seed=H + W)).cuda()
    from . import autotune

    # the autotuner's tile rows per shape class, the same for every form
    tuned = {}
    for (k, d, key, H, W, n) in specs:
        if (k, H, W) not in tuned:
            tuned[(k, H, W)] = autotune.tune_rounds(k, H, W, 3, n)["options"]["tile_rows"]
    budget = ComputeBudget(rates or calibrate())
    hold = {(k, H, W): budget.plan({"kind": k, "H": H, "W": W, "C": 3, "fps": 24})["hold"]
            for (k, H, W) in tuned}

    def contexts():
        cs = [B.Cipher(k, key, H, W, 3, n, 5) for (k, d, key, H, W, n) in specs]
        for c, (k, d, key, H, W, n) in zip(cs, specs):
            c.set_option(B.VC_OPT_TILE_ROWS, tuned[(k, H, W)])
        return cs

    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in specs]

    def form_batched(runahead):
        cs = contexts()
        if runahead:
            for c, (k, d, key, H, W, n) in zip(cs, specs):
                if hold[(k, H, W)]:
                    c.set_option(B.VC_OPT_KS_SM_WARPS, hold[(k, H, W)])
        out = [torch.empty_like(frames[(H, W)]) for (_, _, _, H, W, _) in specs]
        batcher = B.Batcher(graph=True, runahead=runahead)
        B.vc_batcher_set_option(batcher.b, B.VC_BOPT_SPLIT, split)

        def tick():
            batcher.submit([(c, sp[1], frames[(sp[3], sp[4])], out[j], 1) for j, (c, sp) in enumerate(zip(cs, specs))],
                           stream=main)
        return cs, out, tick, batcher

    def form_single(runahead):
        cs = contexts()
        if not runahead:
            for c in cs:
                c.set_option(B.VC_OPT_RUNAHEAD_CALLS, 0)
        out = [torch.empty_like(frames[(H, W)]) for (_, _, _, H, W, _) in specs]

        def tick():
            ev = torch.cuda.Event()
            ev.record(main)
            for j, (c, sp) in enumerate(zip(cs, specs)):
                st = streams[j]
                st.wait_event(ev)
                x = frames[(sp[3], sp[4])]
                if sp[1] == 0:
                    c.encrypt(x, out[j], stream=st)
                else:
                    c.decrypt(x, out[j], stream=st)
            for st in streams:
                main.wait_stream(st)
        return cs, out, tick, None

    def timed(fn):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ticks):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / ticks

    ms, outs, long_jobs = {}, {}, 0
    for name, make, arg in (("batched_inline", form_batched, 0), ("batched_runahead", form_batched, 1),
                            ("per_frame", form_single, True), ("per_frame_inline", form_single, False)):
        cs, out, tick, batcher = make(arg)
        ms[name] = timed(tick)
        if name == "batched_inline":
            long_jobs = B.lib().vc_dbg_batch_split(batcher.b)
        outs[name] = out
        if batcher is not None:
            batcher.close()
        for c in cs:
            c.close()
    ref = outs["per_frame"]
    same = {k: all(torch.equal(x, y) for x, y in zip(v, ref)) for k, v in outs.items()}
    px = sum(H * W for (_, _, _, H, W, _) in specs)
    return {"streams": nstreams, "resolutions": ["480x480", "576x576", "768x768", "1080x1920"],
            "ticks": ticks, "timing": "host wall time between device-wide synchronisations",
            "ms_per_tick": {k: round(v, 3) for k, v in ms.items()},
            "mpixel_s": {k: round(px / v / 1e3, 1) for k, v in ms.items()},
            "batched_ms_per_tick": round(ms["batched_inline"], 3), "per_frame_ms_per_tick": round(ms["per_frame"], 3),
            "outputs_equal": bool(all(same.values())), "batch_long_lane_jobs": int(long_jobs),
            "held_keystream": {f"{k}:{H}x{W}": v for (k, H, W), v in hold.items() if v},
            "tuned_tile_rows": {f"{k}:{H}x{W}": v for (k, H, W), v in tuned.items()}}


def main():
    import argparse
    import json
    import os

    # per-stream keystream production runs on one CUDA stream per served
    # stream: more hardware work queues than the default 8 (read when the CUDA
    # context is created)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    import synth

    ap = argparse.ArgumentParser(description="serving loop measurements")
    ap.add_argument("--mode", choices=["batch", "perframe", "both"], default="both")
    ap.add_argument("--streams", type=int, default=256)
    ap.add_argument("--rate", type=float, default=64.0, help="stream arrivals per second (Poisson)")
    ap.add_argument("--capacity", action="store_true", help="search the 24 FPS stream capacity instead")
    ap.add_argument("--size", type=int, nargs=2, default=[768, 768])
    ap.add_argument("--seconds", type=float, default=4.0)
    ap.add_argument("--budget-gb", type=float, default=160.0)
    ap.add_argument("--batch-mix", type=int, default=0, metavar="N",
                    help="instead: N streams of mixed resolutions, one batch per tick against one call per frame")
    ap.add_argument("--ticks", type=int, default=8, help="timed ticks of --batch-mix")
    ap.add_argument("--warm", type=int, default=3, help="untimed ticks of --batch-mix before the timed ones")
    ap.add_argument("--split", type=int, default=-1, help="VC_BOPT_SPLIT of --batch-mix")
    ap.add_argument("--mixed", action="store_true",
                    help="instead: the mixed Poisson workload with compute-aware admission (both modes)")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    from . import build

    build.build()
    if a.batch_mix:
        print(json.dumps(batch_mix(a.batch_mix, ticks=a.ticks, warm=a.warm, split=a.split)))
        return
    if a.mixed:
        rates = calibrate()
        print(json.dumps({"calibration": rates, **{m: serve_mixed(m, nstreams=a.streams, rate_per_s=a.rate, rates=rates)
                                                   for m in (["batch", "perframe"] if a.mode == "both" else [a.mode])}}))
        return
    modes = ["batch", "perframe"] if a.mode == "both" else [a.mode]
    out = {}
    for mode in modes:
        if a.capacity:
            out[mode] = capacity(mode, a.size[0], a.size[1], seconds=a.seconds,
                                 hbm_budget_bytes=int(a.budget_gb * (1 << 30)))
        else:
            reqs = synth.serving_workload(a.streams, rate_per_s=a.rate)
            srv = Server(hbm_budget_bytes=int(a.budget_gb * (1 << 30)), mode=mode)
            res = srv.run(reqs)
            srv.close()
            out[mode] = res.summary(steady_after_s=1.5)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
