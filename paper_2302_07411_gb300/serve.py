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


@dataclass
class Stream:
    spec: dict
    cipher: B.Cipher
    out: object                      # device ring of output frames
    bytes: int
    frames_total: int = 0
    sid: int = -1                    # handle in the native server


@dataclass
class ServeResult:
    mode: str
    latencies_ms: list = field(default_factory=list)
    arrivals_s: list = field(default_factory=list)   # frame arrival time of each latency sample
    first_frame_ms: list = field(default_factory=list)  # per stream: latency of its first frame
    frames: int = 0
    admitted: int = 0
    rejected: int = 0
    failed: int = 0        # admitted streams whose context could not be created (error kept in `errors`)
    errors: list = field(default_factory=list)
    peak_streams: int = 0
    wall_s: float = 0.0
    ticks: int = 0
    tick_host_ms: list = field(default_factory=list)  # host time of each loop iteration that submitted work
    native_ms: dict = field(default_factory=dict)      # host ms per part of the native ticks

    def summary(self, steady_after_s: float | None = None) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        out = {"mode": self.mode, "frames": self.frames, "fps": round(self.frames / max(self.wall_s, 1e-9), 1),
               "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
               "max_ms": round(float(lat.max()), 3), "admitted": self.admitted, "rejected": self.rejected,
               "failed": self.failed, "peak_concurrent_streams": self.peak_streams, "ticks": self.ticks}
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


class Server:
    """Runs a list of stream requests (synth.serving_workload) in real time."""

    def __init__(self, hbm_budget_bytes: int = 64 << 30, tick_ms: float = 4.0, mode: str = "batch",
                 max_frames_per_tick: int = 4, ring: int = 8, keep_outputs: bool = False,
                 cipher_options: dict | None = None):
        import torch

        self.torch = torch
        self.cipher_options = dict(cipher_options or {})  # enc_set_option values for every stream
        self.budget = hbm_budget_bytes
        self.tick = tick_ms / 1e3
        self.mode = mode
        self.maxf = max_frames_per_tick
        self.ring = ring
        self.stream = torch.cuda.Stream()

        self.inputs = {}  # (H, W, C) -> device frames reused as input content
        from concurrent.futures import ThreadPoolExecutor

        self.pool = ThreadPoolExecutor(max_workers=2)
        self.keep = keep_outputs
        self.finished: list[Stream] = []  # kept when keep_outputs (tests)

    def _open(self, spec: dict, fp: int) -> Stream:
        torch = self.torch
        H, W, C = spec["H"], spec["W"], spec["C"]
        ciph = B.Cipher(spec["kind"], spec["key"], H, W, C, subframes_for(H), 5)
        for opt, val in self.cipher_options.items():
            ciph.set_option(opt, val)
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
        starting = deque()  # futures of streams whose context is being created
        active: dict[int, Stream] = {}
        used = 0
        torch.cuda.synchronize()
        srv = B.NativeServer(0 if self.mode == "batch" else 1, self.maxf, self.stream)
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
                # admissions (HBM budget)
                while pending and pending[0]["arrival"] <= now:
                    spec = pending.popleft()
                    fp = self.footprint(spec, self.ring, self.maxf)
                    if used + fp > self.budget:
                        res.rejected += 1
                        continue
                    used += fp
                    res.admitted += 1
                    # context creation (key schedule on the GPU) off the loop's thread
                    starting.append((self.pool.submit(self._open, spec, fp), fp))
                while starting and starting[0][0].done():
                    fut, fp = starting.popleft()
                    try:
                        st = fut.result()
                    except Exception as e:  # e.g. a key outside the valid ranges: this stream only
                        res.failed += 1
                        res.errors.append(f"{type(e).__name__}: {e}")
                        used -= fp
                        continue
                    H, W, C = st.spec["H"], st.spec["W"], st.spec["C"]
                    st.sid = srv.add(st.cipher, st.spec["direction"], H * W * C, self.input_frames(H, W, C),
                                     self.maxf, st.out, self.ring, float(st.spec["fps"]), st.spec["arrival"],
                                     st.frames_total)
                    active[st.sid] = st
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
                        del active[sid]
                        if self.keep:
                            self.finished.append(st)
                        else:
                            st.cipher.close()
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
            for st in active.values():
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
    # one short untimed run first: one-time costs (module loading, first
    # allocations, shared-memory configuration) stay out of the search
    warm = synth.serving_workload(1, seed=seed, rate_per_s=1.0 / ramp_s, resolutions=((H, W),),
                                  fps_choices=(fps,), duration_s=(0.5, 0.5))
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


def batch_mix(nstreams: int = 64, ticks: int = 6, warm: int = 2) -> dict:
    """Ragged batches against one call per frame.  nstreams streams, each with
    its own key, resolutions cycling 480^2, 576^2, 768^2 and 1920x1080
    (n = ceil(H/4)), maps and directions alternating, one frame per stream per
    tick.  Batched: one vc_batch_submit per tick (one graph replay; keystream,
    rounds and fix-up of every stream inside it).  Per frame: encrypt_frames /
    decrypt_frames per stream, each stream on its own CUDA stream.  Device time
    per tick by CUDA events after `warm` ticks; the outputs of the two forms
    are compared byte for byte after the last tick."""
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
    batched = [B.Cipher(k, key, H, W, 3, n, 5) for (k, d, key, H, W, n) in specs]
    single = [B.Cipher(k, key, H, W, 3, n, 5) for (k, d, key, H, W, n) in specs]
    out_b = [torch.empty_like(frames[(H, W)]) for (_, _, _, H, W, _) in specs]
    out_s = [torch.empty_like(frames[(H, W)]) for (_, _, _, H, W, _) in specs]
    streams = [torch.cuda.Stream() for _ in specs]
    main = torch.cuda.current_stream()
    batcher = B.Batcher(graph=True)

    def tick_batched():
        batcher.submit([(c, sp[1], frames[(sp[3], sp[4])], out_b[j], 1) for j, (c, sp) in enumerate(zip(batched, specs))],
                       stream=main)

    def tick_single():
        ev = torch.cuda.Event()
        ev.record(main)
        for j, (c, sp) in enumerate(zip(single, specs)):
            st = streams[j]
            st.wait_event(ev)
            x = frames[(sp[3], sp[4])]
            if sp[1] == 0:
                c.encrypt(x, out_s[j], stream=st)
            else:
                c.decrypt(x, out_s[j], stream=st)
        for st in streams:
            main.wait_stream(st)

    def timed(fn):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        for _ in range(ticks):
            fn()
        b.record(main)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / ticks

    ms_b = timed(tick_batched)
    ms_s = timed(tick_single)
    same = all(torch.equal(x, y) for x, y in zip(out_b, out_s))
    px = sum(H * W for (_, _, _, H, W, _) in specs)
    batcher.close()
    for c in batched + single:
        c.close()
    return {"streams": nstreams, "resolutions": ["480x480", "576x576", "768x768", "1080x1920"],
            "batched_ms_per_tick": round(ms_b, 3), "per_frame_ms_per_tick": round(ms_s, 3),
            "batched_mpixel_s": round(px / ms_b / 1e3, 1), "per_frame_mpixel_s": round(px / ms_s / 1e3, 1),
            "outputs_equal": bool(same)}


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
    ap.add_argument("--ticks", type=int, default=6, help="timed ticks of --batch-mix")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    from . import build

    build.build()
    if a.batch_mix:
        print(json.dumps(batch_mix(a.batch_mix, ticks=a.ticks)))
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
