#!/usr/bin/env python
"""Benchmark of the GB300 chaotic video cipher (arXiv 2302.07411), one JSON line.

Workload (default): the 240-frame 768 x 768 x 3 uint8 smooth synthetic clip
(gradients + 8 moving Gaussian blobs + N(0, 4^2) noise), n = 4096 subframes,
r = 5 rounds, PLCM key from a seed.  One step = encrypt the whole clip through
the C ABI (keystream + confusion + diffusion of all frames, inputs resident in
HBM); the stream state carries from step to step as it would in a long video.
The 240 input frames (425 MB) exceed the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torch.distributed.run): every rank encrypts its own stream
(its own key) on its own GPU -- replicas with no collective on the data path;
value = total pixels of all ranks / max step time ("scaling": "weak").
--impl reference times the CPU oracle (the plain single-threaded C
implementation) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# Each served stream produces its keystream on its own CUDA stream; with the
# default 8 hardware work queues many of them serialise behind one another.
# Read once, when the CUDA context is created (before any CUDA call here).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# binary64 operations per map iterate, as the method specifies the iterate
# (fixed by the equations and the sine reading, not by any kernel's code):
#  PLCM, Eq. 5: one comparison, up to two additions/subtractions (1 - x and
#    x - p) and one division, the division counted as the seven fused
#    multiply-adds of a Newton-Raphson division with a final correction step
#    (Markstein's sequence) -> 10;
#  logistic map: two products and one difference -> 3;
#  2DLASM, Eq. 6: two sines of the cipher's csin (Cody-Waite reduction, 7
#    operations; degree-17 / degree-16 Taylor polynomial by Horner without
#    fused multiply-adds, 18) and five products and sums per coordinate
#    -> 2 x 25 + 10 = 60.
FP64_OPS_PER_ITER = {"plcm": 10.0, "logistic": 3.0, "2dlasm": 60.0}
# map iterates per 6 keystream bytes: two PLCM or logistic maps (6 bytes each,
# XORed); a 2DLASM pair emits 12 bytes per iterate of its two maps
ITERS_PER_BYTE = {"plcm": 2.0 / 6.0, "logistic": 2.0 / 6.0, "2dlasm": 2.0 / 12.0}
# DRAM read + write bytes per frame of keystream of k_ks_plcm_fx_sm (ncu,
# 40-frame launch at 768x768x3, n = 4096; profiles/k_ks_plcm_fx_sm_*): scaled
# to the bench's launches by their frames
PLCM_KS_DRAM_BYTES_PER_FRAME = (365_568 + 297_627_904) / 40
SWEEP_N = (16, 64, 256, 1024, 4096)

MAP_KIND = {"plcm": 0, "2dlasm": 1, "logistic": 2}  # VC_PLCM, VC_2DLASM, VC_LOGISTIC
METRIC = "5-round enc Mpixel/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--map", choices=["plcm", "2dlasm", "logistic"], default="plcm")
    ap.add_argument("--frames", type=int, default=240)
    ap.add_argument("--size", type=int, default=768)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--rounds", type=int, default=5)
    ap.add_argument("--plcm-fp64", action="store_true", help="PLCM division on the binary64 pipe (A/B)")
    ap.add_argument("--ks-lanes", type=int, default=2, choices=[1, 2], help="lanes per subframe in the keystream")
    ap.add_argument("--chunk", type=int, default=0, help="frames per pass (0 = automatic)")
    ap.add_argument("--no-overlap", action="store_true", help="keystream and rounds on one stream")
    ap.add_argument("--tile-rows", type=int, default=0, help="rows per round-kernel tile (0 = automatic)")
    ap.add_argument("--ks-sm-warps", type=int, default=-1,
                    help="keystream CTAs of this many warps, each holding a whole SM (0 = share all SMs, -1 = auto)")
    ap.add_argument("--direction", choices=["enc", "dec"], default="enc",
                    help="dec times decryption of the clip's ciphertext (not the headline metric)")
    ap.add_argument("--diffusion", choices=["bytes", "per-channel"], default="bytes",
                    help="diffusion chains: over the subframe's bytes (default) or one per colour channel")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    ap.add_argument("--no-serving", action="store_true", help="skip the 24 FPS serving-capacity leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the subframe-count sweep (n = 16 .. 4096)")
    return ap.parse_args()


def workload_name(a) -> str:
    return f"{a.frames}-frame {a.size}x{a.size}x3 smooth clip, n={a.n}, r={a.rounds}, {a.map.upper()}"


def config(a, world: int) -> dict:
    return {"workload": workload_name(a), "plcm_division": "binary64 pipe" if a.plcm_fp64 else "integer pipes",
            "frames": a.frames, "height": a.size, "width": a.size, "channels": 3,
            "n_subframes": a.n, "rounds": a.rounds, "map": a.map, "parallelism": f"replicas{world}",
            "keystream_overlap": not a.no_overlap, "frames_per_pass": a.chunk or "auto",
            "direction": a.direction, "diffusion": a.diffusion, "tile_rows": a.tile_rows or "auto", "ks_sm_warps": a.ks_sm_warps if a.ks_sm_warps >= 0 else "auto",
            "l2": "inputs 425 MB > 129 MB L2, no flush"}


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid: str | None):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_uuid:
            cmd += ["-i", gpu_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.tmp.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle timing

def time_oracle(a, budget_s: float, seed_frames):
    """The oracle as it stands, single thread, on consecutive frames of the
    workload until the time budget is used (at least one frame)."""
    import oracle
    import synth

    kind = MAP_KIND[a.map]
    c = oracle.OracleCipher(kind, synth.key_for_seed(kind, 100), a.size, a.size, 3, a.n, a.rounds,
                            per_channel=a.diffusion == "per-channel")
    done, t0 = 0, time.perf_counter()
    while True:
        c.encrypt(seed_frames[done % len(seed_frames)])
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or done >= a.frames:
            break
    return done, el


def run_reference(a) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth

    frames = synth.smooth_clip(4, a.size, a.size, 3, seed=3)
    px = a.size * a.size
    # each step: a bounded sample (enough consecutive frames for ~budget/steps seconds)
    per_step = max(1.0, min(20.0, 150.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        time_oracle(a, per_step / 4, frames)
    tot_frames, tot_s = 0, 0.0
    for _ in range(a.steps):
        n, s = time_oracle(a, per_step, frames)
        tot_frames += n
        tot_s += s
    value = tot_frames * px / tot_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mpixel/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(1e3 * tot_s / a.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+u8",
            "data": "synthetic", "config": config(a, 1),
            "cpu_baseline": {"value": round(value, 4), "unit": "Mpixel/s", "cores": 1, "kind": "oracle",
                             "sample": f"{tot_frames} consecutive frames of the workload (at most {per_step:.0f} s per step)"},
            "e2e": {"value": round(value, 4), "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- replicas (N > 1)

def stream_seed(rank: int) -> int:
    """Key seed of the video stream a rank encrypts: every rank its own stream."""
    return 100 + rank


def reduce_max(x: float, device) -> float:
    """Max over ranks (the slowest replica sets the step time); identity at N = 1."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(pixels_per_rank: int, world: int, seconds_per_step: float) -> float:
    """Mpixel/s of all ranks together: every rank processed pixels_per_rank."""
    return world * pixels_per_rank / seconds_per_step / 1e6


# ----------------------------------------------------------------- GPU arm

def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def serving_capacity() -> dict:
    """Serving (continuous batching, one graph replay per 4 ms tick, keystream
    run-ahead) against one call per frame (each stream on its own CUDA
    stream), two workloads:

    * capacity: the largest number of concurrent 24 FPS 768x768x3 streams
      (half encrypt / half decrypt, alternating PLCM / 2DLASM, n = 192; and
      PLCM only) whose steady-state p99 per-frame latency stays under 41.7 ms;
    * mixed: 256 streams arriving as a Poisson process (64/s), 480^2 ...
      3840x2160, 24/30/60 FPS, half 2DLASM, half decrypt, admitted by HBM
      budget and compute-aware admission (calibrated device rates), with the
      admitted streams' steady p99, first-frame p99 and the latency split at
      submission (wait for the frame clock and keystream / device time);
    * batch_mix: 64 streams of 480^2 ... 1920x1080, one frame each per tick,
      as one ragged batch per tick against one call per frame."""
    from paper_2302_07411_gb300 import serve

    out = {"resolution": "768x768x3", "fps": 24, "p99_budget_ms": round(1000 / 24, 2)}
    b = serve.capacity("batch", 768, 768, counts=(256, 288, 320, 384, 448, 512), seconds=3.0)
    p = serve.capacity("perframe", 768, 768, counts=(64, 96, 128, 160, 192, 256), seconds=2.5)
    # the same with PLCM streams only (2DLASM keystream is binary64-bound and
    # about eight times the work of PLCM per frame)
    bp = serve.capacity("batch", 768, 768, counts=(640, 768, 896, 1024, 1152, 1280, 1408), seconds=3.0, kinds=(0,))
    out["batched_streams"] = b["max_streams"]
    out["per_frame_streams"] = p["max_streams"]
    out["batched_streams_plcm_only"] = bp["max_streams"]
    out["batched_plcm_only_runs"] = [{k: r.get(k) for k in ("streams", "steady_p50_ms", "steady_p99_ms", "fps")}
                                     for r in bp["runs"]]
    out["criterion"] = b["criterion"]
    out["batched_runs"] = [{k: r.get(k) for k in ("streams", "steady_p50_ms", "steady_p99_ms", "first_frame_p99_ms",
                                                  "fps", "tick_host_p50_ms", "tick_host_p99_ms")} for r in b["runs"]]
    out["per_frame_runs"] = [{k: r.get(k) for k in ("streams", "steady_p50_ms", "steady_p99_ms", "fps")}
                             for r in p["runs"]]
    rates = serve.calibrate()
    keep = ("load_target", "admitted", "rejected", "rejected_load", "rejected_chain", "frames", "fps", "steady_p50_ms",
            "steady_p99_ms", "first_frame_p99_ms", "peak_concurrent_streams")
    mixed = {"calibration": rates}
    for mode in ("batch", "perframe"):
        r = serve.serve_mixed(mode, rates=rates)
        mixed[mode] = {"admitted_within_budget": r["admitted_within_budget"], "load_target": r["load_target"],
                       "runs": [dict({k: x.get(k) for k in keep}, latency_split=x.get("split")) for x in r["runs"]]}
    mixed["workload"] = "256 Poisson streams (64/s), 480^2..3840x2160, 24/30/60 FPS, half 2DLASM, half decrypt"
    out["mixed"] = mixed
    # ragged batch against one call per frame, 64 streams of mixed resolutions
    out["batch_mix"] = serve.batch_mix(64, rates=rates)
    return out


def kernel_chain_cycles(a, kind, key, stream) -> float:
    """Cycles per map iterate of the keystream kernel when its chains run
    alone: one frame of 768x768x3 with n = 16 (32 chains = one warp) in the
    bench's keystream kernel (SM-holding CTAs), timed with CUDA events."""
    import torch

    from paper_2302_07411_gb300 import binding as B

    n, H = 16, 768
    N = H * H * 3
    c = B.Cipher(kind, key, H, H, 3, n, a.rounds)
    c.set_option(B.VC_OPT_OVERLAP, 1)
    ks = torch.empty(a.rounds * N, dtype=torch.uint8, device="cuda")
    sc = torch.empty(1, dtype=torch.int64, device="cuda")
    B.vc_dbg_keystream(c.ctx, ks, sc, 1, stream=stream)  # warm-up, scratch
    torch.cuda.synchronize()
    B.enc_profile_enable(c.ctx, True)
    B.enc_profile_read(c.ctx)
    B.vc_dbg_keystream(c.ctx, ks, sc, 1, stream=stream)
    torch.cuda.synchronize()
    ms = B.enc_profile_read(c.ctx)["keystream"]["ms"]
    c.close()
    iters_per_chain = a.rounds * (N / n) * ITERS_PER_BYTE[a.map] / 2
    return ms * 1e-3 * 2.07e9 / iters_per_chain


def subframe_sweep(a, X, d_in, d_out, kind, key, stream, clock_hz, step_cycles, at_n):
    """The subframe-count sweep on the same clip (n = 16 .. 4096; Sec. 3 and
    Sec. 6 vary the thread count, one subframe per thread): Mpixel/s, the
    keystream and rounds stage times per 240-frame step, and the ceiling that
    2n dependent PLCM chains set (2n chains x clock / the kernel's cycles per
    iterate with one warp of chains, over 5 map iterates per pixel).  n = a.n
    reuses the main measurement."""
    import torch

    from paper_2302_07411_gb300 import binding as B

    F, H, W, Cc = a.frames, a.size, a.size, 3
    rows = []
    for n in SWEEP_N:
        if n == a.n:
            ms, ks_ms, rd_ms = at_n
        else:
            c = B.Cipher(kind, key, H, W, Cc, n, a.rounds)
            steps = 1 if n <= 64 else 3
            for _ in range(1):
                c.encrypt(d_in, d_out, stream=stream)
            torch.cuda.synchronize()
            c.sync()
            B.enc_profile_enable(c.ctx, True)
            B.enc_profile_read(c.ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                c.encrypt(d_in, d_out, stream=stream)
            B.enc_join(c.ctx, stream)  # the keystream the last call generated ahead is inside the window
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            pr = B.enc_profile_read(c.ctx)
            ks_ms = pr["keystream"]["ms"] / steps
            rd_ms = pr["rounds"]["ms"] / steps
            c.close()
        px = F * H * W
        ceiling = 2 * n * clock_hz / step_cycles / 5.0 / 1e6  # Mpixel/s: 5 PLCM iterates per pixel
        rows.append({"n": n, "mpixel_s": round(px / (ms * 1e-3) / 1e6, 2), "ms_per_step": round(ms, 3),
                     "keystream_ms": round(ks_ms, 3), "rounds_ms": round(rd_ms, 3),
                     "chain_ceiling_mpixel_s": round(ceiling, 2),
                     "frac_of_chain_ceiling": round(px / (ms * 1e-3) / 1e6 / ceiling, 4)})
    return rows


def run_ours(a) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    import synth
    from paper_2302_07411_gb300 import binding as B
    from paper_2302_07411_gb300 import build as cuda_build

    cuda_build.build()
    kind = MAP_KIND[a.map]
    F, H, W, Cc = a.frames, a.size, a.size, 3
    N = H * W * Cc
    X = synth.smooth_clip(F, H, W, Cc, seed=3)
    d_in = torch.from_numpy(X).cuda()
    d_out = torch.empty_like(d_in)
    key = synth.key_for_seed(kind, stream_seed(rank))
    ciph = B.Cipher(kind, key, H, W, Cc, a.n, a.rounds)
    ciph.set_option(B.VC_OPT_CHUNK, a.chunk)
    ciph.set_option(B.VC_OPT_OVERLAP, 0 if a.no_overlap else 1)
    ciph.set_option(B.VC_OPT_TILE_ROWS, a.tile_rows)
    ciph.set_option(B.VC_OPT_PLCM_INT, 0 if a.plcm_fp64 else 1)
    ciph.set_option(B.VC_OPT_KS_LANES, a.ks_lanes)
    ciph.set_option(B.VC_OPT_KS_SM_WARPS, a.ks_sm_warps)
    ciph.set_option(B.VC_OPT_DIFFUSION, 1 if a.diffusion == "per-channel" else 0)
    stream = torch.cuda.current_stream()
    if a.direction == "dec":
        # ciphertext of the clip from a separate encrypting context; every step
        # decrypts it again (the context's keystream moves on, the work is the same)
        ce0 = B.Cipher(kind, key, H, W, Cc, a.n, a.rounds)
        ce0.set_option(B.VC_OPT_DIFFUSION, 1 if a.diffusion == "per-channel" else 0)
        ce0.encrypt(d_in, d_out, stream=stream)
        torch.cuda.synchronize()
        ce0.close()
        d_in, d_out = d_out, torch.empty_like(d_out)

    def step():
        if a.direction == "dec":
            ciph.decrypt(d_in, d_out, stream=stream)
        else:
            ciph.encrypt(d_in, d_out, stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    ciph.sync()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    time.sleep(0.3)
    B.enc_profile_enable(ciph.ctx, True)
    B.enc_profile_read(ciph.ctx)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    # the end event also waits for the keystream the last step generated ahead
    # for a next call (the first step's was generated before the window)
    B.enc_join(ciph.ctx, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / a.steps
    prof = B.enc_profile_read(ciph.ctx)
    B.enc_profile_enable(ciph.ctx, False)
    clk = clocks.stop()
    ciph.sync()
    ms = reduce_max(ms, "cuda")

    px_step = F * H * W
    value = whole_job_rate(px_step, world, ms * 1e-3)

    # ---- end to end: host buffers through crypt_frames_host, copies inside
    e2e = None
    if not a.no_e2e:
        h_in = (torch.from_numpy(X) if a.direction == "enc" else d_in.cpu()).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        ce = B.Cipher(kind, key, H, W, Cc, a.n, a.rounds)
        ce.set_option(B.VC_OPT_CHUNK, a.chunk)
        ce.set_option(B.VC_OPT_OVERLAP, 0 if a.no_overlap else 1)
        ce.set_option(B.VC_OPT_TILE_ROWS, a.tile_rows)
        ce.set_option(B.VC_OPT_PLCM_INT, 0 if a.plcm_fp64 else 1)
        ce.set_option(B.VC_OPT_KS_LANES, a.ks_lanes)
        ce.set_option(B.VC_OPT_KS_SM_WARPS, a.ks_sm_warps)
        ce.set_option(B.VC_OPT_DIFFUSION, 1 if a.diffusion == "per-channel" else 0)
        # one host-buffer call per step, consecutive steps pipelined (a step's
        # uploads and keystream start while the previous step's last passes and
        # downloads run); the window ends when the last step's download is done
        hdir = 0 if a.direction == "enc" else 1
        for _ in range(max(1, a.warmup - 1)):
            ce.crypt_host_async(hdir, h_in, h_out, stream=stream)
        ce.sync()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        k2 = max(1, a.steps)
        for _ in range(k2):
            ce.crypt_host_async(hdir, h_in, h_out, stream=stream)
        ce.sync()  # every download, and the keystream the last call generated ahead (the first call's came before t0)
        el = reduce_max((time.perf_counter() - t0) / k2, "cuda")
        e2e = {"value": round(whole_job_rate(px_step, world, el), 3), "unit": "Mpixel/s", "h2d_bytes_per_step": F * N,
               "d2h_bytes_per_step": F * N, "ms_per_step": round(el * 1e3, 3),
               "calls": "crypt_frames_host_async per step from pinned host buffers, steps pipelined"}
        ce.close()

    if rank != 0:
        return

    # ---- roofline of the dominant kernel (the keystream) against fixed bounds
    peaks = load_peaks()
    probes = B.vc_dbg_peaks(stream)  # measured on this GPU in this run
    if a.map == "plcm":
        probes["kernel_iter_cycles"] = kernel_chain_cycles(a, kind, key, stream)
    ks_launches = max(1, prof["keystream"]["launches"])
    ks_ms_step = prof["keystream"]["ms"] / max(1, a.steps)  # summed keystream launch time per step
    ks_ms = prof["keystream"]["ms"] / ks_launches            # per launch
    rd_ms = prof["rounds"]["ms"] / max(1, a.steps)
    sc_ms = prof["schedule"]["ms"] / max(1, a.steps)
    iters = F * a.rounds * N * ITERS_PER_BYTE[a.map]  # map iterates per step
    achieved_iter = iters / (ks_ms_step * 1e-3)
    clock_hz = (clk.get("sm_mhz") or 2070.0) * 1e6
    fp64_ops = probes["fp64_ops_per_s"]
    fp64_bound = fp64_ops / FP64_OPS_PER_ITER[a.map]
    hbm = peaks.get("hbm_gbs")
    alg_bytes = 2 * N * F  # plaintext read once + ciphertext written once
    hbm_achieved = alg_bytes / (ms * 1e-3) / 1e9
    frac_hbm = hbm_achieved / hbm if hbm else None
    lat = None
    if a.map == "plcm":
        # 2n independent chains, each one dependent iterate after another, at
        # the cycles per iterate the same keystream kernel takes when its
        # chains run alone (one warp on the GPU, timed in this run)
        chains = 2 * a.n
        cyc = probes["kernel_iter_cycles"]
        ceiling = chains * clock_hz / cyc
        lat = {"chains": chains, "cycles_per_iterate": round(cyc, 1), "ceiling": round(ceiling / 1e9, 4),
               "frac": round(achieved_iter / ceiling, 4),
               "probe_step_cycles": round(probes["plcm_step_cycles"], 1),
               "basis": ("2n chains x median SM clock / cycles per iterate of the keystream kernel with one "
                         "warp of chains on the GPU (768x768x3, n = 16, one frame, this run)")}
    per_launch = ks_launches // max(1, a.steps)
    traffic = None
    if a.map == "plcm" and a.size == 768 and a.n == 4096 and a.rounds == 5:
        traffic = round(PLCM_KS_DRAM_BYTES_PER_FRAME * F / per_launch)
    roofline = {"bound": "alu", "pipe": "binary64",
                "kernel": {"plcm": "k_ks_plcm_fx_sm", "2dlasm": "k_ks_pair_sm<2DLASM>",
                           "logistic": "k_ks_pair_sm<logistic>"}[a.map],
                "unit": "Giter/s", "achieved": round(achieved_iter / 1e9, 4), "peak": round(fp64_bound / 1e9, 4),
                "frac": round(achieved_iter / fp64_bound, 4), "traffic": traffic,
                "traffic_basis": "scaled from the 40-frame ncu capture (DRAM bytes per frame x frames per launch)"
                                 if traffic else None,
                "peak_basis": (f"measured binary64 FMA rate ({fp64_ops / 1e9:.1f} G/s, this run) / "
                               f"{FP64_OPS_PER_ITER[a.map]:.0f} binary64 operations per map iterate of the method"),
                "frac_fp64": round(achieved_iter / fp64_bound, 4),
                "frac_hbm": round(frac_hbm, 5) if frac_hbm is not None else None,
                "frac_latency": lat["frac"] if lat else None,
                "hbm": {"achieved_gbs": round(hbm_achieved, 2), "peak_gbs": hbm,
                        "basis": "6 B/pixel (plaintext read + ciphertext written) / ms_per_step, of measured copy BW"},
                "latency_bound": lat,
                "measured": {"fp64_gops": round(fp64_ops / 1e9, 2), "imad_gops": round(probes["imad_ops_per_s"] / 1e9, 1),
                             "plcm_step_cycles": round(probes["plcm_step_cycles"], 1)},
                "launch_ms": round(ks_ms, 3), "launches_per_step": per_launch}
    rounds_bytes = 3 * N * F * a.rounds  # per round: read X and the keystream, write Y
    split = {"keystream_ms": round(ks_ms_step, 3), "rounds_ms": round(rd_ms, 3), "schedule_ms": round(sc_ms, 3),
             "overlapped": not a.no_overlap,
             "rounds_alg_gbs": round(rounds_bytes / (rd_ms * 1e-3) / 1e9, 1) if rd_ms > 0 else None,
             "hbm_bound_ms": round(alg_bytes / (hbm * 1e9) * 1e3, 4) if hbm else None}

    sweep = None
    if not a.no_sweep and world == 1 and a.size == 768 and a.map == "plcm":
        sweep = subframe_sweep(a, X, d_in, d_out, kind, key, stream, clock_hz, probes["kernel_iter_cycles"],
                               (ms, ks_ms_step, rd_ms))

    cpu = None
    if not a.no_cpu_baseline:
        n_fr, s = time_oracle(a, a.cpu_seconds, X[:8])
        cpu = {"value": round(n_fr * H * W / s / 1e6, 4), "unit": "Mpixel/s", "cores": 1, "kind": "oracle",
               "sample": f"{n_fr} consecutive frames of the workload, single thread, {s:.1f} s"}

    serving = None
    if not a.no_serving and world == 1:
        serving = serving_capacity()

    launches = sum(v["launches"] for v in prof.values())
    metric = METRIC if a.direction == "enc" else METRIC.replace(" enc ", " dec ")
    line = {"metric": metric, "value": round(value, 3), "unit": "Mpixel/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+u8", "data": "synthetic", "config": config(a, world),
            "roofline": roofline, "split": split, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "sweep": sweep, "serving": serving,
            "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)
    ciph.close()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
