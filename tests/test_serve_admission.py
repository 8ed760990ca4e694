"""Compute-aware admission of the serving loop (host logic, no GPU): a
stream's charge is its keystream iterates per second over the map's
calibrated rate plus its pixels per second over the rounds' rate, and a
stream whose own serial chains cannot keep up with its frame rate is refused
whatever the load."""
from __future__ import annotations

import pytest

from paper_2302_07411_gb300 import serve

RATES = {"ks_iter_per_s": {"0": 200e9, "1": 10e9}, "chain_s_per_iter": {"0": 150e-9, "1": 2.2e-6},
         "rounds_px_per_s": 40e9}


def spec(kind, H, W, fps):
    return {"kind": kind, "H": H, "W": W, "C": 3, "fps": fps}


def test_cost_arithmetic():
    """768x768x3 at 24 FPS, n = 192: subframes of 9216 bytes, 5 rounds, 6 bytes
    per PLCM iterate of each of the two maps."""
    b = serve.ComputeBudget(RATES)
    load, busy = b.cost(spec(0, 768, 768, 24))
    n = 192
    it_chain = 5 * 9216 / 6
    assert busy == pytest.approx(24 * it_chain * 150e-9)
    assert load == pytest.approx(24 * (2 * n * it_chain / 200e9 + 768 * 768 / 40e9))
    # 2DLASM: 12 bytes per step of the pair, so half the iterates per byte
    load2, busy2 = b.cost(spec(1, 768, 768, 24))
    assert busy2 == pytest.approx(24 * (5 * 9216 / 12) * 2.2e-6)
    assert load2 > load


def test_admission_fills_to_the_target_and_releases():
    b = serve.ComputeBudget(RATES, target=0.5)
    s = spec(0, 1080, 1920, 30)
    load, _ = b.cost(s)
    admitted = []
    while True:
        ok, charged, why = b.admit(s)
        if not ok:
            assert why == "load"
            break
        admitted.append(charged)
    assert len(admitted) == int(0.5 // load)
    assert b.used <= 0.5 + 1e-12
    for c in admitted:
        b.release(c)
    assert b.used == pytest.approx(0.0, abs=1e-12)


def test_chains_that_cannot_keep_up_are_refused():
    """A 3840x2160 2DLASM stream at 60 FPS (n = 540: 19,200 steps per chain and
    frame) needs a chain busier than the limit, even on an idle device."""
    b = serve.ComputeBudget(RATES, target=10.0)
    ok, charged, why = b.admit(spec(1, 2160, 3840, 60))
    assert not ok and why == "chain" and charged == 0.0 and b.used == 0.0
    ok, _, _ = b.admit(spec(0, 2160, 3840, 60))
    assert ok


def test_long_chains_get_sm_holding_keystream():
    """With the held-placement rate calibrated, a stream whose chains would be
    busy more than half its frame period on shared SMs gets SM-holding
    keystream CTAs (two warps for 2DLASM) and is charged its SMs' share of the
    device; a short-chain stream stays on shared SMs."""
    rates = dict(RATES, chain_s_per_iter_held={"0": 140e-9, "1": 1.6e-6}, sms=152)
    b = serve.ComputeBudget(rates)
    p = b.plan(spec(1, 1080, 1920, 24))  # 9,600 steps per chain and frame
    assert p["hold"] == 2
    assert p["busy"] == pytest.approx(24 * 9600 * 1.6e-6)
    n = 270
    ctas = -(-2 * n // 64)
    assert p["load"] == pytest.approx(ctas * p["busy"] / 152 + 24 * 1080 * 1920 / 40e9)
    q = b.plan(spec(0, 768, 768, 24))
    assert q["hold"] == 0 and q["busy"] == pytest.approx(24 * (5 * 9216 / 6) * 150e-9)


def test_result_summary_without_gpu():
    """The serving result's summary (latency percentiles, steady-state window,
    admission counters) is host arithmetic."""
    r = serve.ServeResult("batch", latencies_ms=[1.0, 2.0, 3.0, 50.0], arrivals_s=[0.1, 2.0, 2.5, 3.0],
                          first_frame_ms=[1.0], frames=4, admitted=2, rejected_chain=1, wall_s=2.0)
    s = r.summary(steady_after_s=1.5)
    assert s["frames"] == 4 and s["fps"] == 2.0 and s["admitted"] == 2 and s["rejected_chain"] == 1
    assert s["steady_frames"] == 3 and s["steady_p50_ms"] == 3.0
    assert s["first_frame_p99_ms"] == 1.0


def test_latency_split_of_recorded_frames():
    """The split of each frame's latency at its submission (host arithmetic
    over the native server's records): wait = submission - arrival, device =
    completion - submission, frames before the steady window left out; per
    tick, device time and the queue before the device starts it."""
    import numpy as np

    fr = np.array([[0, 0.5, 0.502, 0.510],   # before the window
                   [1, 2.0, 2.004, 2.014],
                   [2, 2.1, 2.101, 2.141],
                   [1, 2.2, 2.210, 2.215]])
    tk = np.array([[0.502, 0.503, 0.509, 1], [2.004, 2.005, 2.013, 2], [2.210, 2.230, 2.240, 1]])
    r = serve.ServeResult("batch", frame_records=fr, tick_records=tk)
    s = r.latency_split(steady_after_s=1.0)
    assert s["frames"] == 3 and s["ticks"] == 2
    assert s["wait_p50_ms"] == pytest.approx(4.0) and s["wait_p99_ms"] == pytest.approx(9.9, abs=0.05)
    assert s["device_p50_ms"] == pytest.approx(10.0) and s["device_p99_ms"] == pytest.approx(39.4, abs=0.05)
    assert s["tick_device_p99_ms"] == pytest.approx(10.0, abs=0.1)
    assert s["tick_queue_p99_ms"] == pytest.approx(19.8, abs=0.05)
    assert serve.ServeResult("batch").latency_split() == {}
