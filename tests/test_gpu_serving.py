"""Serving loop: streams admitted over time, frames batched per tick with
continuous batching; every stream's output equals the same stream run alone
(tolerance: 0 bytes), in both the batched and the per-frame-launch modes, and
admission respects the HBM budget."""
from __future__ import annotations

import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07411_gb300 import binding, build

    build.build()
    binding.lib()
    return binding


def _requests():
    reqs = synth.serving_workload(8, seed=11, rate_per_s=40.0, resolutions=((32, 32), (48, 40), (24, 64)),
                                  fps_choices=(24, 30, 60), duration_s=(0.3, 0.6))
    return reqs


@pytest.mark.parametrize("mode,lanes", [("batch", 1), ("batch", 2), ("batch", 4), ("perframe", None)])
def test_served_streams_equal_solo_runs(B, mode, lanes):
    """lanes: batching tick lanes (consecutive ticks on different batchers and
    CUDA streams, so a stream's frames of consecutive ticks run concurrently)."""
    from paper_2302_07411_gb300 import serve

    reqs = _requests()
    opts = {B.VC_SOPT_LANES: lanes} if lanes else None
    srv = serve.Server(hbm_budget_bytes=1 << 30, tick_ms=3.0, mode=mode, max_frames_per_tick=4, ring=64,
                       keep_outputs=True, server_options=opts)
    res = srv.run(reqs)
    summ = res.summary()
    assert summ["admitted"] == len(reqs) and summ["rejected"] == 0
    assert res.frames == sum(max(1, int(r["duration"] * r["fps"])) for r in reqs)
    assert len(srv.finished) == len(reqs)
    for st in srv.finished:
        sp = st.spec
        H, W, C = sp["H"], sp["W"], sp["C"]
        inp = srv.input_frames(H, W, C)
        solo = B.Cipher(sp["kind"], sp["key"], H, W, C, serve.subframes_for(H), 5)
        for k in range(st.frames_total):
            x = inp[k % srv.maxf: k % srv.maxf + 1]
            ref = solo.encrypt(x) if sp["direction"] == 0 else solo.decrypt(x)
            assert torch.equal(st.out[k % srv.ring], ref[0]), (sp["sid"], k)
        solo.close()
        st.cipher.close()
    srv.close()


def test_admission_respects_hbm_budget(B):
    from paper_2302_07411_gb300 import serve

    reqs = _requests()
    one = max(serve.Server.footprint(r, 8, 4) for r in reqs)
    srv = serve.Server(hbm_budget_bytes=int(2.5 * one), tick_ms=3.0)
    res = srv.run(reqs)
    assert res.rejected > 0 and res.admitted >= 1
    srv.close()


@pytest.mark.parametrize("mode", ["batch", "perframe"])
def test_failed_stream_setup_leaves_the_others_served(B, mode):
    """A fault on the host side of the loop: two requests carry keys outside
    the valid ranges, so their context creation fails on the worker thread.
    The loop counts them as failed, returns their HBM budget, and serves every
    other stream exactly as it would alone."""
    from paper_2302_07411_gb300 import serve

    reqs = _requests()
    bad = {reqs[2]["sid"], reqs[5]["sid"]}
    for r in reqs:
        if r["sid"] in bad:
            r["key"] = [1.5, 0.3, 0.4, 0.2] if r["kind"] == 0 else [0.5, 2.0, 0.5, 0.0]  # x0 >= 1 / mu outside
    srv = serve.Server(hbm_budget_bytes=1 << 30, tick_ms=3.0, mode=mode, max_frames_per_tick=4, ring=64,
                       keep_outputs=True)
    res = srv.run(reqs)
    summ = res.summary()
    assert summ["admitted"] == len(reqs) and summ["failed"] == 2 and len(res.errors) == 2
    good = [r for r in reqs if r["sid"] not in bad]
    assert res.frames == sum(max(1, int(r["duration"] * r["fps"])) for r in good)
    assert sorted(st.spec["sid"] for st in srv.finished) == sorted(r["sid"] for r in good)
    for st in srv.finished:
        sp = st.spec
        H, W, C = sp["H"], sp["W"], sp["C"]
        inp = srv.input_frames(H, W, C)
        solo = B.Cipher(sp["kind"], sp["key"], H, W, C, serve.subframes_for(H), 5)
        for k in range(st.frames_total):
            x = inp[k % srv.maxf: k % srv.maxf + 1]
            ref = solo.encrypt(x) if sp["direction"] == 0 else solo.decrypt(x)
            assert torch.equal(st.out[k % srv.ring], ref[0]), (sp["sid"], k)
        solo.close()
        st.cipher.close()
    srv.close()


def test_server_options_are_checked(B):
    """Batching-server options: tick lanes 1..8, set before the first stream
    and after the batcher options; the queued-tick limit 0..64; none of them
    on a per-frame server."""
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    srv = B.NativeServer(0, 2, st)
    for bad in ((B.VC_SOPT_LANES, 0), (B.VC_SOPT_LANES, 9), (B.VC_SOPT_QUEUED_TICKS, -1),
                (B.VC_SOPT_QUEUED_TICKS, 65), (B.VC_BOPT_RUNAHEAD, 3)):
        with pytest.raises(B.VcError):
            srv.set_option(*bad)
    srv.set_option(B.VC_BOPT_KS_PRIORITY, 1)
    srv.set_option(B.VC_SOPT_QUEUED_TICKS, 2)
    srv.set_option(B.VC_SOPT_LANES, 3)
    with pytest.raises(B.VcError):  # the lanes copied the batcher options: no more of those
        srv.set_option(B.VC_BOPT_SPLIT, 0)
    with pytest.raises(B.VcError):  # lanes only once
        srv.set_option(B.VC_SOPT_LANES, 2)
    srv.close()
    per_frame = B.NativeServer(1, 2, st)
    with pytest.raises(B.VcError):
        per_frame.set_option(B.VC_SOPT_LANES, 2)
    per_frame.close()
