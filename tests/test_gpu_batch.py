"""Ragged batches (many streams per launch, captured CUDA graph): every job's
output equals the same stream run alone, byte for byte, across resolutions,
maps, directions, subframe counts and round counts, over several consecutive
batches (graph replays) and mixed with single-stream calls."""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STREAMS = [  # (kind, H, W, C, n, rounds, direction, frames per batch)
    (0, 48, 64, 3, 12, 5, 0, 2),
    (1, 40, 40, 3, 4, 5, 1, 1),
    (0, 96, 80, 3, 160, 5, 1, 2),
    (0, 33, 47, 1, 5, 3, 0, 3),
    (1, 64, 32, 4, 64, 2, 0, 1),
    (0, 120, 90, 3, 30, 5, 0, 1),
    (2, 56, 72, 3, 24, 5, 0, 2),
    (2, 30, 30, 3, 9, 4, 1, 1),
]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07411_gb300 import binding, build

    build.build()
    binding.lib()
    return binding


@pytest.mark.parametrize("graph,runahead", [(True, 0), (False, 0), (True, 3), (False, 4)])
def test_batch_equals_solo_runs(B, graph, runahead):
    """runahead > 0: each submit also produces the streams' next keystream
    frames into device rings on an internal stream; later batches consume them."""
    batcher = B.Batcher(graph=graph, runahead=runahead)
    mixed, solo, data = [], [], []
    for s, (kind, H, W, C, n, r, direction, F) in enumerate(STREAMS):
        key = synth.key_for_seed(kind, 500 + s)
        mixed.append(B.Cipher(kind, key, H, W, C, n, r))
        solo.append(B.Cipher(kind, key, H, W, C, n, r))
        data.append(synth.uniform_frames(3 * F, H, W, C, seed=600 + s))
    for tick in range(3):  # consecutive batches: graph replays, state carried, rings wrap
        jobs, outs, refs = [], [], []
        for s, (kind, H, W, C, n, r, direction, F) in enumerate(STREAMS):
            x = torch.from_numpy(data[s][tick * F:(tick + 1) * F]).cuda()
            y = torch.empty_like(x)
            jobs.append((mixed[s], direction, x, y, F))
            outs.append(y)
            ref = solo[s].encrypt(x) if direction == 0 else solo[s].decrypt(x)
            refs.append(ref)
        batcher.submit(jobs)
        torch.cuda.synchronize()
        for s in range(len(STREAMS)):
            assert torch.equal(outs[s], refs[s]), f"tick {tick}, stream {s}"
    for s in range(len(STREAMS)):
        assert mixed[s].frame_index == solo[s].frame_index == 3 * STREAMS[s][7]
    for c in mixed + solo:
        c.close()
    batcher.close()


@pytest.mark.parametrize("sine", [0, 1, -1])
def test_batch_sine_forms_equal_solo_runs(B, sine):
    """VC_BOPT_SINE: the 2DLASM chains of a batch's keystream with the
    all-binary64 sine reduction (1), the integer-assisted one (0) or the
    per-batch choice (-1) give the bytes of the streams run alone."""
    shapes = [(1, 40, 40, 3, 4, 0), (1, 72, 64, 3, 18, 1), (0, 48, 64, 3, 12, 0), (1, 30, 50, 4, 7, 0)]
    batcher = B.Batcher(graph=True)
    B.vc_batcher_set_option(batcher.b, B.VC_BOPT_SINE, sine)
    mixed = [B.Cipher(k, synth.key_for_seed(k, 800 + i), H, W, C, n) for i, (k, H, W, C, n, d) in enumerate(shapes)]
    solo = [B.Cipher(k, synth.key_for_seed(k, 800 + i), H, W, C, n) for i, (k, H, W, C, n, d) in enumerate(shapes)]
    for tick in range(2):
        jobs, outs, refs = [], [], []
        for i, (k, H, W, C, n, d) in enumerate(shapes):
            x = torch.from_numpy(synth.uniform_frames(2, H, W, C, seed=810 + 10 * tick + i)).cuda()
            y = torch.empty_like(x)
            jobs.append((mixed[i], d, x, y, 2))
            outs.append(y)
            refs.append(solo[i].encrypt(x) if d == 0 else solo[i].decrypt(x))
        batcher.submit(jobs)
        torch.cuda.synchronize()
        for i in range(len(shapes)):
            assert torch.equal(outs[i], refs[i]), f"tick {tick}, stream {i}"
    with pytest.raises(B.VcError):
        B.vc_batcher_set_option(batcher.b, B.VC_BOPT_SINE, 2)
    for c in mixed + solo:
        c.close()
    batcher.close()


@pytest.mark.parametrize("split", [1, -1, 0])
def test_batch_long_chain_lane_equals_solo_runs(B, split):
    """VC_BOPT_SPLIT: jobs whose chains are much longer than the rest (a large
    2DLASM frame with few subframes beside small PLCM ones) run in the
    batcher's second lane -- keystream in SM-holding CTAs on a side stream --
    and every output equals the stream run alone, over consecutive batches."""
    shapes = [(1, 96, 128, 3, 4, 0), (0, 32, 32, 3, 8, 0), (0, 40, 48, 3, 12, 1), (2, 24, 40, 3, 6, 0),
              (0, 36, 36, 1, 9, 1), (1, 64, 48, 3, 2, 1)]
    batcher = B.Batcher(graph=True)
    B.vc_batcher_set_option(batcher.b, B.VC_BOPT_SPLIT, split)
    mixed = [B.Cipher(k, synth.key_for_seed(k, 820 + i), H, W, C, n) for i, (k, H, W, C, n, d) in enumerate(shapes)]
    solo = [B.Cipher(k, synth.key_for_seed(k, 820 + i), H, W, C, n) for i, (k, H, W, C, n, d) in enumerate(shapes)]
    for tick in range(3):
        jobs, outs, refs = [], [], []
        for i, (k, H, W, C, n, d) in enumerate(shapes):
            x = torch.from_numpy(synth.uniform_frames(2, H, W, C, seed=830 + 10 * tick + i)).cuda()
            y = torch.empty_like(x)
            jobs.append((mixed[i], d, x, y, 2))
            outs.append(y)
            refs.append(solo[i].encrypt(x) if d == 0 else solo[i].decrypt(x))
        batcher.submit(jobs)
        torch.cuda.synchronize()
        for i in range(len(shapes)):
            assert torch.equal(outs[i], refs[i]), f"tick {tick}, stream {i}"
        nlong = B.lib().vc_dbg_batch_split(batcher.b)
        if split == 1:
            assert nlong >= 1  # the two 2DLASM frames with 2 and 4 subframes
        if split == 0:
            assert nlong == 0
    for c in mixed + solo:
        c.close()
    batcher.close()


@pytest.mark.parametrize("split", [-1, 0, 1])
def test_batch_of_alike_jobs_equals_solo_runs(B, split):
    """A batch whose jobs all have chains of the same length (one shape, one
    map; keystream inline): whatever VC_BOPT_SPLIT says, every job runs (in
    one lane, or with the longest in the second lane when forced) and equals
    its stream run alone."""
    shape = (1, 48, 64, 3, 6)
    k, H, W, C, n = shape
    batcher = B.Batcher(graph=True)
    B.vc_batcher_set_option(batcher.b, B.VC_BOPT_SPLIT, split)
    mixed = [B.Cipher(k, synth.key_for_seed(k, 840 + i), H, W, C, n) for i in range(4)]
    solo = [B.Cipher(k, synth.key_for_seed(k, 840 + i), H, W, C, n) for i in range(4)]
    for tick in range(2):
        jobs, outs, refs = [], [], []
        for i in range(4):
            x = torch.from_numpy(synth.uniform_frames(1, H, W, C, seed=850 + 10 * tick + i)).cuda()
            y = torch.full_like(x, 7)
            jobs.append((mixed[i], i % 2, x, y, 1))
            outs.append(y)
            refs.append(solo[i].encrypt(x) if i % 2 == 0 else solo[i].decrypt(x))
        batcher.submit(jobs)
        torch.cuda.synchronize()
        for i in range(4):
            assert torch.equal(outs[i], refs[i]), f"tick {tick}, stream {i}"
        assert B.lib().vc_dbg_batch_split(batcher.b) == (1 if split == 1 else 0)
    for c in mixed + solo:
        c.close()
    batcher.close()


@pytest.mark.parametrize("runahead", [0, 2])
def test_batch_with_per_channel_streams_equals_solo_runs(B, orc, runahead):
    """Streams with per-channel diffusion chains (VC_OPT_DIFFUSION = 1) in the
    same ragged batches as byte-chain streams, both directions, 3 and 4
    channels, over consecutive batches: every output equals the stream run
    alone, and one per-channel stream's first batch equals the oracle's
    per-channel reading."""
    shapes = [(0, 48, 64, 3, 12, 1, 0), (1, 40, 48, 4, 5, 1, 1), (0, 64, 64, 3, 33, 0, 0), (2, 32, 80, 3, 7, 1, 0),
              (0, 72, 48, 4, 9, 1, 1), (0, 30, 50, 3, 6, 1, 0)]  # (kind, H, W, C, n, per channel, direction)
    batcher = B.Batcher(graph=True, runahead=runahead)
    mixed, solo = [], []
    for i, (k, H, W, C, n, pc, d) in enumerate(shapes):
        for lst in (mixed, solo):
            c = B.Cipher(k, synth.key_for_seed(k, 860 + i), H, W, C, n)
            if pc:
                c.set_option(B.VC_OPT_DIFFUSION, 1)
            lst.append(c)
    for tick in range(3):
        jobs, outs, refs, xs = [], [], [], []
        for i, (k, H, W, C, n, pc, d) in enumerate(shapes):
            x = torch.from_numpy(synth.uniform_frames(2, H, W, C, seed=870 + 10 * tick + i)).cuda()
            y = torch.empty_like(x)
            jobs.append((mixed[i], d, x, y, 2))
            outs.append(y)
            xs.append(x)
            refs.append(solo[i].encrypt(x) if d == 0 else solo[i].decrypt(x))
        batcher.submit(jobs)
        torch.cuda.synchronize()
        for i in range(len(shapes)):
            assert torch.equal(outs[i], refs[i]), f"tick {tick}, stream {i}"
        if tick == 0:
            k, H, W, C, n, pc, d = shapes[0]
            o = orc.OracleCipher(k, synth.key_for_seed(k, 860), H, W, C, n, 5, per_channel=True)
            assert np.array_equal(outs[0].cpu().numpy(), o.encrypt(xs[0].cpu().numpy()))
    for c in mixed + solo:
        c.close()
    batcher.close()


def test_batch_round_trip_and_mixing_with_single_calls(B, orc):
    """Encrypt in a batch, continue the same contexts with single-stream calls,
    then decrypt everything in a batch; the oracle agrees on the ciphertext."""
    batcher = B.Batcher()
    shapes = [(0, 60, 60, 3, 8), (1, 30, 50, 3, 5)]
    enc = [B.Cipher(k, synth.key_for_seed(k, 700 + i), H, W, C, n) for i, (k, H, W, C, n) in enumerate(shapes)]
    dec = [B.Cipher(k, synth.key_for_seed(k, 700 + i), H, W, C, n) for i, (k, H, W, C, n) in enumerate(shapes)]
    refs = [orc.OracleCipher(k, synth.key_for_seed(k, 700 + i), H, W, C, n) for i, (k, H, W, C, n) in enumerate(shapes)]
    X = [synth.uniform_frames(4, H, W, C, seed=710 + i) for i, (k, H, W, C, n) in enumerate(shapes)]
    Y = [torch.empty(x.shape, dtype=torch.uint8, device="cuda") for x in X]
    d = [torch.from_numpy(x).cuda() for x in X]
    batcher.submit([(enc[i], 0, d[i][:2].contiguous(), Y[i][:2], 2) for i in range(2)])
    torch.cuda.synchronize()
    for i in range(2):
        enc[i].encrypt(d[i][2:].contiguous(), Y[i][2:])      # single-stream calls continue the streams
    torch.cuda.synchronize()
    for i in range(2):
        assert np.array_equal(Y[i].cpu().numpy(), refs[i].encrypt(X[i]))
    Z = [torch.empty_like(y) for y in Y]
    batcher.submit([(dec[i], 1, Y[i], Z[i], 4) for i in range(2)])
    torch.cuda.synchronize()
    for i in range(2):
        assert np.array_equal(Z[i].cpu().numpy(), X[i])
    batcher.close()


def test_batch_rejects_bad_jobs(B):
    batcher = B.Batcher()
    c = B.Cipher(0, synth.key_for_seed(0, 1), 16, 16, 3, 4)
    x = torch.zeros((1, 16, 16, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.VcError):
        batcher.submit([(c, 0, x, x.clone(), 1), (c, 0, x, x.clone(), 1)])  # same context twice
    with pytest.raises(B.VcError):
        batcher.submit([(c, 2, x, x.clone(), 1)])
    batcher.close()


def test_runahead_guards_single_stream_calls(B):
    batcher = B.Batcher(runahead=2)
    c = B.Cipher(0, synth.key_for_seed(0, 2), 16, 16, 3, 4)
    x = torch.zeros((2, 16, 16, 3), dtype=torch.uint8, device="cuda")
    batcher.submit([(c, 0, x, torch.empty_like(x), 2)])
    batcher.prefetch([c])     # keystream of the next 2 frames produced ahead
    with pytest.raises(B.VcError) as e:
        c.encrypt(x)          # its keystream is already produced ahead by the batcher
    assert e.value.code == 7  # VC_ERR_SEQUENCE
    with pytest.raises(B.VcError):
        batcher.submit([(c, 0, torch.zeros((3, 16, 16, 3), dtype=torch.uint8, device="cuda"),
                         torch.empty((3, 16, 16, 3), dtype=torch.uint8, device="cuda"), 3)])  # more than run-ahead
    batcher.close()


def test_prefetch_and_ready(B, orc):
    """prefetch produces a new stream's keystream ahead; ready() reports when a
    batch would not wait; the ciphertext is the oracle's."""
    import time

    batcher = B.Batcher(runahead=3)
    key = synth.key_for_seed(1, 3)
    c = B.Cipher(1, key, 24, 40, 3, 6)
    ref = orc.OracleCipher(1, key, 24, 40, 3, 6)
    X = synth.uniform_frames(6, 24, 40, 3, seed=4)
    batcher.prefetch([c])
    t0 = time.time()
    while not batcher.ready(c, 3):
        assert time.time() - t0 < 30
        time.sleep(0.001)
    assert not batcher.ready(c, 4)  # beyond the run-ahead nothing is produced
    d = torch.from_numpy(X).cuda()
    out = torch.empty_like(d)
    for k in range(2):
        batcher.submit([(c, 0, d[3 * k:3 * k + 3], out[3 * k:3 * k + 3], 3)])
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref.encrypt(X))
    batcher.close()


def test_config_64_streams_mixed_resolutions(B, orc):
    """64 streams, each with its own key, resolutions cycling 480x480,
    576x576, 768x768 and 1920x1080 (3 channels), n = ceil(H/4), both maps and
    both directions, one frame per stream per tick, two ticks through one
    captured graph with keystream run-ahead: every output equals the stream
    run alone, and one stream of each resolution and map equals the oracle."""
    import math

    res = [(480, 480), (576, 576), (768, 768), (1080, 1920)]
    batcher = B.Batcher(graph=True, runahead=2)
    streams = []
    for s in range(64):
        H, W = res[s % 4]
        kind, direction = (s // 4) % 2, (s // 8) % 2
        key = synth.key_for_seed(kind, 900 + s)
        n = math.ceil(H / 4)
        streams.append(dict(kind=kind, direction=direction, key=key, H=H, W=W, n=n,
                            mixed=B.Cipher(kind, key, H, W, 3, n), solo=B.Cipher(kind, key, H, W, 3, n),
                            X=synth.uniform_frames(2, H, W, 3, seed=1000 + s)))
    batcher.prefetch([st["mixed"] for st in streams])
    first = {}
    for tick in range(2):
        jobs, outs, refs = [], [], []
        for st in streams:
            x = torch.from_numpy(st["X"][tick:tick + 1]).cuda()
            y = torch.empty_like(x)
            jobs.append((st["mixed"], st["direction"], x, y, 1))
            outs.append(y)
            refs.append(st["solo"].encrypt(x) if st["direction"] == 0 else st["solo"].decrypt(x))
        batcher.submit(jobs)
        torch.cuda.synchronize()
        for s in range(64):
            assert torch.equal(outs[s], refs[s]), f"tick {tick}, stream {s}"
        if tick == 0:
            first = {s: outs[s].cpu().numpy() for s in range(64)}
    for s in (0, 1, 2, 3, 4, 5, 6, 7):  # each resolution with each map, encrypting
        st = streams[s]
        ref = orc.OracleCipher(st["kind"], st["key"], st["H"], st["W"], 3, st["n"])
        assert np.array_equal(first[s], ref.encrypt(st["X"][:1])), f"stream {s}"
    for st in streams:
        st["mixed"].close()
        st["solo"].close()
    batcher.close()
