"""The benchmark's own launch configuration, checked against the oracle.

bench.py times encrypt_frames on 240-frame calls of a 768 x 768 x 3 clip with
n = 4096 subframes and r = 5 (Alg. 1 / Alg. 2), with every option at its
default: passes sized automatically (a body of equal passes, then a tail of
shrinking ones), the keystream of each pass generated on an internal stream
while the previous pass's rounds run, the keystream in CTAs that each hold a
whole SM, and the first pass of the next call generated ahead at the end of a
call.  These tests run exactly that sequence -- a 240-frame call, then a
64-frame call whose first pass is the keystream generated ahead -- and compare
the first and last frame of every pass of both calls, and a few frames inside
passes, with the oracle byte for byte (frames in between advance the oracle's
state through its keystream alone).  Every frame of both calls must also
decrypt to its plaintext through a decrypting context with the same options.
Frames given as a pitched set (frames further apart than N bytes) are checked
against the packed entry point.
"""
from __future__ import annotations

import numpy as np
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


def _bench_options(B, g, pc=0):
    """The options bench.py sets for its default run (all defaults; pc: its
    --diffusion per-channel variant)."""
    g.set_option(B.VC_OPT_CHUNK, 0)
    g.set_option(B.VC_OPT_OVERLAP, 1)
    g.set_option(B.VC_OPT_TILE_ROWS, 0)
    g.set_option(B.VC_OPT_PLCM_INT, 1)
    g.set_option(B.VC_OPT_KS_LANES, 2)
    g.set_option(B.VC_OPT_KS_SM_WARPS, -1)
    g.set_option(B.VC_OPT_DIFFUSION, pc)


def _sample(passes, f0, rng):
    """First and last frame of every pass (absolute indices), and one random
    frame inside each pass of more than two frames."""
    out, f = set(), f0
    for nf in passes:
        out.update((f, f + nf - 1))
        if nf > 2:
            out.add(int(f + rng.integers(1, nf - 1)))
        f += nf
    return out


@pytest.mark.parametrize("kind,pc", [(0, 0), (0, 1)])
def test_bench_sequence_768_n4096_two_calls(B, orc, kind, pc):
    H = W = 768
    C, n, r = 3, 4096, 5
    calls = (240, 64)
    total = sum(calls)
    clip = synth.smooth_clip(16, H, W, C, seed=3)
    X = np.ascontiguousarray(np.concatenate([clip] * ((total + 15) // 16))[:total])
    key = synth.key_for_seed(kind, 100)
    g = B.Cipher(kind, key, H, W, C, n, r)
    _bench_options(B, g, pc)
    d_in = torch.from_numpy(X).cuda()
    d_out = torch.empty_like(d_in)
    rng = np.random.default_rng(5)
    sample, f0, plans = set(), 0, []
    for k, nf in enumerate(calls):
        plan = B.vc_dbg_call_plan(g.ctx, nf)
        plans.append(plan)
        assert sum(plan["passes"]) == nf
        sample |= _sample(plan["passes"], f0, rng)
        g.encrypt(d_in[f0:f0 + nf], d_out[f0:f0 + nf])
        f0 += nf
    g.sync()
    # the sequence is the benchmark's: shrinking tail passes, SM-holding
    # keystream CTAs, run-ahead into the second call's first pass
    p1 = plans[0]["passes"]
    assert len(p1) >= 6 and p1[-1] < p1[0] and p1[-2] < p1[-3]
    assert not plans[0]["first_runahead"] and plans[0]["runahead_next"] > 0
    assert plans[1]["first_runahead"] and plans[1]["passes"][0] == plans[0]["runahead_next"]
    assert plans[0]["ks_sm_warps"] > 0
    Y = d_out.cpu().numpy()
    ref = orc.OracleCipher(kind, key, H, W, C, n, r, per_channel=bool(pc))
    for f in range(total):
        if f in sample:
            exp = ref.encrypt(X[f])
            assert np.array_equal(Y[f], exp), f"frame {f}: {(Y[f] != exp).sum()} bytes differ"
        else:
            ref.frame_keystream()
    assert calls[0] in sample  # the first frame of call 2
    # decryption with the same options returns every frame of both calls
    dd = B.Cipher(kind, key, H, W, C, n, r)
    _bench_options(B, dd, pc)
    back = torch.empty_like(d_out)
    f0 = 0
    for nf in calls:
        dd.decrypt(d_out[f0:f0 + nf], back[f0:f0 + nf])
        f0 += nf
    dd.sync()
    assert torch.equal(back, d_in)
    g.close()
    dd.close()


@pytest.mark.parametrize("kind,H,W,C,n,r", [(0, 48, 40, 3, 7, 5), (1, 33, 47, 3, 61, 5), (2, 64, 64, 1, 2048, 3),
                                            (0, 31, 31, 4, 1, 1)])
@pytest.mark.parametrize("extra", [0, 37, 256])
def test_pitched_frames_equal_packed(B, kind, H, W, C, n, r, extra):
    """encrypt_frames_pitched / decrypt_frames_pitched on frames N + extra
    bytes apart (unaligned for extra = 37) give the packed entry points'
    bytes, leave the bytes between frames alone, and work in place."""
    F = 5
    N = H * W * C
    pitch = N + extra
    X = synth.uniform_frames(F, H, W, C, seed=H + extra)
    key = synth.key_for_seed(kind, 600 + n)
    a = B.Cipher(kind, key, H, W, C, n, r)
    a.set_chunk(2)
    ref = a.encrypt(torch.from_numpy(X).cuda())
    buf = torch.full((F, pitch), 0xA5, dtype=torch.uint8, device="cuda")
    buf[:, :N] = torch.from_numpy(X.reshape(F, N)).cuda()
    out = torch.full((F, pitch), 0x5A, dtype=torch.uint8, device="cuda")
    b = B.Cipher(kind, key, H, W, C, n, r)
    b.set_chunk(2)
    B.encrypt_frames_pitched(b.ctx, buf, out, F, pitch if extra else 0)
    b.sync()
    assert torch.equal(out[:, :N].reshape(ref.shape), ref)
    if extra:
        assert bool((out[:, N:] == 0x5A).all())
    # decryption in place on the pitched set
    d = B.Cipher(kind, key, H, W, C, n, r)
    B.decrypt_frames_pitched(d.ctx, out, out, F, pitch if extra else 0)
    d.sync()
    assert torch.equal(out[:, :N], buf[:, :N])
    with pytest.raises(B.VcError) as e:
        B.encrypt_frames_pitched(b.ctx, buf, out, F, N - 1)
    assert e.value.code == 1
    for c in (a, b, d):
        c.close()
