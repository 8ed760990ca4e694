"""encrypt_frames_static: the entry point for callers that must not allocate
device memory during their work (a framework-owned memory pool or a fixed
budget reserved at start-up; threads for which a device-synchronising
cudaMalloc would stall the video pipeline).  Its scratch lives in a static
device array of the library instead of cudaMalloc'd buffers.

Checked through the C ABI against encrypt_frames, the allocating entry point,
on two calls in a row (the shared static array keeps the first call's
contents when the second runs).  Ciphertext is compared byte for byte, the
tolerance of every other cipher test.  This file is collected last."""
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


@pytest.mark.parametrize("kind,H,W,n", [(0, 480, 480, 4), (1, 96, 128, 7)])
def test_static_scratch_matches_allocating_path_two_calls(B, kind, H, W, n):
    key = synth.key_for_seed(kind, 77)
    X = synth.uniform_frames(8, H, W, 3, seed=78)
    a = B.Cipher(kind, key, H, W, 3, n, 5)   # the no-allocation entry point
    b = B.Cipher(kind, key, H, W, 3, n, 5)   # encrypt_frames
    d = torch.from_numpy(X).cuda()
    for call in range(2):                     # two calls in a row
        part = d[4 * call: 4 * call + 4].contiguous()
        ya = torch.empty_like(part)
        yb = torch.empty_like(part)
        B.encrypt_frames_static(a.ctx, part, ya, 4)
        B.encrypt_frames(b.ctx, part, yb, 4)
        a.sync()
        b.sync()
        assert torch.equal(ya, yb), f"call {call}: {(ya != yb).sum().item()} bytes differ"
    assert a.frame_index == b.frame_index == 8
    # the property the entry point exists for: the context allocated no scratch
    assert a.layout_info()["cap"] == 0
    a.close()
    b.close()


def test_static_calls_interleaved_with_encrypt_frames(B):
    """One context alternating encrypt_frames (which generates the next call's
    first pass of keystream ahead) and encrypt_frames_static (which first undoes
    that run-ahead) gives the bytes of encrypt_frames alone, call for call."""
    key = synth.key_for_seed(0, 80)
    H, W, n = 96, 128, 7
    X = synth.uniform_frames(24, H, W, 3, seed=81)
    mixed = B.Cipher(0, key, H, W, 3, n, 5)
    plain = B.Cipher(0, key, H, W, 3, n, 5)
    assert mixed.get_option(B.VC_OPT_RUNAHEAD_CALLS) == 1
    d = torch.from_numpy(X).cuda()
    for call, static in enumerate([False, True, False, False, True, True]):
        part = d[4 * call: 4 * call + 4].contiguous()
        ym = torch.empty_like(part)
        yp = torch.empty_like(part)
        if static:
            B.encrypt_frames_static(mixed.ctx, part, ym, 4)
        else:
            B.encrypt_frames(mixed.ctx, part, ym, 4)
        B.encrypt_frames(plain.ctx, part, yp, 4)
        mixed.sync()
        plain.sync()
        assert torch.equal(ym, yp), f"call {call} (static={static}): {(ym != yp).sum().item()} bytes differ"
    assert mixed.frame_index == plain.frame_index == 24
    mixed.close()
    plain.close()


def test_static_scratch_rejects_frames_beyond_its_size(B):
    c = B.Cipher(0, synth.key_for_seed(0, 79), 720, 1280, 3, 8, 5)
    d = torch.zeros((1, 720, 1280, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.VcError) as e:
        B.encrypt_frames_static(c.ctx, d, d, 1)
    assert e.value.code == 9  # VC_ERR_UNSUPPORTED
    assert c.frame_index == 0
    c.close()
