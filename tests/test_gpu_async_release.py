"""Stream-ordered release of contexts (enc_destroy_async) and the library's
device-memory pool.

A serving loop retires streams while other streams' keystream chains run for
tens of milliseconds.  Releasing a context must not wait for that work (a
plain cudaFree waits for the whole device), and memory given back in stream
order must not be handed to a new context while the old context's work can
still write it.  Checked through the C ABI: ciphertext byte for byte against
a context that never shared the pool with a released one, and the completion
state of a long unrelated chain observed around the release."""
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


def _encrypt(B, c, X, stream=None):
    d = torch.from_numpy(X).cuda()
    y = torch.empty_like(d)
    c.encrypt(d, y, stream=stream)
    return y


@pytest.mark.parametrize("kind", [0, 1])
def test_released_memory_reused_by_the_next_context(B, kind):
    """A context released right after its calls (its run-ahead keystream of
    the next call still in flight) and contexts created at once after it give
    the bytes of a context created before any release."""
    H, W, n = 192, 256, 12
    key = synth.key_for_seed(kind, 31)
    X = synth.uniform_frames(6, H, W, 3, seed=32)
    ref = B.Cipher(kind, key, H, W, 3, n, 5)
    want = [_encrypt(B, ref, X[3 * k: 3 * k + 3]) for k in range(2)]
    torch.cuda.synchronize()
    ref.close()
    for rep in range(4):
        a = B.Cipher(kind, key, H, W, 3, n, 5)
        got = [_encrypt(B, a, X[3 * k: 3 * k + 3]) for k in range(2)]
        a.close(wait=False)  # the keystream generated ahead for a third call may still run
        torch.cuda.synchronize()
        for k in range(2):
            assert torch.equal(got[k], want[k]), f"repeat {rep}, call {k}"


def test_release_does_not_wait_for_other_streams_work(B):
    """While a long 2DLASM chain (1920x1080x3, n = 270, 4 frames: about
    4 x 9,600 dependent map steps per chain) runs on one CUDA stream, creating,
    using and releasing a small context on another returns before that chain is
    done."""
    big = B.Cipher(1, synth.key_for_seed(1, 5), 1080, 1920, 3, 270, 5)
    xb = torch.from_numpy(synth.uniform_frames(4, 1080, 1920, 3, seed=6)).cuda()
    yb = torch.empty_like(xb)
    small = B.Cipher(0, synth.key_for_seed(0, 7), 96, 96, 3, 4, 5)
    xs = torch.from_numpy(synth.uniform_frames(2, 96, 96, 3, seed=8)).cuda()
    ys = torch.empty_like(xs)
    s_big, s_small = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    big.encrypt(xb, yb, stream=s_big)
    done = torch.cuda.Event()
    done.record(s_big)
    small.encrypt(xs, ys, stream=s_small)
    s_small.synchronize()
    small.close(wait=False)
    still_running = not done.query()
    torch.cuda.synchronize()
    big.close()
    assert still_running, "the release waited for an unrelated stream's work"
