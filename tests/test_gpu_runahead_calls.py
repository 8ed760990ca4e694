"""Keystream run-ahead across calls (VC_OPT_RUNAHEAD_CALLS): at the end of a
call the keystream of the next call's first pass is generated speculatively
and the chain state before it kept on the device.  Nothing may be observable
but time: every sequence of calls, checkpoints, batches and option changes
gives the oracle's bytes and frame indices."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


H, W, C, N_SUB, R = 40, 56, 3, 12, 5


def _calls(B, g, X, sizes, direction=0):
    out, f0 = [], 0
    for k in sizes:
        y = g.encrypt(dev(X[f0:f0 + k])) if direction == 0 else g.decrypt(dev(X[f0:f0 + k]))
        out.append(host(y))
        f0 += k
    return np.concatenate(out)


@pytest.mark.parametrize("kind", [0, 1])
def test_calls_of_varying_sizes(B, orc, kind):
    """Run-ahead issued at each call's end, taken whole or in part by the next
    (sizes below, equal to and above the run-ahead pass), encrypt and decrypt."""
    sizes = [24, 1, 2, 30, 5, 24, 3]
    X = synth.uniform_frames(sum(sizes), H, W, C, seed=41)
    key = synth.key_for_seed(kind, 41)
    ref = orc.OracleCipher(kind, key, H, W, C, N_SUB, R)
    Y_ref = ref.encrypt(X)
    g = B.Cipher(kind, key, H, W, C, N_SUB, R)
    assert g.get_option(B.VC_OPT_RUNAHEAD_CALLS) == 1
    Y = _calls(B, g, X, sizes)
    assert np.array_equal(Y, Y_ref)
    assert g.frame_index == sum(sizes)
    d = B.Cipher(kind, key, H, W, C, N_SUB, R)
    assert np.array_equal(_calls(B, d, Y_ref, sizes[::-1], direction=1), X)
    g.close()
    d.close()


def test_checkpoint_with_part_of_the_runahead_taken(B, orc):
    """24 frames (run-ahead of the next first pass issued), 2 frames (taken
    from it), checkpoint (undone: state back at frame 26), resume elsewhere."""
    X = synth.uniform_frames(40, H, W, C, seed=42)
    key = synth.key_for_seed(0, 42)
    ref = orc.OracleCipher(0, key, H, W, C, N_SUB, R)
    Y_ref = ref.encrypt(X)
    g = B.Cipher(0, key, H, W, C, N_SUB, R)
    first = _calls(B, g, X, [24, 2])
    st = g.save_state()
    assert g.frame_index == 26
    rest_same = _calls(B, g, X[26:], [14])  # the same context goes on after the checkpoint
    h = B.Cipher(0, key, H, W, C, N_SUB, R)
    h.load_state(st)
    rest_other = _calls(B, h, X[26:], [6, 8])
    assert np.array_equal(first, Y_ref[:26])
    assert np.array_equal(rest_same, Y_ref[26:])
    assert np.array_equal(rest_other, Y_ref[26:])
    g.close()
    h.close()


def test_load_state_drops_the_runahead(B, orc):
    X = synth.uniform_frames(30, H, W, C, seed=43)
    key = synth.key_for_seed(0, 43)
    ref = orc.OracleCipher(0, key, H, W, C, N_SUB, R)
    Y_ref = ref.encrypt(X)
    g = B.Cipher(0, key, H, W, C, N_SUB, R)
    _calls(B, g, X, [10])
    st = g.save_state()
    _calls(B, g, X[10:], [12, 1])  # run-ahead pending again
    g.load_state(st)                # back to frame 10
    assert g.frame_index == 10
    assert np.array_equal(_calls(B, g, X[10:], [20]), Y_ref[10:])
    g.close()


def test_batch_after_single_stream_calls(B, orc):
    """A batch undoes the run-ahead of its streams' single-stream calls."""
    X = synth.uniform_frames(28, H, W, C, seed=44)
    key = synth.key_for_seed(0, 44)
    ref = orc.OracleCipher(0, key, H, W, C, N_SUB, R)
    Y_ref = ref.encrypt(X)
    g = B.Cipher(0, key, H, W, C, N_SUB, R)
    first = _calls(B, g, X, [24, 1])
    batcher = B.Batcher()
    d = dev(X[25:28])
    out = torch.empty_like(d)
    batcher.submit([(g, 0, d, out, 3)])
    assert np.array_equal(first, Y_ref[:25])
    assert np.array_equal(host(out), Y_ref[25:28])
    batcher.close()
    g.close()


@pytest.mark.parametrize("option,value", [("VC_OPT_TILE_ROWS", 4), ("VC_OPT_OVERLAP", 0),
                                          ("VC_OPT_RUNAHEAD_CALLS", 0), ("VC_OPT_CHUNK", 50)])
def test_options_after_runahead(B, orc, option, value):
    """Options that reallocate scratch or stop the run-ahead undo it first."""
    X = synth.uniform_frames(60, H, W, C, seed=45)
    key = synth.key_for_seed(0, 45)
    ref = orc.OracleCipher(0, key, H, W, C, N_SUB, R)
    Y_ref = ref.encrypt(X)
    g = B.Cipher(0, key, H, W, C, N_SUB, R)
    first = _calls(B, g, X, [24, 3])
    g.set_option(getattr(B, option), value)
    rest = _calls(B, g, X[27:], [33])
    assert np.array_equal(np.concatenate([first, rest]), Y_ref)
    g.close()


def test_debug_keystream_after_runahead(B, orc):
    """The keystream diagnostic reads the chain state directly: undone first."""
    key = synth.key_for_seed(0, 46)
    X = synth.uniform_frames(24, H, W, C, seed=46)
    ref = orc.OracleCipher(0, key, H, W, C, N_SUB, R)
    ref.encrypt(X)
    g = B.Cipher(0, key, H, W, C, N_SUB, R)
    _calls(B, g, X, [24])
    d_ks = torch.empty(2 * R * H * W * C, dtype=torch.uint8, device="cuda")
    d_sc = torch.empty(2, dtype=torch.int64, device="cuda")
    B.vc_dbg_keystream(g.ctx, d_ks, d_sc, 2)
    sc = host(d_sc)
    for f in range(2):
        _, s = ref.frame_keystream()
        assert sc[f] == s
    g.close()


def test_host_entry_takes_the_runahead(B, orc):
    X = synth.uniform_frames(30, H, W, C, seed=47)
    key = synth.key_for_seed(0, 47)
    ref = orc.OracleCipher(0, key, H, W, C, N_SUB, R)
    Y_ref = ref.encrypt(X)
    g = B.Cipher(0, key, H, W, C, N_SUB, R)
    first = _calls(B, g, X, [24])
    h_in = torch.from_numpy(X[24:]).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    g.crypt_host(0, h_in, h_out)
    assert np.array_equal(np.concatenate([first, h_out.numpy()]), Y_ref)
    g.close()
