"""GPU path == CPU oracle, byte for byte (integer/byte work: the bar is exact
equality), through the C ABI.  Stages first (sine, maps, keystream), then whole
frames over the paper's configurations and odd shapes."""
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


# --------------------------------------------------------------------- stages

@pytest.mark.parametrize("variant", [0, 1])
def test_csin_bitwise(B, orc, variant):
    """The cipher's sine == oracle, its reduction all on the binary64 pipe (0)
    or with the rounding, floor and t - k*PIO2_HI on the integer pipes (1)."""
    rng = np.random.default_rng(100)
    t = np.concatenate([rng.uniform(0, 2 * np.pi, 200000), rng.uniform(0, np.pi, 100000),
                        np.array([0.0, 1e-300, np.pi / 4, np.pi / 2, np.pi, 2 * np.pi, 6.283185307179586])])
    out = torch.empty(t.size, dtype=torch.float64, device="cuda")
    B.vc_dbg_csin(dev(t), out, variant)
    got = host(out)
    idx = rng.choice(t.size, 20000, replace=False)
    exp = np.array([orc.csin(float(v)) for v in t[idx]])
    assert np.array_equal(got[idx].view(np.uint64), exp.view(np.uint64))


@pytest.mark.parametrize("variant", [0, 1])
def test_csin_reduction_edges(B, orc, variant):
    """Arguments where the reduction decides, every one against the oracle:
    u = t*2/pi within a few ulp of a half-integer (the rounding of u + 1/2 and
    its floor pick the quadrant), t within a few ulp of a multiple of PIO2_HI
    (t - k*PIO2_HI cancels), the 2DLASM argument range [-24, 3] (negative k),
    signed zeros and large arguments."""
    rng = np.random.default_rng(103)
    pio2_hi = float.fromhex("0x1.921fb544p+0")
    m = np.arange(-300, 301, dtype=np.float64)
    nudges = np.arange(-4, 5, dtype=np.int64)
    half = ((m + 0.5) * (np.pi / 2)).view(np.int64)
    mult = (m * pio2_hi).view(np.int64)
    t = np.concatenate([(half[:, None] + nudges[None, :]).ravel().view(np.float64),
                        (mult[:, None] + nudges[None, :]).ravel().view(np.float64),
                        rng.uniform(-24.0, 3.0, 50000), -rng.uniform(0, 2 * np.pi, 10000),
                        np.array([-0.0, -1e-300, 400.0, -400.0, 402.1, 1e6, -1e6])])
    out = torch.empty(t.size, dtype=torch.float64, device="cuda")
    B.vc_dbg_csin(dev(t), out, variant)
    got = host(out)
    exp = np.array([orc.csin(float(v)) for v in t])
    assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))


def test_csin_integer_reduction_equals_binary64_at_scale(B):
    """2^26 arguments per batch, 4 batches over the ranges the cipher uses (the
    2DLASM argument range, [0, 2 pi), near zero, and wide enough to reach the
    fallback): both reductions return the same bits, non-finite inputs too."""
    g = torch.Generator(device="cuda")
    g.manual_seed(8)
    n = 1 << 26
    for batch in range(4):
        u = torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
        t = [27.0 * u - 24.0, 2 * np.pi * u, (u - 0.5) * 1e-3, (u - 0.5) * 2000.0][batch]
        if batch == 3:
            t[:3] = torch.tensor([float("inf"), float("-inf"), float("nan")], dtype=torch.float64)
        a = torch.empty_like(t)
        b = torch.empty_like(t)
        B.vc_dbg_csin(t, a, 0)
        B.vc_dbg_csin(t, b, 1)
        torch.cuda.synchronize()
        assert torch.equal(a.view(torch.int64), b.view(torch.int64))


@pytest.mark.parametrize("variant", [0, 1])
def test_plcm_step_bitwise(B, orc, variant):
    """Eq. 5 on the binary64 pipe (0) and on the integer pipes (1) == oracle,
    including the edge operands 0, 1/2, 1, x = p and tiny x."""
    rng = np.random.default_rng(101)
    x = np.concatenate([rng.uniform(0, 1, 50000), rng.uniform(0, 1e-6, 1000), 2.0 ** -rng.uniform(30, 1074, 500),
                        np.array([0.0, 0.5, 1.0, 0.25, 0.3, 0.7, 1 - 2 ** -53])])
    p = rng.uniform(0.01, 0.49, x.size)
    p[-7:] = [0.3, 0.3, 0.3, 0.25, 0.3, 0.3, 0.3]
    out = torch.empty(x.size, dtype=torch.float64, device="cuda")
    B.vc_dbg_plcm(dev(x), dev(p), out, variant)
    got = host(out)
    exp = np.array([orc.plcm_step(float(a), float(b)) for a, b in zip(x, p)])
    assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))


def test_plcm_integer_pipe_equals_binary64_pipe_at_scale(B):
    """2^26 random operands per batch, 4 batches: the integer-pipe step returns
    the same bits as the device's binary64 division (which is IEEE-correct)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    n = 1 << 26
    for batch in range(4):
        x = torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
        if batch == 1:
            x = x * 1e-3
        if batch == 2:
            x = 1.0 - x * 1e-9
        p = 0.01 + 0.48 * torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
        a = torch.empty_like(x)
        b = torch.empty_like(x)
        B.vc_dbg_plcm(x, p, a, 0)
        B.vc_dbg_plcm(x, p, b, 1)
        torch.cuda.synchronize()
        assert torch.equal(a.view(torch.int64), b.view(torch.int64))


def test_lasm_step_bitwise(B, orc):
    rng = np.random.default_rng(102)
    n = 20000
    xymu = np.stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0.44, 0.93, n)], axis=1)
    out = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    B.vc_dbg_lasm(dev(xymu.ravel()), out)
    got = host(out).reshape(n, 2)
    exp = np.array([orc.lasm_step(*map(float, r)) for r in xymu])
    assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))


def _oracle_ks_to_frame_layout(ks_cat, bounds, rounds, N):
    """oracle keystream (subframe-major, r*S_i each) -> [round][frame byte q]."""
    out = np.zeros((rounds, N), np.uint8)
    off = 0
    for i in range(len(bounds) - 1):
        S = bounds[i + 1] - bounds[i]
        for j in range(rounds):
            out[j, bounds[i]:bounds[i + 1]] = ks_cat[off + j * S: off + (j + 1) * S]
        off += rounds * S
    return out


@pytest.mark.parametrize("kind,plcm_int,lanes", [(0, 1, 2), (0, 0, 2), (0, 2, 2), (0, 3, 2), (1, 1, 2), (0, 1, 1),
                                                (0, 0, 1), (1, 1, 1), (2, 1, 2), (2, 1, 1)])
@pytest.mark.parametrize("H,W,C,n,r,frames", [(16, 16, 3, 4, 5, 3), (17, 23, 3, 5, 5, 4), (9, 31, 1, 13, 3, 5),
                                               (12, 12, 4, 144, 1, 3), (48, 40, 3, 7, 2, 6), (33, 47, 3, 61, 5, 3),
                                               (48, 48, 3, 16, 5, 3), (80, 88, 1, 16, 5, 3)])
def test_keystream_and_confusion_seeds(B, orc, kind, plcm_int, lanes, H, W, C, n, r, frames):
    """Sec. 3 byte streams and Alg. 1's s_c per frame, across frames (the left
    over bytes of an iterate carry over, R7), for every keystream kernel form.
    48x48x3 with n = 16 fills a warp with equal word-aligned ranges; 80x88x1
    with n = 16 has equal ranges whose frames start 2 bytes into an iterate."""
    key = synth.key_for_seed(kind, 200 + n)
    ref = orc.OracleCipher(kind, key, H, W, C, n, r)
    g = B.Cipher(kind, key, H, W, C, n, r)
    g.set_option(B.VC_OPT_PLCM_INT, plcm_int)
    g.set_option(B.VC_OPT_KS_LANES, lanes)
    N = H * W * C
    d_ks = torch.empty(frames * r * N, dtype=torch.uint8, device="cuda")
    d_sc = torch.empty(frames, dtype=torch.int64, device="cuda")
    B.vc_dbg_keystream(g.ctx, d_ks, d_sc, frames)
    ks = host(d_ks).reshape(frames, r, N)
    sc = host(d_sc)
    bounds = orc.subframe_bounds(H, W, C, n)
    for f in range(frames):
        cat, s = ref.frame_keystream()
        assert sc[f] == s
        assert np.array_equal(ks[f], _oracle_ks_to_frame_layout(cat, bounds, r, N)), f"frame {f}"
    g.close()


# --------------------------------------------------------------------- whole frames

def _check_enc_dec(B, orc, kind, key, X, n, r, chunk=None, inplace=False, tile_rows=0, ks_sm_warps=0, plcm_int=None,
                   per_channel=False):
    F, H, W, C = X.shape
    ref_e = orc.OracleCipher(kind, key, H, W, C, n, r, per_channel=per_channel)
    ref_d = orc.OracleCipher(kind, key, H, W, C, n, r, per_channel=per_channel)
    Y_ref = ref_e.encrypt(X)
    g_e = B.Cipher(kind, key, H, W, C, n, r)
    g_d = B.Cipher(kind, key, H, W, C, n, r)
    if per_channel:
        g_e.set_option(B.VC_OPT_DIFFUSION, 1)
        g_d.set_option(B.VC_OPT_DIFFUSION, 1)
    if chunk:
        g_e.set_chunk(chunk)
        g_d.set_chunk(chunk)
    if tile_rows:
        g_e.set_option(B.VC_OPT_TILE_ROWS, tile_rows)
        g_d.set_option(B.VC_OPT_TILE_ROWS, 1 if tile_rows > 1 else 2)
    if plcm_int is not None:
        g_e.set_option(B.VC_OPT_PLCM_INT, plcm_int)
        g_d.set_option(B.VC_OPT_PLCM_INT, plcm_int)
    if ks_sm_warps:
        g_e.set_option(B.VC_OPT_KS_SM_WARPS, ks_sm_warps)
        g_d.set_option(B.VC_OPT_KS_SM_WARPS, ks_sm_warps)
        assert g_e.get_option(B.VC_OPT_KS_SM_WARPS) == ks_sm_warps
    d = dev(X)
    Yg = g_e.encrypt(d, d if inplace else None)
    g_e.sync()
    Y = host(Yg)
    assert np.array_equal(Y, Y_ref), f"ciphertext differs in {(Y != Y_ref).sum()} bytes"
    Xg = g_d.decrypt(Yg, Yg if inplace else None)
    g_d.sync()
    assert np.array_equal(host(Xg), X)
    assert np.array_equal(ref_d.decrypt(Y_ref), X)
    g_e.close()
    g_d.close()


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_config_single_480_frame(B, orc, kind):
    """480 x 480 x 3, uniform random bytes (seed 1), key from seed 1, n = 4, r = 5:
    encrypt and decrypt bit-exact against the oracle."""
    X = synth.uniform_frames(1, 480, 480, 3, seed=1)
    _check_enc_dec(B, orc, kind, synth.key_for_seed(kind, 1), X, 4, 5)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("n", [4, 8, 12])
def test_config_smooth_576_clip(B, orc, kind, n):
    """576 x 576 x 3 smooth synthetic video, n in {4, 8, 12}: 3 consecutive frames
    of the clip (state carried across frames), encrypt + decrypt."""
    X = synth.smooth_clip(3, 576, 576, 3, seed=2)
    _check_enc_dec(B, orc, kind, synth.key_for_seed(kind, 2 + n), X, n, 5)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("H,W,C,n,r", [
    (17, 23, 3, 5, 5),     # odd sizes, one tile
    (100, 37, 3, 91, 2),   # several tiles, ragged last tile, tiny subframes
    (45, 200, 3, 300, 5),  # W > H: source rows wrap several times
    (200, 45, 1, 12, 5),   # C = 1, tall
    (31, 31, 4, 1, 5),     # n = 1: the subframe seeds from its own last byte
    (64, 64, 1, 2048, 3),  # 2-byte subframes (the minimum)
    (33, 65, 3, 7, 1),     # one round
    (70, 70, 3, 4900, 5),  # one pixel per subframe
])
def test_odd_shapes(B, orc, kind, H, W, C, n, r):
    X = synth.uniform_frames(2, H, W, C, seed=H + W)
    _check_enc_dec(B, orc, kind, synth.key_for_seed(kind, 300 + n), X, n, r)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("H,W,C,n,r", [
    (16, 16, 3, 4, 5),
    (17, 23, 3, 5, 5),     # odd sizes
    (100, 37, 3, 91, 2),   # ragged subframes
    (45, 200, 3, 300, 5),  # W > H
    (200, 45, 1, 12, 5),   # C = 1 (equal to the byte chain)
    (31, 31, 4, 1, 5),     # n = 1: seeds from its own last pixel
    (64, 64, 1, 2048, 3),  # 2-pixel subframes (the minimum)
    (70, 70, 3, 2450, 5),  # 2-pixel subframes, 3 channels
    (33, 65, 3, 7, 1),     # one round, in place below
    # W a multiple of 16 with whole 16-byte rows: the 16-pixel chunk path
    (64, 64, 3, 2048, 3),  # 2-pixel subframes: up to 8 starts in a chunk
    (96, 160, 4, 77, 5),   # 4 channels, subframes across sub-tiles
    (128, 96, 3, 5, 5),    # long subframes across many tiles (carries between tiles)
    (48, 32, 3, 1, 5),     # n = 1
    (40, 48, 4, 3, 1),     # one round, in place below
])
def test_per_channel_diffusion(B, orc, kind, H, W, C, n, r):
    """The per-channel diffusion variant (VC_OPT_DIFFUSION = 1) against the
    oracle's per-channel reading, encrypt and decrypt, in place for one round."""
    X = synth.uniform_frames(2, H, W, C, seed=H * W + n)
    _check_enc_dec(B, orc, kind, synth.key_for_seed(kind, 400 + n), X, n, r, per_channel=True, inplace=(r == 1))


@pytest.mark.parametrize("tile_rows", [1, 2, 4, 8, 32])
@pytest.mark.parametrize("H,W,C,n", [(64, 96, 3, 40), (72, 48, 4, 9), (50, 70, 3, 33)])
def test_per_channel_diffusion_tile_rows(B, orc, tile_rows, H, W, C, n):
    """Per-channel chains under every tile height (tiles of 1 and 2 rows
    gather pixel by pixel; sub-tiles of 1 to 4 rows), chunked and general
    paths, against the oracle."""
    X = synth.uniform_frames(2, H, W, C, seed=H + W + n + tile_rows)
    _check_enc_dec(B, orc, 0, synth.key_for_seed(0, 450 + n), X, n, 5, tile_rows=tile_rows, per_channel=True)


def test_per_channel_diffusion_clip_in_passes(B, orc):
    """A 576 x 576 x 3 smooth clip, n = 8, 5 frames in passes of 2."""
    X = synth.smooth_clip(5, 576, 576, 3, seed=41)
    _check_enc_dec(B, orc, 0, synth.key_for_seed(0, 41), X, 8, 5, chunk=2, per_channel=True)


def test_per_channel_diffusion_limits(B):
    c = B.Cipher(0, synth.key_for_seed(0, 42), 4, 4, 3, 16)  # one pixel per subframe
    with pytest.raises(B.VcError) as e:
        c.set_option(B.VC_OPT_DIFFUSION, 1)
    assert e.value.code == 3  # VC_ERR_LAYOUT
    with pytest.raises(B.VcError):
        c.set_option(B.VC_OPT_DIFFUSION, 2)
    d = B.Cipher(0, synth.key_for_seed(0, 42), 8, 8, 3, 4)
    d.set_option(B.VC_OPT_DIFFUSION, 1)
    assert d.get_option(B.VC_OPT_DIFFUSION) == 1
    x = torch.zeros((1, 8, 8, 3), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(B.VcError) as e:  # the scratch-free entry point keeps the byte chains only
        B.encrypt_frames_static(d.ctx, x, y, 1)
    assert e.value.code == 9  # VC_ERR_UNSUPPORTED
    c.close()
    d.close()


@pytest.mark.parametrize("tile_rows", [1, 4, 8, 16])
def test_tile_shapes_do_not_change_the_ciphertext(B, orc, tile_rows):
    """Rows per round-kernel tile is a tuning option: any shape (and different
    shapes for encryption and decryption) gives the oracle's bytes."""
    X = synth.uniform_frames(2, 50, 44, 3, seed=17)
    _check_enc_dec(B, orc, 0, synth.key_for_seed(0, 17), X, 9, 5, tile_rows=tile_rows)


@pytest.mark.parametrize("tile_rows", [4, 8, 16, 32])
@pytest.mark.parametrize("H,W,C,per_channel", [(50, 64, 3, False), (100, 160, 3, False), (36, 64, 3, True),
                                               (200, 48, 3, False), (72, 48, 4, False), (66, 96, 4, True)])
def test_decrypt_band_heights(B, orc, tile_rows, H, W, C, per_channel):
    """Decryption of the oracle's ciphertext in bands of 4 to 32 rows (the
    scatter form: rows of whole 16-byte pieces), with heights that leave a
    partial last band, widths above and below the height, and words of the
    output shared between the runs of neighbouring bands."""
    n, r = 11, 3
    X = synth.uniform_frames(2, H, W, C, seed=H * W + tile_rows)
    key = synth.key_for_seed(0, 470 + tile_rows)
    ref = orc.OracleCipher(0, key, H, W, C, n, r, per_channel=per_channel)
    Y = ref.encrypt(X)
    g = B.Cipher(0, key, H, W, C, n, r)
    if per_channel:
        g.set_option(B.VC_OPT_DIFFUSION, 1)
    g.set_option(B.VC_OPT_TILE_ROWS, tile_rows)
    Xg = g.decrypt(dev(Y))
    g.sync()
    got = host(Xg)
    assert np.array_equal(got, X), f"{(got != X).sum()} bytes differ"
    g.close()


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("warps", [1, 2, 4])
def test_keystream_on_reserved_sms(B, orc, kind, warps):
    """Keystream CTAs that each hold a whole SM (several passes, so keystream
    and rounds overlap across the two streams) give the oracle's bytes."""
    X = synth.uniform_frames(6, 48, 40, 3, seed=23)
    _check_enc_dec(B, orc, kind, synth.key_for_seed(kind, 23), X, 37, 5, chunk=2, ks_sm_warps=warps)


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("H,W,C,n", [(48, 48, 3, 16), (96, 96, 3, 64)])
def test_exact_fallback_in_full_warps(B, orc, mode, H, W, C, n):
    """Equal word-aligned ranges fill whole warps (the warp-wide exchange); the
    exact fallback rewrites every range (mode 2) or only the odd subframes'
    (mode 3, so lane pairs of one warp take different paths)."""
    X = synth.uniform_frames(4, H, W, C, seed=29)
    _check_enc_dec(B, orc, 0, synth.key_for_seed(0, 29), X, n, 5, chunk=2, plcm_int=mode)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_chunked_and_in_place(B, orc, kind):
    """Frames processed in passes of 2 and in place give the same stream."""
    X = synth.uniform_frames(5, 40, 56, 3, seed=9)
    _check_enc_dec(B, orc, kind, synth.key_for_seed(kind, 9), X, 6, 5, chunk=2, inplace=True)
    _check_enc_dec(B, orc, kind, synth.key_for_seed(kind, 9), X, 6, 1, chunk=3, inplace=True)


def test_state_checkpoint_resume(B):
    """10 frames in one call == 5 + save + load into a fresh context + 5."""
    X = synth.uniform_frames(10, 32, 48, 3, seed=10)
    key = synth.key_for_seed(0, 10)
    a = B.Cipher(0, key, 32, 48, 3, 6, 5)
    full = host(a.encrypt(dev(X)))
    b = B.Cipher(0, key, 32, 48, 3, 6, 5)
    first = host(b.encrypt(dev(X[:5])))
    st = b.save_state()
    assert b.frame_index == 5
    c = B.Cipher(0, key, 32, 48, 3, 6, 5)
    c.load_state(st)
    assert c.frame_index == 5
    second = host(c.encrypt(dev(X[5:])))
    assert np.array_equal(np.concatenate([first, second]), full)
    with pytest.raises(B.VcError):
        B.Cipher(0, key, 32, 48, 3, 7, 5).load_state(st)


@pytest.mark.parametrize("direction", [0, 1])
def test_host_buffer_entry_point(B, direction):
    """crypt_frames_host (host buffers, copies inside) == the device entry point."""
    X = synth.uniform_frames(7, 48, 64, 3, seed=11)
    key = synth.key_for_seed(1, 11)
    a = B.Cipher(1, key, 48, 64, 3, 8, 5)
    a.set_chunk(3)
    out = np.empty_like(X)
    a.crypt_host(direction, X, out)
    b = B.Cipher(1, key, 48, 64, 3, 8, 5)
    ref = host(b.encrypt(dev(X)) if direction == 0 else b.decrypt(dev(X)))
    assert np.array_equal(out, ref)


def test_host_async_calls_pipeline(B):
    """crypt_frames_host_async calls issued back to back (several passes per
    call, so the staging buffers rotate across calls; each call's done event
    waited at the end) give the bytes of synchronous calls, call for call, and
    decrypt back."""
    key = synth.key_for_seed(0, 91)
    H, W, C, n = 96, 128, 3, 7
    X = synth.uniform_frames(24, H, W, C, seed=92)
    a = B.Cipher(0, key, H, W, C, n, 5)
    b = B.Cipher(0, key, H, W, C, n, 5)
    d = B.Cipher(0, key, H, W, C, n, 5)
    for c in (a, b, d):
        c.set_chunk(3)
    h_in = torch.from_numpy(X).pin_memory()
    outs = [torch.empty((8, H, W, C), dtype=torch.uint8).pin_memory() for _ in range(3)]
    back = [torch.empty((8, H, W, C), dtype=torch.uint8).pin_memory() for _ in range(3)]
    evs = [torch.cuda.Event() for _ in range(3)]
    for k in range(3):
        a.crypt_host_async(0, h_in[8 * k: 8 * k + 8], outs[k], done_event=evs[k])
    for k in range(3):
        evs[k].synchronize()
        ref = torch.empty_like(outs[k]).pin_memory()
        b.crypt_host(0, h_in[8 * k: 8 * k + 8], ref)
        assert torch.equal(outs[k], ref), f"call {k}: {(outs[k] != ref).sum().item()} bytes differ"
    for k in range(3):
        d.crypt_host_async(1, outs[k], back[k])
    d.sync()
    for k in range(3):
        assert np.array_equal(back[k].numpy(), X[8 * k: 8 * k + 8]), f"call {k} does not decrypt back"
    assert a.frame_index == b.frame_index == d.frame_index == 24
    for c in (a, b, d):
        c.close()


def test_invalid_arguments_are_errors(B):
    with pytest.raises(B.VcError) as e:
        B.Cipher(0, [0.3, 0.6, 0.5, 0.2], 16, 16)
    assert e.value.code == 2
    with pytest.raises(B.VcError) as e:
        B.Cipher(0, [0.3, 0.2, 0.5, 0.2], 4, 4, 1, 16)
    assert e.value.code == 3
    with pytest.raises(B.VcError) as e:
        B.Cipher(1, [0.3, 0.39, 0.5], 16, 16)
    assert e.value.code == 2
    with pytest.raises(B.VcError) as e:
        B.Cipher(2, [0.3, 3.8, 0.5, 3.95], 16, 16)  # r outside [3.9, 4]
    assert e.value.code == 2
    with pytest.raises(B.VcError) as e:
        B.Cipher(3, [0.3, 0.2, 0.5, 0.2], 16, 16)  # no such map
    assert e.value.code == 2


@pytest.mark.parametrize("kind,H,W,n", [(0, 2160, 3840, 540), (1, 1080, 1920, 270), (0, 1080, 1920, 4096),
                                        (2, 1080, 1920, 270)])
def test_largest_frames(B, orc, kind, H, W, n):
    """The serving workload's largest frames (rows of 11,520 bytes: 8-row tiles,
    wider than tall), two frames per call: equal to the oracle byte for byte,
    and decryption returns the plaintext."""
    X = synth.smooth_clip(2, H, W, 3, seed=13)
    key = synth.key_for_seed(kind, 13)
    g = B.Cipher(kind, key, H, W, 3, n, 5)
    Y = host(g.encrypt(dev(X)))
    assert np.array_equal(Y, orc.OracleCipher(kind, key, H, W, 3, n, 5).encrypt(X))
    dd = B.Cipher(kind, key, H, W, 3, n, 5)
    assert np.array_equal(host(dd.decrypt(dev(Y))), X)
    g.close()
    dd.close()


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_full_size_768_n4096_sampled(B, orc, kind):
    """The benchmark's launch configuration (768 x 768 x 3, n = 4096, r = 5, many
    frames per pass): all 24 frames round-trip; the first 3 equal the oracle
    byte for byte."""
    F = 24
    X = synth.smooth_clip(F, 768, 768, 3, seed=12)
    key = synth.key_for_seed(kind, 12)
    g = B.Cipher(kind, key, 768, 768, 3, 4096, 5)
    g.set_chunk(F)
    d = dev(X)
    Y = g.encrypt(d)
    g.sync()
    Yh = host(Y)
    ref = orc.OracleCipher(kind, key, 768, 768, 3, 4096, 5)
    assert np.array_equal(Yh[:3], ref.encrypt(X[:3]))
    dd = B.Cipher(kind, key, 768, 768, 3, 4096, 5)
    dd.set_chunk(F)
    assert np.array_equal(host(dd.decrypt(Y)), X)
