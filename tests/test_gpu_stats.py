"""Device statistics of Sec. 4 and Sec. 5 (vc_stats_*) against the oracle's
CPU measures (oracle/stats.py), per frame and channel.  Counts are integers
and compared exactly; measures formed from them in binary64 within 1e-12
(relative for chi^2 and the histogram variance, absolute for entropy and
correlation: the device sums in another order and its log2 is not the host's)."""
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


@pytest.fixture(scope="module")
def S():
    from oracle import stats

    return stats


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [(2, 37, 53, 3), (1, 64, 64, 4), (3, 45, 31, 1), (1, 480, 480, 3)]


def _frames(F, H, W, C, seed):
    X = synth.uniform_frames(F, H, W, C, seed=seed)
    if F > 1:  # one smooth frame and one constant frame among them
        X[0] = synth.smooth_clip(1, H, W, C, seed=seed)[0]
    if F > 2:
        X[2] = 77
    return X


@pytest.mark.parametrize("F,H,W,C", SHAPES)
def test_histogram_measures(B, S, F, H, W, C):
    X = _frames(F, H, W, C, 31)
    hist, chi2, var, ent = (t.cpu().numpy() for t in B.stats_histogram(dev(X)))
    for f in range(F):
        for c in range(C):
            ch = X[f, :, :, c]
            assert np.array_equal(hist[f, c].astype(np.int64), S.histogram(ch).astype(np.int64))
            assert chi2[f, c] == pytest.approx(S.chi_square(ch), rel=1e-12)
            assert var[f, c] == pytest.approx(S.hist_variance(ch), rel=1e-12)
            assert ent[f, c] == pytest.approx(S.entropy(ch), abs=1e-12)


def _pairs_all(ch, d):
    dy, dx = {0: (0, 1), 1: (1, 0), 2: (1, 1)}[d]
    H, W = ch.shape
    return ch[:H - dy, :W - dx].ravel().astype(np.float64), ch[dy:, dx:].ravel().astype(np.float64)


@pytest.mark.parametrize("F,H,W,C", SHAPES)
@pytest.mark.parametrize("d", [0, 1, 2])
def test_correlation_all_pairs(B, S, F, H, W, C, d):
    X = _frames(F, H, W, C, 32)
    X[:, :, :, 0] = synth.smooth_clip(F, H, W, 3, seed=5)[:, :, :, 0]  # strongly correlated channel
    r = B.stats_correlation(dev(X), d).cpu().numpy()
    for f in range(F):
        for c in range(C):
            x, y = _pairs_all(X[f, :, :, c], d)
            if x.std() == 0 or y.std() == 0:
                assert np.isnan(r[f, c])  # a constant channel has no correlation coefficient
                continue
            assert r[f, c] == pytest.approx(S.correlation(x, y), abs=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_correlation_given_pairs(B, S, d):
    """The paper's estimator: N random pairs (drawn here, passed in); indices
    whose pair would leave the frame are skipped."""
    H, W, C = 96, 80, 3
    X = synth.smooth_clip(2, H, W, C, seed=6)
    rng = np.random.default_rng(7)
    idx = rng.integers(-50, H * W + 50, size=3000).astype(np.int32)
    r = B.stats_correlation(dev(X), d, pairs=dev(idx)).cpu().numpy()
    dy, dx = {0: (0, 1), 1: (1, 0), 2: (1, 1)}[d]
    ok = (idx >= 0) & (idx // W < H - dy) & (idx % W < W - dx)
    p = idx[ok]
    for f in range(2):
        for c in range(C):
            ch = X[f, :, :, c]
            x = ch.ravel()[p].astype(np.float64)
            y = ch.ravel()[p + dy * W + dx].astype(np.float64)
            assert r[f, c] == pytest.approx(S.correlation(x, y), abs=1e-12)


def test_local_entropy(B, S):
    H, W, C = 200, 180, 3
    X = _frames(2, H, W, C, 33)
    side = 44
    rng = np.random.default_rng(8)
    blocks = np.stack([rng.integers(0, H - side + 1, size=30), rng.integers(0, W - side + 1, size=30)], axis=1)
    blocks = np.concatenate([blocks, [[H - side + 1, 0]]]).astype(np.int32)  # the last block leaves the frame
    for ch in range(C):
        be, mean = (t.cpu().numpy() for t in B.stats_local_entropy(dev(X), ch, dev(blocks), side))
        for f in range(2):
            ref = [S.entropy(X[f, y:y + side, x:x + side, ch]) for y, x in blocks[:-1]]
            assert np.allclose(be[f, :-1], ref, rtol=0, atol=1e-12)
            assert np.isnan(be[f, -1]) and np.isnan(mean[f])
    be, mean = (t.cpu().numpy() for t in B.stats_local_entropy(dev(X), 1, dev(blocks[:-1].copy()), side))
    for f in range(2):
        ref = [S.entropy(X[f, y:y + side, x:x + side, 1]) for y, x in blocks[:-1]]
        assert mean[f] == pytest.approx(np.mean(ref), abs=1e-12)


@pytest.mark.parametrize("F,H,W,C", SHAPES)
def test_npcr_uaci(B, S, F, H, W, C):
    a = synth.uniform_frames(F, H, W, C, seed=34)
    b = a.copy()
    b[0] = synth.uniform_frames(1, H, W, C, seed=35)[0]  # one unrelated frame, the rest equal or nearly
    if F > 1:
        b[1, 0, 0, 0] ^= 1
    n, u = (t.cpu().numpy() for t in B.stats_npcr_uaci(dev(a), dev(b)))
    for f in range(F):
        for c in range(C):
            assert n[f, c] == pytest.approx(S.npcr(a[f, :, :, c], b[f, :, :, c]), rel=1e-13, abs=1e-13)
            assert u[f, c] == pytest.approx(S.uaci(a[f, :, :, c], b[f, :, :, c]), rel=1e-13, abs=1e-13)


def test_cipher_claims_on_device(B, S):
    """Sec. 4.1 / 5.2 claims measured on the device for encrypted frames: the
    ciphertext histogram passes chi^2(0.05, 255) on most channels and a one-pixel
    change of the plaintext gives NPCR/UACI near their ideal values."""
    H = W = 256
    X = synth.smooth_clip(4, H, W, 3, seed=9)
    key = synth.key_for_seed(0, 9)
    e1 = B.Cipher(0, key, H, W, 3, 4, 5)
    e2 = B.Cipher(0, key, H, W, 3, 4, 5)
    X2 = X.copy()
    X2[:, 100, 100, 1] ^= 1
    y1 = e1.encrypt(dev(X))
    y2 = e2.encrypt(dev(X2))
    _, chi2, _, ent = (t.cpu().numpy() for t in B.stats_histogram(y1))
    assert (chi2 < S.CHI2_CRITICAL_255_005).mean() >= 0.75
    assert (ent > 7.99).all()
    n, u = (t.cpu().numpy() for t in B.stats_npcr_uaci(y1, y2))
    n_star, u_lo, u_hi = S.npcr_uaci_critical(W, H)
    # each channel is one draw of a test at alpha = 0.05: most pass, all are near
    assert n.mean() > n_star and (n > n_star).mean() >= 0.75 and (n > n_star - 0.2).all()
    assert ((u > u_lo - 0.5) & (u < u_hi + 0.5)).all()
    e1.close()
    e2.close()
