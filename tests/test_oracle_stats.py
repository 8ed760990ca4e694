"""The paper's statistical and security claims (Sec. 4, Sec. 5) checked on the
oracle's ciphertext for random keys and a smooth synthetic video frame, and the
statistics helpers pinned to the values the paper prints."""
from __future__ import annotations

import os

import numpy as np
import pytest

import synth
from oracle import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def paper_values() -> dict:
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


def test_critical_values_reproduce_the_paper():
    """Sec. 5.2 prints NPCR* = 99.5893% and UACI* in [33.3730%, 33.5541%] for
    512 x 512 at alpha = 0.05; Sec. 4.1 prints chi^2(0.05, 255) = 293.25."""
    from scipy.stats import chi2

    pv = paper_values()
    n_star, u_lo, u_hi = stats.npcr_uaci_critical(512, 512, 0.05)
    assert round(n_star, 4) == pv["npcr_critical_512_0.05"]
    assert round(u_lo, 4) == pv["uaci_low_512_0.05"]
    assert round(u_hi, 4) == pv["uaci_high_512_0.05"]
    assert round(chi2.ppf(0.95, 255), 2) == pv["chi2_critical_255_0.05"] == stats.CHI2_CRITICAL_255_005


def test_statistics_helpers_on_known_inputs():
    """Closed forms: a flat histogram has chi^2 = 0 and variance 0, entropy 8;
    a constant image has entropy 0; identical images give NPCR = UACI = 0;
    complementary images give UACI = 100 * mean|2x - 255| / 255."""
    flat = np.tile(np.arange(256, dtype=np.uint8), 16).reshape(64, 64)
    assert stats.chi_square(flat) == 0.0
    assert stats.hist_variance(flat) == 0.0
    assert abs(stats.entropy(flat) - 8.0) < 1e-12
    assert stats.entropy(np.zeros((8, 8), np.uint8)) == 0.0
    assert stats.npcr(flat, flat) == 0.0 and stats.uaci(flat, flat) == 0.0
    comp = (255 - flat).astype(np.uint8)
    assert abs(stats.uaci(flat, comp) - 100 * np.abs(2 * flat.astype(float) - 255).mean() / 255) < 1e-12
    x = np.arange(100, dtype=float)
    assert abs(stats.correlation(x, 2 * x + 1) - 1.0) < 1e-12
    assert abs(stats.correlation(x, -x) + 1.0) < 1e-12


@pytest.mark.parametrize("kind", [0, 1])
def test_cipher_statistics_on_smooth_video(orc, kind):
    """Sec. 4: near-flat ciphertext histograms, adjacent pixel correlation near
    0 (20,000 pairs per direction), entropy near 8 and local entropy of
    (30, 1936) blocks near its ideal, while the plaintext is strongly
    correlated.  chi^2 of an ideal cipher is itself chi^2(255)-distributed, so
    one channel exceeds the 293.25 of Sec. 4.1 about one time in twenty; the
    check is therefore that the mean over 4 keys x 3 channels is near 255 and no
    channel exceeds the alpha = 0.001 quantile."""
    from scipy.stats import chi2

    H = W = 256
    X = synth.smooth_clip(1, H, W, 3, seed=3)[0]
    chis = []
    for s in range(4):
        enc = orc.OracleCipher(kind, synth.key_for_seed(kind, 40 + 10 * s + kind), H, W, 3, 8)
        Y = enc.encrypt(X)
        chis += [stats.chi_square(Y[..., ch]) for ch in range(3)]
    assert max(chis) < chi2.ppf(0.999, 255)
    assert abs(np.mean(chis) - 255.0) < 4 * np.sqrt(2 * 255 / len(chis))
    for ch in range(3):
        xp, yp = stats.adjacent_pairs(X[..., ch], "H", 20000, seed=ch)
        assert stats.correlation(xp, yp) > 0.9
        for d in "HVD":
            a, b = stats.adjacent_pairs(Y[..., ch], d, 20000, seed=7 + ch)
            assert abs(stats.correlation(a, b)) < 0.02
        # expected deficit of an ideal source: 255 / (2 N ln 2) bits
        assert stats.entropy(Y[..., ch]) > 8.0 - 2.0 * 255 / (2 * H * W * np.log(2))
        assert stats.local_entropy(Y[..., ch], 30, 1936, seed=ch) > 7.89


@pytest.mark.parametrize("kind", [0, 1])
def test_npcr_uaci_one_pixel_change(orc, kind):
    """Sec. 5.2: one changed plaintext byte, re-encrypted with the same byte
    sequences (state checkpoint), changes ~99.6% of the ciphertext with UACI near
    33.46%; the mean over trials lies beyond the critical values of this size."""
    H = W = 192
    key = synth.key_for_seed(kind, 50 + kind)
    X = synth.smooth_clip(1, H, W, 3, seed=4)[0]
    enc = orc.OracleCipher(kind, key, H, W, 3, 8)
    st = enc.save_state()
    C1 = enc.encrypt(X)
    rng = np.random.default_rng(16)
    n_star, u_lo, u_hi = stats.npcr_uaci_critical(W, H, 0.05)
    npcrs, uacis = [], []
    for _ in range(12):
        X2 = X.copy()
        a, o, ch = int(rng.integers(H)), int(rng.integers(W)), int(rng.integers(3))
        X2[a, o, ch] = np.uint8((int(X2[a, o, ch]) + 1) % 256)
        enc.load_state(st)
        C2 = enc.encrypt(X2)
        npcrs.append([stats.npcr(C1[..., c], C2[..., c]) for c in range(3)])
        uacis.append([stats.uaci(C1[..., c], C2[..., c]) for c in range(3)])
    npcrs, uacis = np.array(npcrs), np.array(uacis)
    assert (npcrs.min(axis=0) > 99.0).all()
    assert (npcrs.mean(axis=0) > n_star).all()
    assert ((uacis.mean(axis=0) > u_lo) & (uacis.mean(axis=0) < u_hi)).all()


@pytest.mark.parametrize("kind", [0, 1])
def test_key_sensitivity(orc, kind):
    """Sec. 5.1: decrypting with a key off by delta = 1e-9 (initial value, then
    control parameter) yields an image uncorrelated with the correct decryption."""
    H = W = 128
    key = synth.key_for_seed(kind, 60 + kind)
    X = synth.smooth_clip(1, H, W, 3, seed=5)[0]
    Y = orc.OracleCipher(kind, key, H, W, 3, 4).encrypt(X)
    for idx in (0, 1):
        bad = list(key)
        bad[idx] += 1e-9
        D = orc.OracleCipher(kind, bad, H, W, 3, 4).decrypt(Y)
        for ch in range(3):
            r = stats.correlation(D[..., ch].ravel(), X[..., ch].ravel())
            assert abs(r) < 0.02
