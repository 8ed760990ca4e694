"""Robustness and round-count experiments (paper_2302_07411_gb300.experiments)
on small cases: the invariants the curves must satisfy."""
from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07411_gb300 import build, experiments

    build.build()
    return experiments


@pytest.mark.parametrize("kind", [0, 1])
def test_error_propagation_bounded(E, kind):
    """One flipped ciphertext bit corrupts between 1 and 3^r decrypted bytes."""
    for row in E.error_propagation(kind, H=32, W=40, n=3, rounds=(1, 2, 3), trials=6):
        assert 1 <= row["max_bytes_wrong"] <= row["bound"]


def test_noise_and_loss_degrade_gracefully(E):
    noise = E.noise_robustness(0, H=64, W=64, n=4, rates=(0.0, 0.01, 0.05))
    assert noise[0]["bytes_exact"] == 1.0 and noise[0]["psnr_db"] == float("inf")
    assert noise[1]["psnr_db"] > noise[2]["psnr_db"]
    assert 0.0 < noise[2]["bytes_exact"] < noise[1]["bytes_exact"] < 1.0
    loss = E.data_loss(0, H=64, W=64, n=4, sides=(0, 8, 16))
    assert loss[0]["bytes_exact"] == 1.0
    assert loss[1]["bytes_exact"] > loss[2]["bytes_exact"]


def test_rounds_sweep_reaches_random_ciphertext(E):
    rows = E.rounds_sweep(0, H=128, W=128, n=4, rounds=(1, 2, 5))
    assert rows[0]["npcr"] < rows[-1]["npcr"]  # one round diffuses only part of the frame
    assert rows[-1]["npcr"] > 99.4 and 33.0 < rows[-1]["uaci"] < 34.0
    assert max(rows[-1][f"abs_corr_{d}"] for d in "HVD") < 0.02


# ----------------------------------------------------------------- oracle cross-checks
# One small case per experiment, recomputed from the oracle's ciphertexts and
# decryptions with the same seeded damage; counts and exact-byte fractions must
# be equal, PSNR and the statistics (oracle/stats.py) equal to rounding.

def _psnr(a, b):
    import math

    import numpy as np

    mse = float(np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * math.log10(255.0 ** 2 / mse)


@pytest.mark.parametrize("kind", [0, 1])
def test_error_propagation_equals_oracle(E, orc, kind):
    import numpy as np

    import synth

    H, W, n, rounds, trials, seed = 32, 40, 3, (1, 2, 3), 5, 3
    rows = E.error_propagation(kind, H=H, W=W, n=n, rounds=rounds, trials=trials, seed=seed)
    X = synth.uniform_frames(1, H, W, 3, seed=seed)
    key = synth.key_for_seed(kind, seed)
    rng = np.random.default_rng(seed)  # the experiment's draws, in its order
    for r, row in zip(rounds, rows):
        Y = orc.OracleCipher(kind, key, H, W, 3, n, r).encrypt(X)
        worst, total = 0, 0
        for _ in range(trials):
            Z = Y.copy()
            q = int(rng.integers(Z.size))
            Z.reshape(-1)[q] ^= np.uint8(1 << int(rng.integers(8)))
            bad = int((orc.OracleCipher(kind, key, H, W, 3, n, r).decrypt(Z) != X).sum())
            worst, total = max(worst, bad), total + bad
        assert row["max_bytes_wrong"] == worst and row["mean_bytes_wrong"] == total / trials


def test_noise_and_loss_equal_oracle(E, orc):
    import numpy as np

    import synth

    H, W, n, seed = 48, 56, 4, 1
    noise = E.noise_robustness(0, H=H, W=W, n=n, rates=(0.01,), seed=seed)[0]
    X = synth.smooth_clip(1, H, W, 3, seed=seed)
    key = synth.key_for_seed(0, seed)
    Y = orc.OracleCipher(0, key, H, W, 3, n, 5).encrypt(X).copy()
    rng = np.random.default_rng(seed + int(0.01 * 1e6))
    hit = rng.random(Y.shape) < 0.01
    Y[hit] = np.where(rng.random(int(hit.sum())) < 0.5, 0, 255).astype(np.uint8)
    D = orc.OracleCipher(0, key, H, W, 3, n, 5).decrypt(Y)
    assert noise["bytes_hit"] == int(hit.sum())
    assert noise["bytes_exact"] == round(float((D == X).mean()), 5)
    assert noise["psnr_db"] == pytest.approx(round(_psnr(D, X), 3), abs=1e-9)

    seed = 2
    loss = E.data_loss(0, H=H, W=W, n=n, sides=(16,), seed=seed)[0]
    X = synth.smooth_clip(1, H, W, 3, seed=seed)
    key = synth.key_for_seed(0, seed)
    Y = orc.OracleCipher(0, key, H, W, 3, n, 5).encrypt(X).copy()
    Y[0, :16, :16, :] = 0
    D = orc.OracleCipher(0, key, H, W, 3, n, 5).decrypt(Y)
    assert loss["bytes_exact"] == round(float((D == X).mean()), 5)
    assert loss["psnr_db"] == pytest.approx(round(_psnr(D, X), 3), abs=1e-9)


def test_rounds_sweep_equals_oracle_statistics(E, orc):
    import numpy as np

    import synth
    from oracle import stats

    H, W, n, seed = 64, 64, 4, 4
    rows = E.rounds_sweep(0, H=H, W=W, n=n, rounds=(1, 2, 3), seed=seed)
    X = synth.smooth_clip(1, H, W, 3, seed=seed)
    X2 = X.copy()
    X2[0, H // 2, W // 2, 0] ^= 1
    key = synth.key_for_seed(0, seed)
    for r, row in zip((1, 2, 3), rows):
        y1 = orc.OracleCipher(0, key, H, W, 3, n, r).encrypt(X)[0]
        y2 = orc.OracleCipher(0, key, H, W, 3, n, r).encrypt(X2)[0]
        npcr = np.mean([stats.npcr(y1[..., c], y2[..., c]) for c in range(3)])
        uaci = np.mean([stats.uaci(y1[..., c], y2[..., c]) for c in range(3)])
        assert row["npcr"] == pytest.approx(round(float(npcr), 4), abs=1e-9)
        assert row["uaci"] == pytest.approx(round(float(uaci), 4), abs=1e-9)
        for d, (dy, dx) in zip("HVD", ((0, 1), (1, 0), (1, 1))):  # every adjacent pair of each channel
            rs = [abs(stats.correlation(y1[: H - dy, : W - dx, c].ravel(), y1[dy:, dx:, c].ravel())) for c in range(3)]
            assert row[f"abs_corr_{d}"] == pytest.approx(round(float(np.mean(rs)), 5), abs=2e-5)
