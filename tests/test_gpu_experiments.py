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
