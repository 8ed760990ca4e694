"""The seeded synthetic inputs: keys inside every map's valid ranges (checked
by the oracle's own validation), reproducible frames and clips, and serving
workloads with the stated arrival, resolution, rate and direction mix."""
from __future__ import annotations

import numpy as np

import synth


def test_keys_are_valid_and_reproducible(orc):
    for kind in (synth.PLCM, synth.DLASM, synth.LOGISTIC):
        for seed in range(200):
            key = synth.key_for_seed(kind, seed)
            assert orc.key_valid(kind, key), (kind, seed, key)
            assert key == synth.key_for_seed(kind, seed)
        assert synth.key_for_seed(kind, 1) != synth.key_for_seed(kind, 2)


def test_frames_are_seeded():
    a = synth.uniform_frames(2, 9, 7, 3, seed=4)
    assert a.shape == (2, 9, 7, 3) and a.dtype == np.uint8
    assert np.array_equal(a, synth.uniform_frames(2, 9, 7, 3, seed=4))
    c = synth.smooth_clip(3, 40, 48, 3, seed=5)
    assert c.shape == (3, 40, 48, 3) and c.dtype == np.uint8
    assert np.array_equal(c, synth.smooth_clip(3, 40, 48, 3, seed=5))
    # smooth video: neighbouring pixels are strongly correlated, unlike uniform bytes
    x = c[0, :, :-1, 0].astype(float).ravel()
    y = c[0, :, 1:, 0].astype(float).ravel()
    assert np.corrcoef(x, y)[0, 1] > 0.5


def test_serving_workload_mix():
    reqs = synth.serving_workload(400, seed=7, rate_per_s=50.0)
    t = np.array([r["arrival"] for r in reqs])
    assert (np.diff(t) > 0).all()
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.25 / 50.0  # Poisson arrivals at the stated rate
    assert {r["fps"] for r in reqs} == {24, 30, 60}
    assert {(r["H"], r["W"]) for r in reqs} <= {(480, 480), (576, 576), (768, 768), (720, 1280), (1080, 1920),
                                              (2160, 3840)}
    assert [r["kind"] for r in reqs[:4]] == [0, 1, 0, 1]
    assert 0.35 < np.mean([r["direction"] for r in reqs]) < 0.65
    assert all(2.0 <= r["duration"] <= 6.0 for r in reqs)
    assert reqs == synth.serving_workload(400, seed=7, rate_per_s=50.0)
