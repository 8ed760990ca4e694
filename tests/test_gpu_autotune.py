"""The autotuner times real launches, caches its choice per GPU and shape, and
whatever it picks leaves the ciphertext unchanged."""
from __future__ import annotations

import json
import os

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


def test_stream_tuning_is_cached_and_exact(B, orc, tmp_path, monkeypatch):
    from paper_2302_07411_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    res = autotune.tune_stream(0, 64, 80, 3, 16, frames=6)
    assert set(res["options"]) == {"ks_lanes", "tile_rows", "overlap", "ks_sm_warps"}
    assert len(res["trials"]) == 30 and all(t["ms"] > 0 for t in res["trials"])
    assert autotune.tune_stream(0, 64, 80, 3, 16, frames=6) == res  # served from the cache
    assert json.load(open(tmp_path / "tune.json"))
    key = synth.key_for_seed(0, 90)
    X = synth.uniform_frames(3, 64, 80, 3, seed=91)
    c = B.Cipher(0, key, 64, 80, 3, 16)
    autotune.apply_stream(c, res["options"])
    Y = c.encrypt(torch.from_numpy(X).cuda())
    assert np.array_equal(Y.cpu().numpy(), orc.OracleCipher(0, key, 64, 80, 3, 16).encrypt(X))


def test_batch_tuning(B, tmp_path, monkeypatch):
    from paper_2302_07411_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    res = autotune.tune_batch([(0, 48, 48, 3, 12), (1, 32, 64, 3, 8)])
    assert res["options"]["ctas_per_sm"] in (0, 1, 2) and res["options"]["tile_rows"] in (0, 16)
