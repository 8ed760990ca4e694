"""Robustness and round-count experiments of Sec. 5.3 and Sec. 6 (the paper's
figures: salt-and-pepper noise and data loss on the ciphertext, NPCR / UACI
and correlation against the number of rounds), run with the CUDA library on
seeded synthetic video and reported as curves (the paper gives figures only).

Every cipher step and every measure runs in libvcrypt (encrypt_frames,
decrypt_frames, vc_stats_*); this module draws the damage and the inputs,
drives the calls and collects numbers.

  python -m paper_2302_07411_gb300.experiments --out curves.json
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import binding as B


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * math.log10(255.0 ** 2 / mse)


def _clip(frames: int, H: int, W: int, seed: int):
    import synth

    return synth.smooth_clip(frames, H, W, 3, seed=seed)


def noise_robustness(kind: int = 0, H: int = 256, W: int = 256, n: int = 4, rounds: int = 5,
                     rates=(0.0, 0.01, 0.03, 0.05), seed: int = 1) -> list[dict]:
    """Salt-and-pepper noise at each rate on the ciphertext bytes (Sec. 5.3,
    noise attack), then decryption: PSNR of the decrypted frame against the
    plaintext and the fraction of bytes recovered exactly."""
    import synth

    X = _clip(1, H, W, seed)
    key = synth.key_for_seed(kind, seed)
    out = []
    for rate in rates:
        enc = B.Cipher(kind, key, H, W, 3, n, rounds)
        dec = B.Cipher(kind, key, H, W, 3, n, rounds)
        Y = _host(enc.encrypt(_dev(X)))
        rng = np.random.default_rng(seed + int(rate * 1e6))
        hit = rng.random(Y.shape) < rate
        Y = Y.copy()
        Y[hit] = np.where(rng.random(int(hit.sum())) < 0.5, 0, 255).astype(np.uint8)
        D = _host(dec.decrypt(_dev(Y)))
        out.append({"rate": rate, "psnr_db": round(_psnr(D, X), 3), "bytes_exact": round(float((D == X).mean()), 5),
                    "bytes_hit": int(hit.sum())})
        enc.close()
        dec.close()
    return out


def data_loss(kind: int = 0, H: int = 512, W: int = 512, n: int = 4, rounds: int = 5,
              sides=(0, 64, 128, 256), seed: int = 2) -> list[dict]:
    """A side x side block of the ciphertext set to zero (Sec. 5.3, data loss;
    the paper's text and figure disagree on the sizes, so several are run):
    PSNR and the fraction of bytes recovered exactly after decryption."""
    import synth

    X = _clip(1, H, W, seed)
    key = synth.key_for_seed(kind, seed)
    out = []
    for side in sides:
        enc = B.Cipher(kind, key, H, W, 3, n, rounds)
        dec = B.Cipher(kind, key, H, W, 3, n, rounds)
        Y = _host(enc.encrypt(_dev(X))).copy()
        Y[0, :side, :side, :] = 0
        D = _host(dec.decrypt(_dev(Y)))
        out.append({"block": side, "lost_fraction": round(side * side / (H * W), 5),
                    "psnr_db": round(_psnr(D, X), 3), "bytes_exact": round(float((D == X).mean()), 5)})
        enc.close()
        dec.close()
    return out


def error_propagation(kind: int = 0, H: int = 64, W: int = 64, n: int = 4, rounds=(1, 2, 3, 5),
                      trials: int = 16, seed: int = 3) -> list[dict]:
    """One flipped ciphertext bit, then decryption: decrypted bytes that
    differ (each round spreads a byte error to at most 3 bytes before the
    inverse permutation, so at most 3^r)."""
    import synth

    X = synth.uniform_frames(1, H, W, 3, seed=seed)
    key = synth.key_for_seed(kind, seed)
    rng = np.random.default_rng(seed)
    out = []
    for r in rounds:
        enc = B.Cipher(kind, key, H, W, 3, n, r)
        Y = _host(enc.encrypt(_dev(X)))
        worst, total = 0, 0
        for _ in range(trials):
            Z = Y.copy()
            q = int(rng.integers(Z.size))
            Z.reshape(-1)[q] ^= np.uint8(1 << int(rng.integers(8)))
            dec = B.Cipher(kind, key, H, W, 3, n, r)
            D = _host(dec.decrypt(_dev(Z)))
            dec.close()
            bad = int((D != X).sum())
            worst = max(worst, bad)
            total += bad
        out.append({"rounds": r, "max_bytes_wrong": worst, "mean_bytes_wrong": total / trials, "bound": 3 ** r})
        enc.close()
    return out


def rounds_sweep(kind: int = 0, H: int = 256, W: int = 256, n: int = 4, rounds=tuple(range(1, 11)),
                 seed: int = 4) -> list[dict]:
    """NPCR / UACI between the ciphertexts of two plaintexts differing in one
    pixel, and the adjacent-pixel correlation of the ciphertext, for r rounds
    (the paper's round-count figures), measured with the device statistics."""
    import synth

    X = _clip(1, H, W, seed)
    X2 = X.copy()
    X2[0, H // 2, W // 2, 0] ^= 1
    key = synth.key_for_seed(kind, seed)
    out = []
    for r in rounds:
        e1 = B.Cipher(kind, key, H, W, 3, n, r)
        e2 = B.Cipher(kind, key, H, W, 3, n, r)
        y1 = e1.encrypt(_dev(X))
        y2 = e2.encrypt(_dev(X2))
        npcr, uaci = (_host(t) for t in B.stats_npcr_uaci(y1, y2))
        corr = {d: float(np.abs(_host(B.stats_correlation(y1, i))).mean()) for i, d in enumerate("HVD")}
        out.append({"rounds": r, "npcr": round(float(npcr.mean()), 4), "uaci": round(float(uaci.mean()), 4),
                    **{f"abs_corr_{d}": round(v, 5) for d, v in corr.items()}})
        e1.close()
        e2.close()
    return out


def main():
    import argparse

    import torch

    ap = argparse.ArgumentParser(description="robustness and round-count curves")
    ap.add_argument("--out", default=None)
    ap.add_argument("--map", choices=["plcm", "2dlasm", "logistic"], default="plcm")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    from . import build

    build.build()
    kind = {"plcm": 0, "2dlasm": 1, "logistic": 2}[a.map]
    res = {"map": a.map, "noise": noise_robustness(kind), "data_loss": data_loss(kind),
           "error_propagation": error_propagation(kind), "rounds": rounds_sweep(kind)}
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
