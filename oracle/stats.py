"""Statistical and security measures of Sec. 4 and Sec. 5 (CPU, numpy).

Test infrastructure: used to check the paper's statistical claims on the
cipher's output (oracle and CUDA path alike).  Each function cites the passage
that defines it.
"""
from __future__ import annotations

import math

import numpy as np


def histogram(channel: np.ndarray) -> np.ndarray:
    """Counts z_0..z_255 of one channel (Sec. 4.1)."""
    return np.bincount(np.asarray(channel, dtype=np.uint8).ravel(), minlength=256).astype(np.float64)


def hist_variance(channel: np.ndarray) -> float:
    """var(Z) = 1/256^2 * sum_i sum_j (z_i - z_j)^2 / 2   (Sec. 4.1)."""
    z = histogram(channel)
    d = z[:, None] - z[None, :]
    return float((0.5 * d * d).sum() / 256.0 ** 2)


def chi_square(channel: np.ndarray) -> float:
    """chi^2 = sum_i (z_i - N/256)^2 / (N/256)   (Sec. 4.1)."""
    z = histogram(channel)
    e = z.sum() / 256.0
    return float(((z - e) ** 2 / e).sum())


CHI2_CRITICAL_255_005 = 293.25  # chi^2(0.05, 255) as printed in Sec. 4.1


def adjacent_pairs(channel: np.ndarray, direction: str, npairs: int, seed: int):
    """``npairs`` random pairs of horizontally/vertically/diagonally adjacent
    pixels (Sec. 4.2)."""
    a = np.asarray(channel)
    H, W = a.shape
    rng = np.random.Generator(np.random.PCG64(seed))
    dy, dx = {"H": (0, 1), "V": (1, 0), "D": (1, 1)}[direction]
    ys = rng.integers(0, H - dy, size=npairs)
    xs = rng.integers(0, W - dx, size=npairs)
    return a[ys, xs].astype(np.float64), a[ys + dy, xs + dx].astype(np.float64)


def correlation(x: np.ndarray, y: np.ndarray) -> float:
    """r = cov(x, y) / sqrt(D(x) D(y)) with 1/N moments (Sec. 4.2)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ex, ey = x.mean(), y.mean()
    cov = ((x - ex) * (y - ey)).mean()
    dx = ((x - ex) ** 2).mean()
    dy = ((y - ey) ** 2).mean()
    return float(cov / math.sqrt(dx * dy))


def entropy(channel: np.ndarray) -> float:
    """H(m) = sum p log2(1/p) over the 256 symbols (Sec. 4.3)."""
    z = histogram(channel)
    p = z[z > 0] / z.sum()
    return float(-(p * np.log2(p)).sum())


def local_entropy(channel: np.ndarray, k: int = 30, tb: int = 1936, seed: int = 0) -> float:
    """(k, T_B) local Shannon entropy: mean entropy of k random non-overlapping
    blocks of T_B pixels (square blocks of side sqrt(T_B) = 44) (Sec. 4.3)."""
    a = np.asarray(channel)
    H, W = a.shape
    side = int(round(math.sqrt(tb)))
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = [(by, bx) for by in range(H // side) for bx in range(W // side)]
    pick = rng.choice(len(cells), size=min(k, len(cells)), replace=False)
    hs = [entropy(a[cells[c][0] * side:(cells[c][0] + 1) * side, cells[c][1] * side:(cells[c][1] + 1) * side])
          for c in pick]
    return float(np.mean(hs))


def npcr(c1: np.ndarray, c2: np.ndarray) -> float:
    """NPCR = sum D(i,j) / (w h) * 100%, D = [c1 != c2]   (Sec. 5.2)."""
    return float((np.asarray(c1) != np.asarray(c2)).mean() * 100.0)


def uaci(c1: np.ndarray, c2: np.ndarray) -> float:
    """UACI = sum |c1 - c2| / (w h 255) * 100%   (Sec. 5.2)."""
    d = np.abs(np.asarray(c1, dtype=np.int32) - np.asarray(c2, dtype=np.int32))
    return float(d.mean() / 255.0 * 100.0)


def npcr_uaci_critical(width: int, height: int, alpha: float = 0.05):
    """Critical values of the NPCR/UACI randomness tests for a w x h 8-bit
    image (Sec. 5.2 quotes them for 512 x 512 at alpha = 0.05):

    NPCR* = (F - z_alpha * sqrt(F / (w h))) / (F + 1),
    UACI*- / UACI*+ = mu_U -/+ z_{alpha/2} * sigma_U, with
    mu_U = (F + 2) / (3F + 3),
    sigma_U^2 = (F + 2)(F^2 + 2F + 3) / (18 (F + 1)^2 w h F),  F = 255.
    Returned in percent.
    """
    from scipy.stats import norm

    F = 255.0
    MN = float(width) * float(height)
    z1 = norm.ppf(1.0 - alpha)
    z2 = norm.ppf(1.0 - alpha / 2.0)
    n_star = (F - z1 * math.sqrt(F / MN)) / (F + 1.0)
    mu = (F + 2.0) / (3.0 * F + 3.0)
    sig = math.sqrt((F + 2.0) * (F * F + 2.0 * F + 3.0) / (18.0 * (F + 1.0) ** 2 * MN * F))
    return n_star * 100.0, (mu - z2 * sig) * 100.0, (mu + z2 * sig) * 100.0
