"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the cipher's arithmetic: it only draws keys inside the
paper's valid parameter ranges (Eq. 5, Eq. 6; the logistic map's r in [3.9, 4])
and makes HWC uint8 video frames.
The paper's own inputs (its test images and the trace-library videos of its
speed evaluation, Sec. 3) are not available; these generators stand in for
them:

* ``uniform_frames``: i.i.d. uniform bytes.
* ``smooth_clip``: a video with the strong adjacent-pixel correlation of natural
  footage -- per-channel linear gradients, 8 Gaussian blobs moving on straight
  lines at 1-4 px/frame, and N(0, 4^2) noise, rounded and clipped to [0, 255].
"""
from __future__ import annotations

import numpy as np

PLCM, DLASM, LOGISTIC = 0, 1, 2


def key_for_seed(kind: int, seed: int) -> list[float]:
    """A key drawn with numpy PCG64 from ``seed``.

    PLCM (Eq. 5): x0 ~ U(0.01, 0.99) avoiding |x0 - 0.5| < 1e-3 and
    p ~ U(0.01, 0.49) avoiding |p - 0.25| < 1e-3, for both maps.
    2DLASM (Eq. 6): x0, y0 ~ U(0.01, 0.99), mu ~ U(0.44, 0.93); returned as
    (x0, mu, y0), the order of the paper's key.
    Logistic map (the third map): x0 ~ U(0.01, 0.99) avoiding |x0 - 0.5| < 1e-3
    and r ~ U(3.9, 4.0), for both maps.
    """
    rng = np.random.Generator(np.random.PCG64(seed))

    def draw(lo, hi, avoid):
        while True:
            v = float(rng.uniform(lo, hi))
            if abs(v - avoid) >= 1e-3:
                return v

    if kind == PLCM:
        return [draw(0.01, 0.99, 0.5), draw(0.01, 0.49, 0.25),
                draw(0.01, 0.99, 0.5), draw(0.01, 0.49, 0.25)]
    if kind == DLASM:
        x0 = float(rng.uniform(0.01, 0.99))
        mu = float(rng.uniform(0.44, 0.93))
        y0 = float(rng.uniform(0.01, 0.99))
        return [x0, mu, y0]
    if kind == LOGISTIC:
        return [draw(0.01, 0.99, 0.5), float(rng.uniform(3.9, 4.0)),
                draw(0.01, 0.99, 0.5), float(rng.uniform(3.9, 4.0))]
    raise ValueError(kind)


def uniform_frames(nframes: int, H: int, W: int, C: int = 3, seed: int = 1) -> np.ndarray:
    """``nframes`` x H x W x C uniform random bytes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 256, size=(nframes, H, W, C), dtype=np.uint8)


def smooth_clip(nframes: int, H: int, W: int, C: int = 3, seed: int = 2,
                nblobs: int = 8, noise_sigma: float = 4.0) -> np.ndarray:
    """A smooth synthetic clip (see module docstring), ``nframes`` x H x W x C."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yy = np.arange(H, dtype=np.float32)[:, None]
    xx = np.arange(W, dtype=np.float32)[None, :]
    base = np.empty((H, W, C), dtype=np.float32)
    for ch in range(C):
        gy, gx = rng.uniform(-0.25, 0.25, size=2) * 256.0 / max(H, W)
        off = rng.uniform(64, 192)
        base[:, :, ch] = off + gy * (yy - H / 2) + gx * (xx - W / 2)
    sig = rng.uniform(20, 60, size=nblobs).astype(np.float32)
    amp = (rng.uniform(40, 80, size=(nblobs, C)) * rng.choice([-1.0, 1.0], size=(nblobs, C))).astype(np.float32)
    pos0 = np.stack([rng.uniform(0, H, nblobs), rng.uniform(0, W, nblobs)], axis=1)
    speed = rng.uniform(1, 4, nblobs)
    ang = rng.uniform(0, 2 * np.pi, nblobs)
    vel = np.stack([speed * np.sin(ang), speed * np.cos(ang)], axis=1)
    out = np.empty((nframes, H, W, C), dtype=np.uint8)
    for f in range(nframes):
        img = base.copy()
        for b in range(nblobs):
            cy, cx = pos0[b] + vel[b] * f
            cy, cx = cy % H, cx % W
            r = int(3 * sig[b]) + 1
            y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
            x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
            if y0 >= y1 or x0 >= x1:
                continue
            dy = (yy[y0:y1] - np.float32(cy)) ** 2
            dx = (xx[:, x0:x1] - np.float32(cx)) ** 2
            g = np.exp(-(dy + dx) / np.float32(2 * sig[b] * sig[b]))
            img[y0:y1, x0:x1, :] += g[:, :, None] * amp[b][None, None, :]
        img += rng.normal(0.0, noise_sigma, size=img.shape).astype(np.float32)
        np.clip(np.rint(img), 0, 255, out=img)
        out[f] = img.astype(np.uint8)
    return out


def serving_workload(nstreams: int, seed: int = 5, rate_per_s: float = 64.0,
                     resolutions=((480, 480), (576, 576), (768, 768), (720, 1280), (1080, 1920), (2160, 3840)),
                     fps_choices=(24, 30, 60), duration_s=(2.0, 6.0)) -> list[dict]:
    """Seeded stream requests for the serving loop: Poisson arrivals at
    ``rate_per_s``, each stream with its own key (map alternating PLCM /
    2DLASM), a resolution (H, W) from ``resolutions``, a frame rate from
    ``fps_choices``, encrypt or decrypt (50/50) and a duration."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for s in range(nstreams):
        t += float(rng.exponential(1.0 / rate_per_s))
        kind = s % 2
        H, W = resolutions[int(rng.integers(len(resolutions)))]
        out.append({"sid": s, "arrival": t, "kind": kind, "key": key_for_seed(kind, 1000 + s), "H": H, "W": W,
                    "C": 3, "fps": int(fps_choices[int(rng.integers(len(fps_choices)))]),
                    "direction": int(rng.integers(2)), "duration": float(rng.uniform(*duration_s))})
    return out
