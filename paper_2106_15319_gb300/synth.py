"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no Serial-EMD arithmetic: it only draws signals and noise with
numpy's PCG64 generator. Both the CUDA path and the CPU oracle consume what it
returns, so neither side depends on the other.

Stand-ins for the paper's data (its datasets are not available here):
  * multivariate tone + chirp series   -> the 6-variate synthetic set of Sec. 4.1
  * oriented 2D sinusoidal gratings    -> the artificial texture image of Sec. 4.2
  * smooth blob fields with a grating  -> the AT&T face images of Sec. 4.3
Every generator takes an explicit seed; the default seeds are 20210629 + workload
number, so the workloads named below are reproducible run to run.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20210629


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def tone_chirp_series(channels: int, samples: int, seed: int, f1=(60.0, 120.0),
                      f2=(5.0, 15.0), chirp=(5.0, 40.0), noise_std: float = 0.05,
                      duration: float = 1.0) -> np.ndarray:
    """(channels, samples) series: sin(2 pi f1 t) + 0.5 sin(2 pi f2 t) + linear chirp + noise.

    t = n / samples * duration, n < samples. f1 ~ U[f1], f2 ~ U[f2] per channel; the
    chirp sweeps chirp[0] -> chirp[1] Hz over the duration.
    """
    g = rng(seed)
    t = np.arange(samples, dtype=np.float64) / samples * duration
    a = chirp[0]
    b = (chirp[1] - chirp[0]) / (2.0 * duration)
    out = np.empty((channels, samples), np.float64)
    for c in range(channels):
        fa = g.uniform(*f1)
        fb = g.uniform(*f2)
        out[c] = (np.sin(2 * np.pi * fa * t) + 0.5 * np.sin(2 * np.pi * fb * t)
                  + np.sin(2 * np.pi * (a * t + b * t * t))
                  + g.normal(0.0, noise_std, samples))
    return out


def grating_image(side: int, seed: int, periods=(4.0, 16.0, 64.0),
                  noise_std: float = 0.05) -> np.ndarray:
    """(side, side) sum of oriented sinusoidal gratings (random angle, phase) + noise."""
    g = rng(seed)
    y, x = np.mgrid[0:side, 0:side].astype(np.float64)
    img = np.zeros((side, side), np.float64)
    for p in periods:
        th = g.uniform(0.0, np.pi)
        ph = g.uniform(0.0, 2 * np.pi)
        img += np.sin(2 * np.pi * (x * np.cos(th) + y * np.sin(th)) / p + ph)
    img += g.normal(0.0, noise_std, (side, side))
    return img


def blob_field(side: int, g: np.random.Generator, blobs: int = 6,
               noise_std: float = 0.02) -> np.ndarray:
    """Smooth face-like field: anisotropic Gaussian blobs + a fine grating + noise."""
    y, x = np.mgrid[0:side, 0:side].astype(np.float64)
    img = np.zeros((side, side), np.float64)
    for _ in range(blobs):
        A = g.uniform(0.5, 1.5)
        cx, cy = g.uniform(0, side, 2)
        sx, sy = g.uniform(side / 16.0, side / 4.0, 2)
        rot = g.uniform(0.0, np.pi)
        dx, dy = x - cx, y - cy
        u = dx * np.cos(rot) + dy * np.sin(rot)
        v = -dx * np.sin(rot) + dy * np.cos(rot)
        img += A * np.exp(-0.5 * ((u / sx) ** 2 + (v / sy) ** 2))
    period = g.uniform(3.0, 8.0)
    th = g.uniform(0.0, np.pi)
    ph = g.uniform(0.0, 2 * np.pi)
    img += 0.3 * np.sin(2 * np.pi * (x * np.cos(th) + y * np.sin(th)) / period + ph)
    img += g.normal(0.0, noise_std, (side, side))
    return img


def uneven_images(count: int, seed: int, side_range=(32, 128)) -> list[np.ndarray]:
    """count square blob fields, side ~ U{side_range[0] .. side_range[1]}."""
    g = rng(seed)
    sides = g.integers(side_range[0], side_range[1] + 1, size=count)
    return [blob_field(int(s), g) for s in sides]


def white_noise(trials: int, length: int, seed: int) -> np.ndarray:
    """(trials, length) standard normal realizations w^(m) for EEMD."""
    return rng(seed).standard_normal((trials, length))


def serving_mix(count: int, seed: int, rate_hz: float, big_fraction: float = 0.02,
                big_side: int = 2048, max_series: int = 65536, max_side: int = 1024):
    """Poisson arrival times plus request shapes for the serving mix.

    Half the requests are tone+chirp series (2..16 channels x 1k..64k samples, log-
    uniform length), half are grating images (side log-uniform 32..1024); a small
    fraction are big_side^2 images (4M samples). Returns a list of
    (arrival_s, kind, array) with arrival times from exponential gaps at rate_hz.
    """
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += g.exponential(1.0 / rate_hz)
        s = int(g.integers(0, 2**31 - 1))
        if g.uniform() < big_fraction:
            out.append((t, "image", grating_image(big_side, s)))
        elif g.uniform() < 0.5:
            ch = int(g.integers(2, 17))
            n = int(round(math.exp(g.uniform(math.log(1024), math.log(max_series)))))
            out.append((t, "series", tone_chirp_series(ch, n, s)))
        else:
            side = int(round(math.exp(g.uniform(math.log(32), math.log(max_side)))))
            out.append((t, "image", grating_image(side, s)))
    return out


# --- the named workloads (seeds SEED_BASE + workload number) -----------------------------

def workload_series_3x1024() -> np.ndarray:
    """3-channel series, 1024 samples per channel (tones + chirp + N(0, 0.05^2))."""
    return tone_chirp_series(3, 1024, SEED_BASE + 1)


def workload_texture_256() -> np.ndarray:
    """256 x 256 texture: gratings of period 4, 16, 64 px + N(0, 0.05^2)."""
    return grating_image(256, SEED_BASE + 2)


def workload_uneven_images(count: int = 2048) -> list[np.ndarray]:
    """count blob-field images with side U{32..128}."""
    return uneven_images(count, SEED_BASE + 3)


def workload_eemd_512(trials: int = 256):
    """512 x 512 grating image and (trials, 262144) white noise for EEMD."""
    img = grating_image(512, SEED_BASE + 4)
    w = white_noise(trials, 512 * 512, SEED_BASE + 40)
    return img, w


def paper_mask_components(samples: int = 1000, fs: float = 1000.0):
    """The parts of the 6-variate tone set of Sec. 4.1: the tones 32/16/8/2 Hz (4, samples)
    and the pickup mask (4 tones x 6 variates U..Z). The sample rate is not printed in
    the paper; 1 kHz and 1000 samples are assumed."""
    mask = np.array([[1, 1, 0, 1, 0, 0],
                     [1, 1, 1, 0, 1, 0],
                     [1, 1, 1, 1, 1, 1],
                     [1, 0, 1, 1, 0, 1]], np.float64)
    f = np.array([32.0, 16.0, 8.0, 2.0])
    t = np.arange(samples) / fs
    tones = np.sin(2 * np.pi * f[:, None] * t[None, :])
    return tones, mask


def paper_mask_series(samples: int = 1000, fs: float = 1000.0) -> np.ndarray:
    """The 6-variate tone set of Sec. 4.1 (6, samples): variate v is the sum of the tones
    the mask picks for it."""
    tones, mask = paper_mask_components(samples, fs)
    return (mask.T @ tones).astype(np.float64)
