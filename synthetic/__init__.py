"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws *data* only: datasets shaped like the image-classification
workloads of the paper's experiments (Sec. 4: 10-class 28x28 grayscale images,
and colour images for the CNN), a small Gaussian-mixture problem, and a
linear-Gaussian regression problem whose posterior is known in closed form.
It holds none of the sampler's arithmetic: no likelihood, gradient, weight,
schedule or resampling code lives here, and it imports neither `oracle` nor the
CUDA package.  Randomness that the *method* draws (initial particles, momenta,
resampling uniforms) is not produced here either; tests pass such draws in as
explicit inputs.

All generators use numpy's PCG64 stream seeded by the caller.  A test split is
drawn with the same class structure (same seed) but an independent sample
stream, so train and test share their class templates.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_mixture",
    "template_images",
    "smooth_field_images",
    "linear_gaussian",
    "particles",
    "normals",
    "uniforms",
    "normalised_weights",
]


def _streams(seed: int, test: bool):
    """Class-structure stream (shared by train/test) and a sample stream."""
    structure = np.random.default_rng([int(seed), 0xC1A55])
    samples = np.random.default_rng([int(seed), 0x7E57 if test else 0x7121])
    return structure, samples


def _balanced_labels(rng, n: int, n_classes: int) -> np.ndarray:
    y = np.arange(n, dtype=np.int64) % n_classes
    rng.shuffle(y)
    return y.astype(np.int32)


def gaussian_mixture(n: int, d: int = 16, n_classes: int = 4, seed: int = 0,
                     test: bool = False, mean_std: float = 2.0):
    """16-d, 4-class Gaussian mixture: class means ~ N(0, mean_std^2 I) drawn
    once per seed, x = mu_y + N(0, I), labels balanced then shuffled.
    Returns (x float32 [n, d], y int32 [n])."""
    structure, samples = _streams(seed, test)
    mu = structure.normal(0.0, mean_std, size=(n_classes, d))
    y = _balanced_labels(samples, n, n_classes)
    x = mu[y] + samples.normal(size=(n, d))
    return x.astype(np.float32), y


def template_images(n: int, seed: int = 0, test: bool = False, side: int = 28,
                    n_classes: int = 10, noise_std: float = 0.3,
                    bumps: int = 3, chunk: int = 8192):
    """MNIST-shaped stand-in: per class a template made of `bumps` random 2-D
    Gaussian bumps (std 2-4 px, centres in [6, side-6]^2, peak 1, summed and
    clipped to 1); a sample is clip(T_y + N(0, noise_std^2), 0, 1).
    Returns (x float32 [n, side*side], y int32 [n])."""
    structure, samples = _streams(seed, test)
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64)
    templates = np.zeros((n_classes, side, side))
    for c in range(n_classes):
        for _ in range(bumps):
            cy, cx = structure.uniform(6.0, side - 6.0, size=2)
            s = structure.uniform(2.0, 4.0)
            templates[c] += np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s))
    templates = np.minimum(templates, 1.0).reshape(n_classes, side * side)
    y = _balanced_labels(samples, n, n_classes)
    x = np.empty((n, side * side), dtype=np.float32)
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        noise = samples.standard_normal(size=(s1 - s0, side * side), dtype=np.float32)
        x[s0:s1] = np.clip(templates[y[s0:s1]].astype(np.float32) + noise_std * noise, 0.0, 1.0)
    return x, y


def _smooth(field: np.ndarray, sigma: float) -> np.ndarray:
    """Gaussian-filter the last two axes (periodic, via FFT) and rescale each
    field to unit standard deviation."""
    h, w = field.shape[-2:]
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.fftfreq(w)[None, :]
    g = np.exp(-2.0 * (np.pi ** 2) * (sigma ** 2) * (fy ** 2 + fx ** 2))
    out = np.fft.ifft2(np.fft.fft2(field) * g).real
    sd = out.std(axis=(-2, -1), keepdims=True)
    return out / np.maximum(sd, 1e-12)


def smooth_field_images(n: int, seed: int = 0, test: bool = False, side: int = 32,
                        channels: int = 3, n_classes: int = 10, chunk: int = 4096):
    """CIFAR-shaped stand-in: per class a smooth field F_c (white noise,
    Gaussian-filtered with std 3 px, per channel, unit std); per sample a smooth
    field G_i (std 2 px, unit std); x = clip(0.5 + 0.25 (F_y + 0.5 G_i), 0, 1).
    Returns (x float32 [n, channels*side*side] in (c, h, w) order, y int32 [n])."""
    structure, samples = _streams(seed, test)
    F = _smooth(structure.normal(size=(n_classes, channels, side, side)), 3.0)
    y = _balanced_labels(samples, n, n_classes)
    x = np.empty((n, channels * side * side), dtype=np.float32)
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        G = _smooth(samples.normal(size=(s1 - s0, channels, side, side)), 2.0)
        img = np.clip(0.5 + 0.25 * (F[y[s0:s1]] + 0.5 * G), 0.0, 1.0)
        x[s0:s1] = img.reshape(s1 - s0, -1).astype(np.float32)
    return x, y


def linear_gaussian(n: int, d: int = 3, seed: int = 0, noise_std: float = 0.5,
                    test: bool = False):
    """Regression data y = x . w* + noise_std * e, x ~ N(0, I_d), w* ~ N(0, I_d)
    drawn once per seed.  Returns (x float32 [n, d], y float32 [n], w*)."""
    structure, samples = _streams(seed, test)
    w_star = structure.normal(size=d)
    x = samples.normal(size=(n, d))
    y = x @ w_star + noise_std * samples.normal(size=n)
    return x.astype(np.float32), y.astype(np.float32), w_star


def particles(J: int, D: int, seed: int, std: float = 1.0) -> np.ndarray:
    """A [J, D] float32 block of N(0, std^2) draws, used as injected initial
    particles or momenta in parity tests."""
    rng = np.random.default_rng([int(seed), 0x9A27])
    return (std * rng.standard_normal(size=(J, D))).astype(np.float32)


def normals(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng([int(seed), 0x40E5])
    return rng.standard_normal(size=shape).astype(np.float32)


def uniforms(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([int(seed), 0x0F0F])
    return rng.random(n)


def normalised_weights(J: int, seed: int, spread: float = 2.0) -> np.ndarray:
    """Random positive weights that sum to one (float64), for resampling tests."""
    rng = np.random.default_rng([int(seed), 0x3E16])
    lw = spread * rng.standard_normal(J)
    w = np.exp(lw - lw.max())
    return w / w.sum()
