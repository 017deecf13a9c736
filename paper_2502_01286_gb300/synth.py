"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on three photographs (Socket 539x959, Darts 538x508,
Split city 4032x3024; Section 6, Table 1) that are not available, so these
generators stand in for them.  This module holds none of the method's
arithmetic: it only makes source images and templates, so both the CUDA path
and the CPU oracle draw identical inputs from it.  It depends on numpy alone.

Recipe (every parameter the paper leaves open is a stated choice):
  blobs        base 128 + sum_j A_j exp(-r^2 / (2 s_j^2)), A_j ~ U(-100, 100),
               centres uniform over the image, s_j ~ U(8, 40) px
  uniform      additive U(-a, a) noise
  fractal      white Gaussian noise whose FFT amplitude is scaled by 1/|w|
               (DC removed), rescaled so that its standard deviation
               ("rms") or its largest magnitude ("max") equals the amplitude;
               the HD case uses rms (so the swept thresholds 5/10/20 stay
               below the template's std, as Section 3 requires), the
               high-texture case uses max (several thousand segments at
               threshold 5)
  rectangles   axis-aligned rectangles, sides U(4, 512), intensity U(0, 255),
               painted in order over a mid-grey canvas
  quantise     clip to [0, 255], round half to even, uint8
  template     crop at a seeded uniform offset, plus N(0, sigma^2) noise,
               rounded and clipped
Generator: numpy Generator(PCG64(seed)).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 2502012860


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def blobs(g: np.random.Generator, M: int, N: int, count: int = 20, base: float = 128.0) -> np.ndarray:
    """Float image (N, M): base plus `count` Gaussian blobs."""
    img = np.full((N, M), base, np.float64)
    yy = np.arange(N, dtype=np.float64)[:, None]
    xx = np.arange(M, dtype=np.float64)[None, :]
    for _ in range(count):
        a = g.uniform(-100.0, 100.0)
        cx = g.uniform(0.0, M)
        cy = g.uniform(0.0, N)
        s = g.uniform(8.0, 40.0)
        img += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * s * s))
    return img


def fractal_noise(g: np.random.Generator, M: int, N: int, amplitude: float, scale: str = "max") -> np.ndarray:
    """1/f noise (N, M) whose max |value| (scale="max") or standard deviation
    (scale="rms") equals amplitude."""
    w = g.standard_normal((N, M))
    F = np.fft.rfft2(w)
    fy = np.fft.fftfreq(N)[:, None]
    fx = np.fft.rfftfreq(M)[None, :]
    r = np.sqrt(fx * fx + fy * fy)
    r[0, 0] = 1.0
    F = F / r
    F[0, 0] = 0.0
    out = np.fft.irfft2(F, s=(N, M))
    m = np.std(out) if scale == "rms" else np.max(np.abs(out))
    return out * (amplitude / m) if m > 0 else out


def rectangles(g: np.random.Generator, M: int, N: int, count: int = 300) -> np.ndarray:
    img = np.full((N, M), 128.0)
    for _ in range(count):
        w = int(g.integers(4, 513))
        h = int(g.integers(4, 513))
        x = int(g.integers(-w + 1, M))
        y = int(g.integers(-h + 1, N))
        val = float(g.integers(0, 256))
        img[max(y, 0):max(min(y + h, N), 0), max(x, 0):max(min(x + w, M), 0)] = val
    return img


def quantise(img: np.ndarray) -> np.ndarray:
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)


def crop_template(g: np.random.Generator, f: np.ndarray, W: int, H: int, noise_sigma: float):
    """Crop W x H at a seeded uniform offset and add N(0, sigma^2) noise.
    Returns (template uint8 (H, W), (u0, v0))."""
    N, M = f.shape
    u0 = int(g.integers(0, M - W + 1))
    v0 = int(g.integers(0, N - H + 1))
    crop = f[v0:v0 + H, u0:u0 + W].astype(np.float64)
    if noise_sigma > 0:
        crop = crop + g.normal(0.0, noise_sigma, size=crop.shape)
    return quantise(crop), (u0, v0)


@dataclass
class Case:
    name: str
    f: np.ndarray          # (N, M) uint8 or float32
    t: np.ndarray          # (H, W)
    origin: tuple          # crop offset (u0, v0)
    sigma_max: float       # split-and-merge std threshold
    precision: float       # coarse precision p (tau_c = p * rho_max)
    seed: int


def case_plain(M: int = 256, N: int = 256, W: int = 32, H: int = 32, seed: int = BASE_SEED + 0,
               noise: float = 2.0, sigma_max: float = 10.0, precision: float = 0.9) -> Case:
    """Blobs (20) plus U(-4, 4) noise; a template cropped with Gaussian noise."""
    g = rng(seed)
    img = blobs(g, M, N, 20) + g.uniform(-4.0, 4.0, size=(N, M))
    f = quantise(img)
    t, org = crop_template(g, f, W, H, noise)
    return Case("plain", f, t, org, sigma_max, precision, seed)


def case_hd(M: int = 1920, N: int = 1080, W: int = 64, H: int = 64, seed: int = BASE_SEED + 1,
            noise: float = 3.0, sigma_max: float = 10.0, precision: float = 0.85) -> Case:
    """Blobs plus 1/f fractal noise of rms amplitude 60; a template with sigma-3 noise."""
    g = rng(seed)
    img = blobs(g, M, N, 20) + fractal_noise(g, M, N, 60.0, "rms")
    f = quantise(img)
    t, org = crop_template(g, f, W, H, noise)
    return Case("hd", f, t, org, sigma_max, precision, seed)


def case_texture(M: int = 4096, N: int = 4096, W: int = 256, H: int = 256, seed: int = BASE_SEED + 2,
                 noise: float = 0.0, sigma_max: float = 5.0, precision: float = 0.85) -> Case:
    """Random rectangles plus 1/f noise of peak amplitude 40 (high texture)."""
    g = rng(seed)
    img = rectangles(g, M, N, 300) + fractal_noise(g, M, N, 40.0, "max")
    f = quantise(img)
    t, org = crop_template(g, f, W, H, noise)
    return Case("texture", f, t, org, sigma_max, precision, seed)


def batch_sources(count: int = 8, M: int = 1024, N: int = 1024, seed: int = BASE_SEED + 3) -> list:
    """Sources of the batched workload: blobs plus 1/f noise of rms amplitude
    60 (the HD reading, so thresholds up to 25 stay below template stds)."""
    g = rng(seed)
    return [quantise(blobs(g, M, N, 20) + fractal_noise(g, M, N, 60.0, "rms")) for _ in range(count)]


def batch_templates(sources: list, count: int = 64, seed: int = BASE_SEED + 4, lo: int = 16, hi: int = 256):
    """Templates with sides U{lo..hi} (independently, so non-square), cropped
    from the sources in turn, and std thresholds U(4, 25)."""
    g = rng(seed)
    out = []
    for i in range(count):
        W = int(g.integers(lo, hi + 1))
        H = int(g.integers(lo, hi + 1))
        src = sources[i % len(sources)]
        t, org = crop_template(g, src, W, H, 2.0)
        sigma = float(g.uniform(4.0, 25.0))
        out.append((t, org, sigma))
    return out


def random_image(seed: int, M: int, N: int, lo: int = 0, hi: int = 256) -> np.ndarray:
    """Uniform random uint8 image (N, M) for small edge-case tests."""
    return rng(seed).integers(lo, hi, size=(N, M), dtype=np.int64).astype(np.uint8)


def random_image_u8(seed: int, M: int, N: int, lo: int = 0, hi: int = 256) -> np.ndarray:
    """Uniform random uint8 image (N, M) drawn as bytes directly, for sources
    of hundreds of megapixels."""
    return rng(seed).integers(lo, hi, size=(N, M), dtype=np.uint8)


def case_diff(M: int = 512, N: int = 512, W: int = 48, H: int = 48, seed: int = BASE_SEED + 5,
              noise: float = 2.0, sigma_max: float = 12.0):
    """Float source for the differentiation workload: 20 blobs plus 1/f noise
    of rms 30 (so the std threshold 12 stays below the template's std, as
    Section 3 requires), scaled linearly to [0, 255] (float32, not quantised);
    the template is a W x H crop plus N(0, noise^2), float32.
    Returns (f, t, origin, sigma)."""
    g = rng(seed)
    img = blobs(g, M, N, 20) + fractal_noise(g, M, N, 30.0, "rms")
    img = (img - img.min()) * (255.0 / (img.max() - img.min()))
    f = img.astype(np.float32)
    u0 = int(g.integers(0, M - W + 1))
    v0 = int(g.integers(0, N - H + 1))
    t = (f[v0:v0 + H, u0:u0 + W].astype(np.float64) + g.normal(0.0, noise, size=(H, W))).astype(np.float32)
    return f, t, (u0, v0), sigma_max
