"""Seeded synthetic inputs shaped like the paper's workloads.

Shared by the tests, the benchmark and the oracle's test drivers. It holds no
step of the denoising or phase-retrieval method: only random phantoms, noise,
batch size draws, transfer functions of the optical propagator (inputs of the
method, Eq. (23)) and the simulation of an intensity measurement.

All generators use numpy's PCG64 (``np.random.default_rng(seed)``) and FP64,
and round to complex64 only through ``to_c64``.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np


def to_c64(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(x.astype(np.complex64))


def phantom(m: int, n: int, seed: int, n_shapes: int = 12,
            amp=(0.5, 1.0), phase=(-math.pi, math.pi)) -> np.ndarray:
    """Piecewise-constant complex phantom: a background and ``n_shapes``
    rectangles / disks (p = 1/2 each) painted in order, each with a value
    a e^{i phi}, a ~ U[amp], phi ~ U[phase]. Rectangle sides are U[0.05, 0.4]
    times the image side at a uniform position; disk radii are U[0.03, 0.2]
    times min(m, n)."""
    rng = np.random.default_rng(seed)

    def value():
        return rng.uniform(*amp) * np.exp(1j * rng.uniform(*phase))

    x = np.full((m, n), value(), dtype=np.complex128)
    jj, kk = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    for _ in range(n_shapes):
        val = value()
        if rng.uniform() < 0.5:
            h = max(1, int(round(rng.uniform(0.05, 0.4) * m)))
            w = max(1, int(round(rng.uniform(0.05, 0.4) * n)))
            j0 = int(rng.integers(0, max(1, m - h + 1)))
            k0 = int(rng.integers(0, max(1, n - w + 1)))
            x[j0:j0 + h, k0:k0 + w] = val
        else:
            rad = rng.uniform(0.03, 0.2) * min(m, n)
            cj, ck = rng.uniform(0, m), rng.uniform(0, n)
            x[(jj - cj) ** 2 + (kk - ck) ** 2 <= rad * rad] = val
    return x


def complex_noise(shape, sigma: float, seed: int) -> np.ndarray:
    """Circular complex Gaussian CN(0, sigma^2): real and imaginary parts are
    independent N(0, sigma^2 / 2)."""
    rng = np.random.default_rng(seed)
    s = sigma / math.sqrt(2.0)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


def noisy_phantom(m: int, n: int, sigma: float, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """(clean, noisy) complex128 pair; round with ``to_c64`` before use."""
    clean = phantom(m, n, seed)
    return clean, clean + complex_noise((m, n), sigma, seed + 7919)


def support_rect(m: int, n: int) -> Tuple[int, int, int, int]:
    """Rectangular support [m/8, 7m/8) x [n/8, 7n/8) as (j0, k0, j1, k1)."""
    return (m // 8, n // 8, (7 * m) // 8, (7 * n) // 8)


def batch_shapes(count: int, lo: int, hi: int, seed: int) -> List[Tuple[int, int]]:
    """Image sides m and n drawn independently and log-uniformly in [lo, hi]."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(math.log(lo), math.log(hi), size=(count, 2))
    return [(int(round(math.exp(a))), int(round(math.exp(b)))) for a, b in e]


def batch_params(count: int, seed: int):
    """Per-image lambda ~ U[0.01, 0.1] and TV type uniform over the four types."""
    rng = np.random.default_rng(seed)
    lams = rng.uniform(0.01, 0.1, size=count)
    types = rng.integers(0, 4, size=count)
    return lams, types


# --------------------------------------------------------------------------
# Phase-retrieval inputs
# --------------------------------------------------------------------------
def gaussian_blur(img: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(img, sigma, mode="nearest")


def pr_object(m: int, n: int, seed: int, amp=(0.6, 1.0), blur_sigma: float = 8.0) -> np.ndarray:
    """Object with piecewise-constant amplitude in [0.6, 1] and a smooth phase:
    the phase of a phantom, Gaussian-blurred and rescaled to [0, pi]."""
    a = np.abs(phantom(m, n, seed, amp=(0.0, 1.0)))
    a = amp[0] + (amp[1] - amp[0]) * (a - a.min()) / max(a.max() - a.min(), 1e-12)
    ph = np.angle(phantom(m, n, seed + 1))
    ph = gaussian_blur(ph, blur_sigma)
    ph = math.pi * (ph - ph.min()) / max(ph.max() - ph.min(), 1e-12)
    return a * np.exp(1j * ph)


def freq_grid(M: int, N: int, dx: float):
    fy = np.fft.fftfreq(M, d=dx)
    fx = np.fft.fftfreq(N, d=dx)
    return np.meshgrid(fy, fx, indexing="ij")


def fresnel_tf(M: int, N: int, wavelength: float, dx: float, z: float) -> np.ndarray:
    """Fresnel transfer function exp(i k z) exp(-i pi wavelength z (fx^2 + fy^2))
    on the FFT frequency grid of an M x N field with pixel pitch dx."""
    FY, FX = freq_grid(M, N, dx)
    k = 2 * math.pi / wavelength
    return np.exp(1j * k * z) * np.exp(-1j * math.pi * wavelength * z * (FX ** 2 + FY ** 2))


def angular_spectrum_tf(M: int, N: int, wavelength: float, dx: float, z: float) -> np.ndarray:
    """Transfer function of Eq. (23): exp(i 2 pi z / wavelength sqrt(1 - (wl fx)^2 - (wl fy)^2)),
    with the evanescent part (negative radicand) set to 0."""
    FY, FX = freq_grid(M, N, dx)
    arg = 1.0 - (wavelength * FX) ** 2 - (wavelength * FY) ** 2
    H = np.exp(1j * 2 * math.pi * z / wavelength * np.sqrt(np.maximum(arg, 0.0)))
    return np.where(arg >= 0, H, 0.0)


def simulate_intensity(x: np.ndarray, H: np.ndarray, seed: int, photons: float = 1e4) -> np.ndarray:
    """Measured intensity y = Poisson(photons |A x|^2) / photons, where A pads x
    into the top-left corner of H's grid, applies H in the Fourier domain and
    crops back (the measurement model of Sec. V-A). photons <= 0 gives y = |A x|^2."""
    m, n = x.shape
    M, N = H.shape
    buf = np.zeros((M, N), dtype=np.complex128)
    buf[:m, :n] = x
    xi = np.fft.ifft2(np.fft.fft2(buf) * H)[:m, :n]
    y = np.abs(xi) ** 2
    if photons > 0:
        rng = np.random.default_rng(seed)
        y = rng.poisson(photons * y) / photons
    return y


def phase_object(m: int, n: int, seed: int) -> np.ndarray:
    """Pure phase object exp(i phi) with a piecewise-constant phi in [0, pi]
    (the phase of a phantom, rescaled), standing in for the test images of the
    paper's simulated phase-retrieval experiments."""
    ph = np.angle(phantom(m, n, seed))
    ph = math.pi * (ph - ph.min()) / max(ph.max() - ph.min(), 1e-12)
    return np.exp(1j * ph)


def intensity_with_gaussian_noise(x: np.ndarray, H: np.ndarray, level: float, seed: int) -> np.ndarray:
    """y = |A x|^2 + n, n ~ N(0, (level * mean |A x|^2)^2), clipped at 0 (the
    "10% Gaussian noise added to the calculated intensity" of Sec. VI-A, read as
    a standard deviation of level times the mean intensity)."""
    y = simulate_intensity(x, H, seed, photons=0)
    rng = np.random.default_rng(seed)
    return np.maximum(y + rng.normal(0.0, level * float(y.mean()), y.shape), 0.0)


def phase_rmse(x: np.ndarray, x_true: np.ndarray) -> float:
    """RMSE of the phase of x against x_true with the global phase offset removed
    (the error measure of Sec. VI-A)."""
    d = np.angle(x * np.conj(x_true))
    d = np.angle(np.exp(1j * (d - np.angle(np.exp(1j * d).mean()))))
    return float(np.sqrt((d ** 2).mean()))
