"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Holds none of the method's arithmetic: it only draws the random Young's
modulus fields that stand in for the paper's random microstructures
(Sec. 3.4 uses a low-pass-filtered Gaussian field with L_cut = 6 ell and
STD 0.3; those realisations are not published).

Recipe: z = seeded (NumPy PCG64) white noise, filtered in Fourier space with
exp(-|2 pi q|^2 lc^2 / 4) (so its covariance is proportional to
exp(-r^2 / (2 lc^2)), a Gaussian correlation of length lc pixels), shifted and
scaled to empirical zero mean and unit variance; then
E = exp(0.3 z) / mean(exp(0.3 z)).
"""
import numpy as np


def white_noise(ny, nx, seed):
    """Seeded standard normal samples, one per grid point (the xi of Sec. 3.3 before filtering)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((ny, nx))


def gaussian_field(ny, nx, lc, seed):
    """Zero-mean, unit-variance periodic Gaussian random field with correlation length lc (pixels)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((ny, nx))
    qy = np.fft.fftfreq(ny)
    qx = np.fft.fftfreq(nx)
    q2 = qy[:, None] ** 2 + qx[None, :] ** 2
    z = np.fft.ifft2(np.fft.fft2(w) * np.exp(-(2.0 * np.pi) ** 2 * q2 * lc * lc / 4.0)).real
    z -= z.mean()
    z /= z.std()
    return z


def modulus_field(ny, nx, lc, seed, amplitude=0.3):
    """E = exp(a z) / mean(exp(a z)) with z from ``gaussian_field``."""
    e = np.exp(amplitude * gaussian_field(ny, nx, lc, seed))
    return e / e.mean()


def eps_M(E0=1.0, nu=0.2, Gc=1.0, ell=1.0):
    """Homogeneous AT1 uniaxial elastic-limit strain sqrt(3 Gc / (8 ell (lambda + 2 mu))) (Sec. 3.3)."""
    lam = E0 * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E0 / (2.0 * (1.0 + nu))
    return float(np.sqrt(3.0 * Gc / (8.0 * ell * (lam + 2.0 * mu))))


# Workloads: sizes, correlation lengths, models (stated as data, used by tests and bench).
WORKLOADS = {
    "grid64_at1_spectral": dict(n=64, lc=8.0, ell=2.0, fracture="AT1", split="SPECTRAL",
                                irreversibility="CRACK_SET", increments=40, tol=1e-8),
    "grid512_fourway": dict(n=512, lc=32.0, ell=4.0, load_steps=200, tol=1e-8),
    "batch64_grid256": dict(n=256, batch=64, lc=16.0, ell=2.0, fracture="AT1", split="SPECTRAL",
                            irreversibility="CRACK_SET"),
    "grid2048_at2_spectral": dict(n=2048, lc=64.0, ell=2.0, fracture="AT2", split="SPECTRAL", load_steps=300),
}
