"""Seeded synthetic inputs for the thermal LBM workloads.

This module holds no lattice Boltzmann arithmetic: it only builds host FP64
initial fields (density rho, lattice-unit velocity U, and theta = T / T0, the
temperature in units of the model's reference temperature) from a seed.  The
caller converts theta to lattice units with its own T0, so the CUDA path and
the FP64 oracle consume the identical arrays.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
evaluated at (seed, linear cell index); doubles take the top 53 bits.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_SEEDMUL = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counter ``index`` (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        z = (index.astype(np.uint64) + np.uint64(1)) * _GOLDEN + np.uint64(seed) * _SEEDMUL
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, index: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, index) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on counters (2k, 2k+1)."""
    k = np.arange(n, dtype=np.uint64)
    u1 = uniform01(seed, 2 * k)
    u2 = uniform01(seed, 2 * k + 1)
    r = np.sqrt(-2.0 * np.log1p(-u1))           # 1 - u1 in (0, 1]
    return r * np.cos(2.0 * np.pi * u2)


@dataclass
class Fields:
    """Initial fields on an [Nz, Ny, Nx] grid (x fastest)."""
    rho: np.ndarray                 # [Nz, Ny, Nx]
    U: np.ndarray                   # [D, Nz, Ny, Nx], lattice units
    theta: np.ndarray               # [Nz, Ny, Nx], T / T0
    meta: dict = field(default_factory=dict)


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x, y, z


def riemann_planar(D, nx, ny, nz, split, left, right, seed=1, noise=1e-4):
    """Planar diaphragm normal to x: cells with x < split take ``left`` = (rho, theta),
    the others ``right``; U = 0; uniform noise in [-noise, noise) added to rho."""
    x, _, _ = _grid(nx, ny, nz)
    rho = np.where(x < split, left[0], right[0]).astype(np.float64)
    theta = np.where(x < split, left[1], right[1]).astype(np.float64)
    if noise:
        idx = np.arange(rho.size, dtype=np.uint64).reshape(rho.shape)
        rho = rho + noise * (2.0 * uniform01(seed, idx) - 1.0)
    U = np.zeros((D,) + rho.shape)
    return Fields(rho, U, theta, {"diaphragm": "x<%d" % split, "left": left, "right": right,
                                  "seed": seed, "noise": noise})


def riemann_oblique(nx, ny, nz, left, right, seed=1, noise=1e-4):
    """Diaphragm plane with normal (1,1,0)/sqrt(2) through the centre:
    s = (i - nx/2) + (j - ny/2); left state where s < 0, right state otherwise."""
    x, y, _ = _grid(nx, ny, nz)
    s = (x - nx // 2) + (y - ny // 2)
    rho = np.where(s < 0, left[0], right[0]).astype(np.float64)
    theta = np.where(s < 0, left[1], right[1]).astype(np.float64)
    if noise:
        idx = np.arange(rho.size, dtype=np.uint64).reshape(rho.shape)
        rho = rho + noise * (2.0 * uniform01(seed, idx) - 1.0)
    U = np.zeros((3,) + rho.shape)
    return Fields(rho, U, theta, {"diaphragm": "oblique (1,1,0)", "seed": seed})


def gaussian_random_field(nx, ny, nz, seed, corr_len=4.0, rms=1e-3):
    """White N(0,1) per cell convolved periodically with a Gaussian kernel of
    standard deviation corr_len/sqrt(2) (field correlation exp(-r^2/(2 corr_len^2))),
    scaled to the given RMS."""
    w = normal(seed, nx * ny * nz).reshape(nz, ny, nx)
    sig = corr_len / np.sqrt(2.0)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.fftfreq(nx)[None, None, :]
    k2 = (2 * np.pi) ** 2 * (kx * kx + ky * ky + kz * kz)
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.5 * sig * sig * k2)))
    f = f - f.mean()
    return f * (rms / np.sqrt((f * f).mean()))


def sphere_field(nx, ny, nz, seed, radius=16, hot=1.2, corr_len=4.0, rms=1e-3):
    """rho = 1 + Gaussian random field; theta = hot inside the integer sphere
    (i-cx)^2 + (j-cy)^2 + (k-cz)^2 <= radius^2 at the centre, else 1; U = 0."""
    x, y, z = _grid(nx, ny, nz)
    rho = 1.0 + gaussian_random_field(nx, ny, nz, seed, corr_len, rms)
    r2 = (x - nx // 2) ** 2 + (y - ny // 2) ** 2 + (z - nz // 2) ** 2
    theta = np.where(r2 <= radius * radius, hot, 1.0)
    U = np.zeros((3,) + rho.shape)
    return Fields(rho, U, theta.astype(np.float64), {"seed": seed, "radius": radius})


# ------------------------------------------------------------------ named workloads

@dataclass(frozen=True)
class Workload:
    name: str
    model: str               # "D2Q33" or "D3Q95"
    storage: str             # "fp64", "fp32", "fp16", "bf16"
    dims: tuple              # (nx, ny, nz)
    steps: int
    omega: float

    @property
    def cells(self) -> int:
        return self.dims[0] * self.dims[1] * self.dims[2]


def d2q33_riemann(nx=256, ny=8, seed=1):
    """D2Q33, FP64, 256 x 8, 200 steps, omega 1.5: x < nx/2 (rho, theta) = (1, 1),
    else (0.5, 0.8); noise 1e-4 on rho."""
    wl = Workload("d2q33_riemann_%dx%d" % (nx, ny), "D2Q33", "fp64", (nx, ny, 1), 200, 1.5)
    return wl, riemann_planar(2, nx, ny, 1, nx // 2, (1.0, 1.0), (0.5, 0.8), seed)


def d3q95_riemann(nx=128, ny=64, nz=64, seed=1, storage="fp32"):
    """D3Q95, FP32, 128 x 64 x 64, 1000 steps, omega 1.6: x < nx/2 (1, 1), else (0.6, 0.75)."""
    wl = Workload("d3q95_riemann_%dx%dx%d" % (nx, ny, nz), "D3Q95", storage, (nx, ny, nz), 1000, 1.6)
    return wl, riemann_planar(3, nx, ny, nz, nx // 2, (1.0, 1.0), (0.6, 0.75), seed)


def d3q95_sweep(nx=512, ny=256, nz=256, seed=1, storage="fp32"):
    """D3Q95 precision sweep, 200 steps, omega 1.8, the D2Q33 workload's states
    (1, 1) | (0.5, 0.8) with the diaphragm at x = nx/2.  The error grid is 128 x 32 x 32."""
    wl = Workload("d3q95_sweep_%dx%dx%d" % (nx, ny, nz), "D3Q95", storage, (nx, ny, nz), 200, 1.8)
    return wl, riemann_planar(3, nx, ny, nz, nx // 2, (1.0, 1.0), (0.5, 0.8), seed)


def d3q95_adjoint(n=128, seed=1, storage="fp32"):
    """D3Q95 adjoint, n^3, 500 steps, omega 1.6, checkpoint every 22:
    rho = 1 + GRF(rms 1e-3, correlation 4), theta = 1.2 in the radius-16 sphere."""
    wl = Workload("d3q95_adjoint_%d^3" % n, "D3Q95", storage, (n, n, n), 500, 1.6)
    return wl, sphere_field(n, n, n, seed, radius=max(1, (16 * n) // 128))


def d3q95_oblique(nx=768, ny=384, nz=384, seed=1, storage="fp16"):
    """D3Q95 oblique Riemann, FP16 deviations, 300 steps, omega 1.7:
    (1, 1) where (i - nx/2) + (j - ny/2) < 0, else (0.6, 0.75)."""
    wl = Workload("d3q95_oblique_%dx%dx%d" % (nx, ny, nz), "D3Q95", storage, (nx, ny, nz), 300, 1.7)
    return wl, riemann_oblique(nx, ny, nz, (1.0, 1.0), (0.6, 0.75), seed)
