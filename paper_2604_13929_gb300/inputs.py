"""Seeded synthetic inputs: spinodal pore masks and simple test geometries.

This module holds no Monte Carlo arithmetic.  It only makes the binary masks
that both the CUDA library and the CPU oracle consume.

Spinodal masks follow the Cahn-Hilliard route of Sec. 2.2 of arXiv 2604.13929
in the form the benchmark configurations fix:

* order parameter c in [-1, 1], c_t = lap(c^3 - c - lap c), periodic, dx = 1;
* semi-implicit Fourier spectral step (Eq. CH_spectral with kappa = 1):
  c_hat <- (c_hat - dt k^2 FT(c^3 - c)) / (1 + dt k^4), k = 2 pi fftfreq;
* dt = 0.1, a fixed number of steps, start from seeded uniform noise +-0.05
  (numpy default_rng(seed).uniform, float64);
* rank-based binarisation (App. A): the round(phi * N) voxels with the
  highest c become pore (1), ties broken by the lower linear index, so the
  porosity is exact.

Masks are uint8 arrays of shape (nz, ny, nx), x fastest, 1 = pore.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def initial_noise(shape, seed: int, amplitude: float = 0.05) -> np.ndarray:
    """Seeded uniform noise in [-amplitude, amplitude), float64."""
    return np.random.default_rng(seed).uniform(-amplitude, amplitude, size=tuple(shape))


def cahn_hilliard(shape, steps: int, seed: int = 0, dt: float = 0.1,
                  device: str | torch.device = "cpu", dtype=torch.float64,
                  seeds=None) -> torch.Tensor:
    """Integrate c_t = lap(c^3 - c - lap c) from seeded noise; returns c.

    ``seeds`` (a list) integrates several same-shape fields at once, one per
    seed, stacked along a leading axis."""
    nz, ny, nx = shape
    dev = torch.device(device)
    many = seeds is not None
    noise = np.stack([initial_noise(shape, sd) for sd in (seeds if many else [seed])])
    c = torch.from_numpy(noise).to(device=dev, dtype=dtype)
    kz = 2 * math.pi * torch.fft.fftfreq(nz, d=1.0, dtype=dtype, device=dev)
    ky = 2 * math.pi * torch.fft.fftfreq(ny, d=1.0, dtype=dtype, device=dev)
    kx = 2 * math.pi * torch.fft.rfftfreq(nx, d=1.0, dtype=dtype, device=dev)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    num = dt * k2
    den = 1.0 + dt * k2 * k2
    dims = (-3, -2, -1)
    c_hat = torch.fft.rfftn(c, dim=dims)
    for _ in range(int(steps)):
        nl = torch.fft.rfftn(c * c * c - c, dim=dims)
        c_hat = (c_hat - num * nl) / den
        c = torch.fft.irfftn(c_hat, s=(nz, ny, nx), dim=dims)
    return c if many else c[0]


def rank_threshold(c, porosity: float) -> np.ndarray:
    """The round(porosity*N) highest voxels of c become pore (1); stable ties."""
    t = c if isinstance(c, torch.Tensor) else torch.from_numpy(np.asarray(c))
    flat = t.reshape(-1)
    n = flat.numel()
    n_pore = int(round(porosity * n))
    order = torch.sort(-flat, stable=True).indices
    m = torch.zeros(n, dtype=torch.uint8, device=flat.device)
    m[order[:n_pore]] = 1
    return m.reshape(t.shape).cpu().numpy()


def spinodal_mask(n: int | tuple, porosity: float, steps: int, seed: int = 0,
                  device: str | torch.device = "cpu") -> np.ndarray:
    """Cahn-Hilliard spinodal mask of shape n^3 (or (nz, ny, nx))."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    return rank_threshold(cahn_hilliard(shape, steps, seed=seed, device=device), porosity)


def batch_workload(n_masks: int = 64, seed: int = 3, ch_steps: int = 1000,
                   sizes=(64, 96, 128, 160, 192, 224, 256), device: str | None = None):
    """Masks of uneven size and random optics for batched launches.

    Sizes are drawn from ``sizes`` (cubes), porosity from U[0.50, 0.95], solid
    mu_s h log-uniform on [0.1, 2.0], mu_a h uniform on [0.001, 0.05], g
    uniform on [0, 0.9] (numpy default_rng(seed)).  Each mask is a
    Cahn-Hilliard field of ``ch_steps`` steps in FP32 from noise seed
    1000 + i, rank-thresholded to its porosity.  Returns a list of
    (mask, mu_s h, mu_a h, g)."""
    rng = np.random.default_rng(seed)
    size = rng.choice(np.asarray(sizes), n_masks)
    phi = rng.uniform(0.50, 0.95, n_masks)
    mus = np.exp(rng.uniform(np.log(0.1), np.log(2.0), n_masks))
    mua = rng.uniform(0.001, 0.05, n_masks)
    g = rng.uniform(0.0, 0.9, n_masks)
    dev = device or default_device()
    masks = [None] * n_masks
    for n in np.unique(size):
        idx = [i for i in range(n_masks) if size[i] == n]
        c = cahn_hilliard((int(n),) * 3, ch_steps, device=dev, dtype=torch.float32,
                          seeds=[1000 + i for i in idx])
        for j, i in enumerate(idx):
            masks[i] = rank_threshold(c[j], float(phi[i]))
    return [(masks[i], float(mus[i]), float(mua[i]), float(g[i])) for i in range(n_masks)]


def default_device() -> str:
    return "cuda" if torch.cuda.is_available() else "cpu"


# ---------------------------------------------------------- simple masks --

def all_pore(nz: int, ny: int, nx: int) -> np.ndarray:
    return np.ones((nz, ny, nx), dtype=np.uint8)


def all_solid(nz: int, ny: int, nx: int) -> np.ndarray:
    return np.zeros((nz, ny, nx), dtype=np.uint8)


def layered(pattern, ny: int, nx: int) -> np.ndarray:
    """Laterally uniform layers: pattern[z] = 1 for a pore layer, 0 solid."""
    p = np.asarray(pattern, dtype=np.uint8)
    return np.ascontiguousarray(np.broadcast_to(p[:, None, None], (p.size, ny, nx)))


def random_mask(shape, porosity: float, seed: int) -> np.ndarray:
    """Uncorrelated Bernoulli mask (tie-free traversal tests, not physics)."""
    return (np.random.default_rng(seed).random(tuple(shape)) < porosity).astype(np.uint8)


def radial_psd_peak(mask: np.ndarray) -> float:
    """Dominant structural length (voxels) from the radial power spectrum peak."""
    m = mask.astype(np.float64)
    m = m - m.mean()
    p = np.abs(np.fft.fftn(m)) ** 2
    nz, ny, nx = m.shape
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.fftfreq(nx)[None, None, :]
    k = np.sqrt(kz ** 2 + ky ** 2 + kx ** 2)
    nb = min(nz, ny, nx) // 2
    idx = np.minimum((k * min(nz, ny, nx)).astype(np.int64), nb)
    prof = np.bincount(idx.ravel(), weights=p.ravel(), minlength=nb + 1)
    cnt = np.bincount(idx.ravel(), minlength=nb + 1)
    prof = prof / np.maximum(cnt, 1)
    kb = int(np.argmax(prof[1:nb]) + 1)
    return min(nz, ny, nx) / kb
