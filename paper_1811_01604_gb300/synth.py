"""Seeded synthetic inputs: Whittle-Matern Gaussian fields and sampling masks.

This module holds none of the method's arithmetic; it only makes the grids
that both the CUDA library and the FP64 oracle are fed (Sect. 4 of the paper:
Gaussian random fields with Whittle-Matern covariance, Eq. 7, simulated by the
spectral method, with p% of the sites removed at random).

Readings of what the paper leaves open:
  * kappa is the inverse correlation length (xi = 1/kappa);
  * the spectral method uses the exact lattice spectrum of Eq. 7 (the FFT of the
    covariance on a larger periodic grid), so the field has the Eq. 7
    covariance at lattice lags, with variance sigma^2;
  * the lognormal variant is y = m exp(0.5 g - 0.125) with g = (z - m)/sigma.
"""
from __future__ import annotations

import numpy as np


def wm_field(L: int, nu: float, xi: float, seed: int, m: float = 50.0, sigma: float = 10.0,
             W: int | None = None) -> np.ndarray:
    """Whittle-Matern Gaussian field of H=L rows and W (default L) columns, float32.

    Spectral method with the exact lattice spectrum (circulant embedding): Eq. 7
    is evaluated at the minimum-image lags of a periodic grid that is larger than
    the output by at least 16 correlation lengths, its 2-D FFT gives the spectrum
    (negative round-off eigenvalues are set to 0), and white noise filtered by the
    square root of that spectrum has the Eq. 7 covariance at every lattice lag
    shorter than half the periodic grid.  The first H x W block is returned.
    """
    from scipy import fft as sfft
    H = int(L)
    W = int(W or L)
    pad = int(max(32, 16 * xi))
    ny = sfft.next_fast_len(H + pad)
    nx = sfft.next_fast_len(W + pad)
    dy = np.minimum(np.arange(ny), ny - np.arange(ny)).astype(np.float64)
    dx = np.minimum(np.arange(nx), nx - np.arange(nx)).astype(np.float64)
    h = np.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2)
    C = wm_covariance(h, nu, xi, 1.0)
    lam = np.maximum(sfft.rfft2(C).real, 0.0)
    del C, h
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((ny, nx))
    g = sfft.irfft2(np.sqrt(lam) * sfft.rfft2(w), s=(ny, nx))
    z = m + sigma * g[:H, :W]
    return z.astype(np.float32)


def wm_field_gpu(H: int, W: int, nu: float, xi: float, seed: int, m: float = 50.0,
                 sigma: float = 10.0, device="cuda"):
    """Same spectral method as wm_field, computed with torch on a GPU (for large batches of
    inputs).  Eq. 7 in closed form for nu in {0.5, 1, 1.5, 2.5} (K_1 for nu = 1).  The white
    noise comes from torch's generator, so fields differ from wm_field's for one seed."""
    import torch
    pad = int(max(32, 16 * xi))
    ny, nx = H + pad, W + pad
    ny += ny % 2
    nx += nx % 2
    dy = torch.arange(ny, device=device, dtype=torch.float64)
    dx = torch.arange(nx, device=device, dtype=torch.float64)
    dy = torch.minimum(dy, ny - dy)
    dx = torch.minimum(dx, nx - dx)
    kh = torch.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2) / float(xi)
    if nu == 0.5:
        C = torch.exp(-kh)
    elif nu == 1.5:
        C = (1.0 + kh) * torch.exp(-kh)
    elif nu == 2.5:
        C = (1.0 + kh + kh * kh / 3.0) * torch.exp(-kh)
    elif nu == 1.0:
        C = torch.where(kh > 0, kh * torch.special.modified_bessel_k1(torch.clamp(kh, min=1e-300)),
                        torch.ones_like(kh))
    else:
        raise ValueError("nu must be one of 0.5, 1, 1.5, 2.5")
    lam = torch.clamp(torch.fft.rfft2(C).real, min=0.0)
    del C, kh
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    w = torch.randn((ny, nx), generator=gen, device=device, dtype=torch.float64)
    g = torch.fft.irfft2(torch.sqrt(lam) * torch.fft.rfft2(w), s=(ny, nx))
    return (m + sigma * g[:H, :W]).to(torch.float32).contiguous()


def batch_workload(n: int = 256, L_min: int = 128, L_max: int = 2048, seed: int = 4):
    """Parameters of the batched workload: per grid g (seed + g) a side L log-uniform in
    [L_min, L_max], nu in {0.5, 1, 2.5}, correlation length uniform in [4, 64], missing
    fraction uniform in [0.2, 0.7]."""
    out = []
    for g in range(n):
        rng = np.random.Generator(np.random.PCG64(seed + g))
        L = int(round(float(np.exp(rng.uniform(np.log(L_min), np.log(L_max))))))
        nu = float(rng.choice([0.5, 1.0, 2.5]))
        xi = float(rng.uniform(4.0, 64.0))
        p = float(rng.uniform(0.2, 0.7))
        out.append(dict(L=L, nu=nu, xi=xi, p=p, seed=seed + g))
    return out


def mask_uniform_gpu(H: int, W: int, p: float, seed: int, device="cuda"):
    """uint8 [H][W] with exactly round(p*H*W) gaps (0) placed uniformly, via torch."""
    import torch
    n = H * W
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    perm = torch.randperm(n, generator=gen, device=device)
    m = torch.ones(n, dtype=torch.uint8, device=device)
    m[perm[: int(round(p * n))]] = 0
    return m.view(H, W)


def wm_covariance(h, nu: float, xi: float, sigma: float = 10.0):
    """Eq. 7, the Whittle-Matern covariance at distance h (for generator checks)."""
    from scipy.special import gamma, kv
    h = np.asarray(h, np.float64)
    kh = h / float(xi)
    out = np.empty_like(kh)
    zero = kh == 0
    out[zero] = sigma * sigma
    khn = kh[~zero]
    out[~zero] = sigma * sigma * 2.0 ** (1.0 - nu) / gamma(nu) * khn ** nu * kv(nu, khn)
    return out


def lognormal(z: np.ndarray, m: float = 50.0, sigma: float = 10.0) -> np.ndarray:
    g = (z.astype(np.float64) - m) / sigma
    return (m * np.exp(0.5 * g - 0.125)).astype(np.float32)


def mask_uniform(H: int, W: int, p: float, seed: int) -> np.ndarray:
    """uint8 [H][W], 1 = sample, 0 = gap; exactly round(p*H*W) gaps, uniformly placed."""
    n = H * W
    n_gap = int(round(p * n))
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.ones(n, np.uint8)
    m[rng.permutation(n)[:n_gap]] = 0
    return m.reshape(H, W)


def mask_disks(H: int, W: int, p: float, seed: int, disk_frac: float = 0.25,
               r_min: int = 8, r_max: int = 64) -> np.ndarray:
    """Cloud-like gaps: random disks (radius uniform in [r_min, r_max]) until disk_frac of the
    grid is covered, then uniformly random sites until round(p*H*W) gaps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.ones((H, W), np.uint8)
    n = H * W
    target_disk = int(round(disk_frac * n))
    yy = np.arange(H)[:, None]
    xx = np.arange(W)[None, :]
    covered = 0
    while covered < target_disk:
        cy = int(rng.integers(0, H)); cx = int(rng.integers(0, W)); r = int(rng.integers(r_min, r_max + 1))
        y0, y1 = max(0, cy - r), min(H, cy + r + 1)
        x0, x1 = max(0, cx - r), min(W, cx + r + 1)
        sub = (yy[y0:y1] - cy) ** 2 + (xx[:, x0:x1] - cx) ** 2 <= r * r
        m[y0:y1, x0:x1][sub] = 0
        covered = n - int(m.sum())
    n_gap = int(round(p * n))
    rest = n_gap - covered
    if rest > 0:
        idx = np.flatnonzero(m.ravel())
        pick = rng.permutation(idx.size)[:rest]
        m.ravel()[idx[pick]] = 0
    return m


def config(name: str):
    """Named synthetic workloads: returns dict(z, mask, truth, meta)."""
    if name == "grid64":          # 64 x 64, nu 0.5, correlation length 4, 33% uniform gaps
        z = wm_field(64, 0.5, 4.0, seed=0)
        mask = mask_uniform(64, 64, 0.33, seed=1_000_000)
        return dict(z=z, mask=mask, meta=dict(L=64, nu=0.5, xi=4.0, p=0.33, M=10))
    if name == "grid1024":        # 1024 x 1024, nu 0.5, correlation length 16, 33% gaps
        z = wm_field(1024, 0.5, 16.0, seed=1)
        mask = mask_uniform(1024, 1024, 0.33, seed=1_000_001)
        return dict(z=z, mask=mask, meta=dict(L=1024, nu=0.5, xi=16.0, p=0.33, M=100))
    if name == "grid4096":        # 4096 x 4096, nu 1, correlation length 32, 50% disk+random
        z = wm_field(4096, 1.0, 32.0, seed=3)
        mask = mask_disks(4096, 4096, 0.5, seed=1_000_003)
        return dict(z=z, mask=mask, meta=dict(L=4096, nu=1.0, xi=32.0, p=0.5, M=100))
    if name == "paper1024":       # Table 2/3 setting: nu 0.5, kappa 0.2, L 1024
        z = wm_field(1024, 0.5, 5.0, seed=7)
        mask = mask_uniform(1024, 1024, 0.33, seed=1_000_007)
        return dict(z=z, mask=mask, meta=dict(L=1024, nu=0.5, xi=5.0, p=0.33, M=100))
    raise KeyError(name)
