"""Seeded synthetic fields shaped like the paper's workloads.

This module holds input generators only -- no step of the compression
method.  Both the CUDA path and the oracle are fed from it.

The paper's datasets (Nyx, WarpX, Magnetic Reconnection, Miranda; Table 4)
are not available, so these fields stand in for them with the same shapes
and dtypes:

* ``sinusoids`` -- a sum of random 3D (or 2D) sinusoids with small Gaussian
  noise (the 128^3 smoke / parity workload);
* ``grf`` -- a Gaussian random field with power spectrum ``k**slope``
  synthesised by FFT filtering of white noise, optionally exponentiated to a
  positive, log-normal density-like field (stand-in for Nyx baryon density:
  slope -3, sigma 1.5) or left Gaussian (turbulence-like, slope -5/3);
* ``banded2d`` -- smooth 2D sinusoid sums with latitude-like bands.

Every generator takes an integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2509016


def seed_for(config: int, index: int = 0) -> int:
    """Seed of field `index` of workload `config`."""
    return BASE_SEED + 100 * config + index


def _axes(shape):
    return [np.arange(n, dtype=np.float64) / n for n in shape]


def sinusoids(shape, seed: int, n_terms: int = 16, fmin: float = 1.0, fmax: float = 8.0,
              noise: float = 1e-3, dtype=np.float32) -> np.ndarray:
    """sum_j A_j sin(2 pi f_j . r + phi_j) + N(0, noise^2); r in [0,1)^d,
    f_j uniform in [fmin, fmax] cycles per domain per axis, A_j ~ N(0,1),
    phi_j ~ U[0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = len(shape)
    out = np.zeros(shape, dtype=np.float64)
    ax = _axes(shape)
    for _ in range(n_terms):
        f = rng.uniform(fmin, fmax, size=d)
        amp = rng.normal()
        phi = rng.uniform(0.0, 2.0 * np.pi)
        # exp(i(a + b + c)) as an outer product of 1D factors
        term = np.exp(1j * (2.0 * np.pi * f[0] * ax[0] + phi))
        for a in range(1, d):
            term = np.multiply.outer(term, np.exp(2j * np.pi * f[a] * ax[a]))
        out += amp * term.imag
    if noise > 0:
        out += rng.normal(0.0, noise, size=shape)
    return out.astype(dtype)


def grf(shape, seed: int, slope: float = -3.0, lognormal_sigma: float | None = 1.5,
        dtype=np.float32, device: str = "cpu", white_source: str = "numpy",
        as_tensor: bool = False):
    """Gaussian random field with P(k) ~ k**slope (k = 0 removed), unit
    standard deviation; with lognormal_sigma set, returns exp(sigma * g).
    White noise from PCG64 (white_source "numpy") or from a torch generator
    on `device` seeded with `seed` ("torch", for fields too large to draw on
    the host); the FFT filter runs in float64 with torch on `device` (numpy
    when torch is absent).  as_tensor: return the torch tensor on `device`."""
    try:
        import torch

        if white_source == "torch":
            gen = torch.Generator(device=device).manual_seed(int(seed))
            t = torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
        else:
            rng = np.random.Generator(np.random.PCG64(seed))
            t = torch.from_numpy(rng.standard_normal(size=shape)).to(device)
        spec = torch.fft.rfftn(t)
        del t
        ks = []
        for a, n in enumerate(shape):
            if a == len(shape) - 1:
                k = torch.fft.rfftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
            else:
                k = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
            view = [1] * len(shape)
            view[a] = -1
            ks.append(k.view(view))
        k2 = ks[0] ** 2
        for k in ks[1:]:
            k2 = k2 + k ** 2
        amp = torch.where(k2 > 0, k2.clamp_min(1e-300) ** (slope / 4.0), torch.zeros_like(k2))
        del k2
        spec *= amp
        del amp
        g = torch.fft.irfftn(spec, s=shape)
        del spec
        g = (g - g.mean()) / g.std()
        if lognormal_sigma is not None:
            g = torch.exp(lognormal_sigma * g)
        g = g.to(torch.float64 if dtype == np.float64 else torch.float32)
        return g if as_tensor else g.cpu().numpy()
    except ImportError:
        rng = np.random.Generator(np.random.PCG64(seed))
        white = rng.standard_normal(size=shape)
        spec = np.fft.rfftn(white)
        ks = []
        for a, n in enumerate(shape):
            k = np.fft.rfftfreq(n, d=1.0 / n) if a == len(shape) - 1 else np.fft.fftfreq(n, d=1.0 / n)
            view = [1] * len(shape)
            view[a] = -1
            ks.append(k.reshape(view))
        k2 = sum(k ** 2 for k in ks)
        with np.errstate(divide="ignore"):
            amp = np.where(k2 > 0, k2 ** (slope / 4.0), 0.0)
        g = np.fft.irfftn(spec * amp, s=shape)
        g = (g - g.mean()) / g.std()
        if lognormal_sigma is not None:
            g = np.exp(lognormal_sigma * g)
        return g.astype(dtype)


def banded2d(shape, seed: int, n_terms: int = 8, dtype=np.float32) -> np.ndarray:
    """sum_j A_j sin(2 pi f_j . (y, x) + phi_j) + B cos(pi lat m), lat = y/ny."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ny, nx = shape
    y = np.arange(ny, dtype=np.float64)[:, None] / ny
    x = np.arange(nx, dtype=np.float64)[None, :] / nx
    out = np.zeros(shape, dtype=np.float64)
    for _ in range(n_terms):
        fy, fx = rng.uniform(1.0, 8.0, size=2)
        out += rng.normal() * np.sin(2 * np.pi * (fy * y + fx * x) + rng.uniform(0, 2 * np.pi))
    m = int(rng.integers(2, 9))
    out += rng.normal() * np.cos(np.pi * y * m) * np.ones_like(x)
    return out.astype(dtype)


def random_boxes(shape, n: int, seed: int, emin: int, emax: int):
    """n boxes [lo, hi) with per-axis edge uniform in [emin, emax] (clipped to
    the field) and origin uniform inside."""
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes = []
    for _ in range(n):
        lo, hi = [], []
        for d in shape:
            e = int(min(d, rng.integers(emin, emax + 1)))
            o = int(rng.integers(0, d - e + 1))
            lo.append(o)
            hi.append(o + e)
        boxes.append((tuple(lo), tuple(hi)))
    return boxes


def sinusoids_device(shape, seed: int, n_terms: int = 16, fmin: float = 1.0, fmax: float = 8.0,
                     noise: float = 1e-3, dtype=np.float32, device: str = "cuda"):
    """The recipe of ``sinusoids`` evaluated with torch on `device` (for
    large fields): the terms' frequencies, amplitudes and phases are drawn
    from PCG64 in the same order; the noise comes from a torch generator on
    `device` seeded with `seed`.  Returns a torch tensor."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    d = len(shape)
    ax = [torch.arange(n, dtype=torch.float64, device=device) / n for n in shape]
    out = torch.zeros(shape, dtype=torch.float64, device=device)
    for _ in range(n_terms):
        f = rng.uniform(fmin, fmax, size=d)
        amp = rng.normal()
        phi = rng.uniform(0.0, 2.0 * np.pi)
        ph = None
        for a in range(d):
            view = [1] * d
            view[a] = -1
            v = (2.0 * np.pi * float(f[a]) * ax[a]).view(view)
            ph = v if ph is None else ph + v
        out += float(amp) * torch.sin(ph + float(phi))
    if noise > 0:
        gen = torch.Generator(device=device).manual_seed(int(seed))
        out += noise * torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
    return out.to(torch.float64 if dtype == np.float64 else torch.float32)


def banded2d_device(shape, seed: int, n_terms: int = 8, dtype=np.float32, device: str = "cuda"):
    """The recipe of ``banded2d`` evaluated with torch on `device`."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    ny, nx = shape
    y = (torch.arange(ny, dtype=torch.float64, device=device) / ny)[:, None]
    x = (torch.arange(nx, dtype=torch.float64, device=device) / nx)[None, :]
    out = torch.zeros(shape, dtype=torch.float64, device=device)
    for _ in range(n_terms):
        fy, fx = rng.uniform(1.0, 8.0, size=2)
        amp = rng.normal()
        phi = rng.uniform(0, 2 * np.pi)
        out += float(amp) * torch.sin(2 * np.pi * (float(fy) * y + float(fx) * x) + float(phi))
    m = int(rng.integers(2, 9))
    out += float(rng.normal()) * torch.cos(np.pi * y * m) * torch.ones_like(x)
    return out.to(torch.float64 if dtype == np.float64 else torch.float32)


def batch_workload(seed_index: int = 0):
    """The mixed batch: 40 3D float32 fields with each dim uniform in
    [64, 512] (8-term sinusoid sums with 1e-3 noise), 16 2D float32 fields
    1800 x 3600 (sinusoids with latitude bands), 8 3D float64 fields 256^3
    (smooth 4-term sums); per-field relative bound from {1e-2, 1e-3, 1e-4}.
    Returns a list of (kind, shape, dtype, seed, eb)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(3, 1000 + seed_index)))
    items = []
    for i in range(40):
        shape = tuple(int(v) for v in rng.integers(64, 513, size=3))
        items.append(("sin3d", shape, np.float32, seed_for(3, i)))
    for i in range(16):
        items.append(("band2d", (1800, 3600), np.float32, seed_for(3, 40 + i)))
    for i in range(8):
        items.append(("smooth3d", (256, 256, 256), np.float64, seed_for(3, 56 + i)))
    ebs = rng.choice(np.array([1e-2, 1e-3, 1e-4]), size=len(items))
    return [it + (float(eb),) for it, eb in zip(items, ebs)]


def make_batch_field(item, device: str = "cuda"):
    kind, shape, dtype, seed, _ = item
    if kind == "sin3d":
        return sinusoids_device(shape, seed, n_terms=8, noise=1e-3, dtype=dtype, device=device)
    if kind == "band2d":
        return banded2d_device(shape, seed, dtype=dtype, device=device)
    return sinusoids_device(shape, seed, n_terms=4, fmin=1.0, fmax=3.0, noise=0.0, dtype=dtype,
                            device=device)
