"""Seeded synthetic input fields for the z_re(x) path.

This module is the one piece shared by the GPU path's tests/bench and the
oracle's tests: it makes INPUTS only and holds none of the method's
arithmetic (no radiation kernel, no ranking, no abundance matching).

Recipe (stand-in for the paper's 2LPT + excursion-set source fields, Sec. 3.2
and 3.3; no dataset is used):

* white noise w(x) ~ N(0,1) from a counter-based generator: SplitMix64 of
  (seed * 2^40 + cell index) gives two 53-bit uniforms per cell, then
  Box-Muller (float64).  Integer steps are exact, so the same seed gives the
  same noise on any device;
* Gaussian density delta: w shaped in Fourier space by sqrt(P(k)) with
  P(k) = k^-2.5 exp(-(k/k_c)^2), k_c = 0.5 k_Nyquist, P(0) = 0, then rescaled
  to mean 0 and population standard deviation sigma (default 1.5);
* source S = (1 + max(delta, -0.99)) * erfc((1.686 - delta)/(sqrt(2) * 0.7)),
  divided by its mean (an excursion-set collapsed-fraction analogue, Sec. 3.3);
* cell mass = 1 + max(delta, -0.99).
* realisation r uses seed 1000 + r.

torch is used for the noise and the Fourier shaping so that 1024^3 inputs can
be made on the device in seconds; this is input preparation, not the path.
"""
from __future__ import annotations

import math

import torch

_MASK64 = (1 << 64) - 1


def _s64(v: int) -> int:
    """Python int in [0, 2^64) -> the int64 with the same bits."""
    v &= _MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_M1 = _s64(0xBF58476D1CE4E5B9)
_M2 = _s64(0x94D049BB133111EB)


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bits."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64(counter: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output for each int64 counter (wrapping arithmetic)."""
    z = counter + _GOLDEN
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def white_noise(n: int, seed: int, device="cpu") -> torch.Tensor:
    """N(0,1) float64 noise on an n^3 grid, cell order [z][y][x]."""
    cells = n * n * n
    out = torch.empty(cells, dtype=torch.float64, device=device)
    chunk = 1 << 26
    base = (seed << 40)
    two_pi = 2.0 * math.pi
    for s in range(0, cells, chunk):
        e = min(cells, s + chunk)
        idx = torch.arange(s, e, dtype=torch.int64, device=device)
        c = (base + idx) * 2
        u1 = (_srl(splitmix64(c), 11).to(torch.float64) + 1.0) * (2.0 ** -53)   # (0, 1]
        u2 = _srl(splitmix64(c + 1), 11).to(torch.float64) * (2.0 ** -53)       # [0, 1)
        out[s:e] = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(two_pi * u2)
    return out.view(n, n, n)


def gaussian_density(n: int, box: float, seed: int, sigma: float = 1.5, slope: float = -2.5,
                     device="cpu") -> torch.Tensor:
    """delta with power spectrum k^slope exp(-(k/k_c)^2), k_c = k_Ny/2 (float64)."""
    w = white_noise(n, seed, device)
    wk = torch.fft.rfftn(w)
    del w
    kf = 2.0 * math.pi / box
    ky = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64, device=device) * kf
    kx = torch.arange(n // 2 + 1, dtype=torch.float64, device=device) * kf
    k_ny = math.pi * n / box
    kc = 0.5 * k_ny
    for iz in range(n):  # plane by plane to bound temporaries at large n
        k2 = ky[iz] ** 2 + ky[:, None] ** 2 + kx[None, :] ** 2
        k = torch.sqrt(k2)
        p = torch.where(k > 0, k.clamp_min(1e-300) ** slope * torch.exp(-(k / kc) ** 2),
                        torch.zeros_like(k))
        wk[iz] *= torch.sqrt(p)
    d = torch.fft.irfftn(wk, s=(n, n, n))
    del wk
    d -= d.mean()
    d *= sigma / torch.sqrt((d * d).mean())
    return d


def source_and_mass(delta: torch.Tensor, delta_c: float = 1.686, sigma_f: float = 0.7):
    """(S, mass) as float32 from delta (recipe in the module docstring)."""
    dm = torch.clamp(delta, min=-0.99)
    mass = 1.0 + dm
    S = mass * torch.special.erfc((delta_c - delta) / (math.sqrt(2.0) * sigma_f))
    S /= S.mean()
    return S.to(torch.float32), mass.to(torch.float32)


def realisation(n: int, box: float, r: int = 0, sigma: float = 1.5, device="cpu"):
    """(S, mass) float32 [n,n,n] for realisation r (seed 1000 + r)."""
    d = gaussian_density(n, box, 1000 + r, sigma=sigma, device=device)
    S, m = source_and_mass(d)
    del d
    return S, m
