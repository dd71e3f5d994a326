"""Closed-form results used to pin the oracle (TEST INFRASTRUCTURE ONLY).

* Sec. 2.1: a Heaviside initial condition diffuses into an erfc profile.  The
  printed formula lacks the square root of 4 D t and its sign convention is
  garbled; the reading used here, for mass 1 on the side x < x0 (left) or
  x >= x0 (right) of an infinite domain, is
      C(x, t) = 1/2 erfc((x - x0) / sqrt(4 D t))     (left)
      C(x, t) = 1/2 erfc((x0 - x) / sqrt(4 D t))     (right)
  with D the total diffusion coefficient (random walk plus mass transfer).
* Sec. 3: concentration from masses, C = N M / L^d.
* A Gaussian point source of variance s0^2 per axis keeps its shape with
  variance s0^2 + 2 D t per axis.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc


def erf_profile(x, t: float, D: float, x0: float, side: str = "left"):
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(4.0 * D * t)
    if side == "left":
        return 0.5 * erfc((x - x0) / s)
    return 0.5 * erfc((x0 - x) / s)


def concentration(mass, n_particles: int, L: float, dim: int):
    """C = N M / L^d (Sec. 3, last equation)."""
    return n_particles * np.asarray(mass, dtype=np.float64) / (L ** dim)


def binned_profile(x, mass, lo: float, hi: float, nbins: int):
    """Mean particle mass in equal slabs of x (the per-particle concentration
    at unit density); returns (bin centres, mean mass, counts)."""
    x = np.asarray(x)
    edges = np.linspace(lo, hi, nbins + 1)
    idx = np.clip(np.searchsorted(edges, x, side="right") - 1, 0, nbins - 1)
    sums = np.bincount(idx, weights=mass, minlength=nbins)
    counts = np.bincount(idx, minlength=nbins)
    centres = 0.5 * (edges[:-1] + edges[1:])
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(counts > 0, sums / np.maximum(counts, 1), np.nan)
    return centres, mean, counts


def rmse(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ok = np.isfinite(a) & np.isfinite(b)
    return float(np.sqrt(np.mean((a[ok] - b[ok]) ** 2)))


def point_source_variance(s0: float, D: float, t: float) -> float:
    return s0 * s0 + 2.0 * D * t
