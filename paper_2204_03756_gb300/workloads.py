"""Seeded synthetic inputs (initial particle states) for the MTPT step.

This module holds no part of the method's arithmetic: it only draws initial
positions and assigns initial masses, the inputs that the CUDA path and the
CPU oracle both consume.  Positions are uniform in the box (Sec. 2.1: "randomly
scattered"), drawn with numpy's Philox bit generator under the workload seed;
masses follow the initial conditions of each workload.

Workloads (sizes and parameters of the paper's test problem family, Sec. 2):

* ``heaviside_2d``   N = 10,000 in [0,100]^2, mass 1 where x < 50 else 0,
  D = 1, kappa = 0.5, dt = 0.1, 100 steps.
* ``gaussian_2d``    N = 4,000,000 in [0,2000]^2 (density 1), mass
  exp(-|x - c|^2 / (2 * 5^2)) with c the box centre, D = 1, dt = 0.1,
  1,000 steps.
* ``heaviside_3d``   N = 2,000,000 in [0,126]^3 (density ~1), mass 1 where
  x < 63 else 0, D = 1, dt = 0.05, 500 steps.
* ``uniform_mass_2d`` N = 250,000 in [0,500]^2, mass U(0,1), D = 0.5,
  dt = 0.1, 200 steps.
* ``advection_2d``   N = 4,000,000 in [0,2000]^2 (density 1), mass 1 where
  x < 500 else 0, D = 1, kappa = 0.5, dt = 0.1, uniform velocity
  v = (0.1, 0.05) (the advection term of the model equation, Sec. 2), 1,000
  steps.  The velocity is small so that over the run the particles carried
  into the downstream walls (where zero-flux reflection piles them up in a
  thin dense layer) stay a small fraction of the whole.
* ``reaction_2d``    N = 4,000,000 in [0,2000]^2 (density 1), species A 1
  where x < 1000, species B its complement, D = 1, kappa = 0.5, dt = 0.1,
  A + B -> 0 with rate constant k = 1 (the reaction extension of Sec. 8),
  1,000 steps: the two species meet along the line x = 1000.

Every workload takes kappa = 0.5, beta = 1 and lambda = 3 (cutoff
psi = 3 sqrt(4 D_MT dt)), and may be scaled down (``n`` with the box scaled
to keep the density) for tests.

``ensemble_2d`` (see :func:`ensemble`) is a batch of independent 2-d
realisations: counts log-uniform in [5,000, 200,000], densities uniform in
[0.5, 2] (square box of side sqrt(N_k / rho_k)), D uniform in [0.1, 2],
dt = 0.1, 200 steps, Heaviside mass (1 where x < L_k / 2), one seed each.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

SEED_BASE = 2204037560


@dataclass
class Workload:
    name: str
    dim: int
    n: int
    lo: tuple
    hi: tuple
    D: float
    kappa: float
    dt: float
    steps: int
    mass_kind: str           # "heaviside_left", "gaussian_centre", "uniform01", "ones"
    beta: float = 1.0
    lam: float = 3.0
    seed: int = SEED_BASE
    mass_param: float = 0.0  # Heaviside split x, or Gaussian sigma
    v: tuple = (0.0, 0.0, 0.0)  # uniform velocity (advection)
    react_k: float = 0.0     # rate constant of A + B -> 0 (0: no second species)

    def scaled(self, n: int) -> "Workload":
        """Same density and parameters with ``n`` particles: every box edge
        is scaled by (n / N)^(1/d) about the lower corner."""
        f = (n / self.n) ** (1.0 / self.dim)
        lo = tuple(self.lo[a] for a in range(self.dim))
        hi = tuple(self.lo[a] + (self.hi[a] - self.lo[a]) * f for a in range(self.dim))
        mp = self.mass_param * f if self.mass_kind == "heaviside_left" else self.mass_param
        return replace(self, n=n, lo=lo, hi=hi, mass_param=mp)


WORKLOADS = {
    "heaviside_2d": Workload("heaviside_2d", 2, 10_000, (0.0, 0.0), (100.0, 100.0),
                             1.0, 0.5, 0.1, 100, "heaviside_left", seed=SEED_BASE + 1,
                             mass_param=50.0),
    "gaussian_2d": Workload("gaussian_2d", 2, 4_000_000, (0.0, 0.0), (2000.0, 2000.0),
                            1.0, 0.5, 0.1, 1000, "gaussian_centre", seed=SEED_BASE + 2,
                            mass_param=5.0),
    "heaviside_3d": Workload("heaviside_3d", 3, 2_000_000, (0.0, 0.0, 0.0),
                             (126.0, 126.0, 126.0), 1.0, 0.5, 0.05, 500, "heaviside_left",
                             seed=SEED_BASE + 3, mass_param=63.0),
    "uniform_mass_2d": Workload("uniform_mass_2d", 2, 250_000, (0.0, 0.0), (500.0, 500.0),
                                0.5, 0.5, 0.1, 200, "uniform01", seed=SEED_BASE + 5),
    "advection_2d": Workload("advection_2d", 2, 4_000_000, (0.0, 0.0), (2000.0, 2000.0),
                             1.0, 0.5, 0.1, 1000, "heaviside_left", seed=SEED_BASE + 7,
                             mass_param=500.0, v=(0.1, 0.05, 0.0)),
    "reaction_2d": Workload("reaction_2d", 2, 4_000_000, (0.0, 0.0), (2000.0, 2000.0),
                            1.0, 0.5, 0.1, 1000, "heaviside_left", seed=SEED_BASE + 8,
                            mass_param=1000.0, react_k=1.0),
}


def positions(w: Workload) -> np.ndarray:
    """Uniform positions in the box, shape (dim, n), float64."""
    rng = np.random.Generator(np.random.Philox(w.seed))
    pos = np.empty((w.dim, w.n), dtype=np.float64)
    for a in range(w.dim):
        pos[a] = rng.uniform(w.lo[a], w.hi[a], size=w.n)
    return pos


def masses(w: Workload, pos: np.ndarray) -> np.ndarray:
    """Initial masses of the workload's initial condition, float64."""
    if w.mass_kind == "heaviside_left":
        return (pos[0] < w.mass_param).astype(np.float64)
    if w.mass_kind == "gaussian_centre":
        c = [0.5 * (w.lo[a] + w.hi[a]) for a in range(w.dim)]
        r2 = sum((pos[a] - c[a]) ** 2 for a in range(w.dim))
        return np.exp(-r2 / (2.0 * w.mass_param ** 2))
    if w.mass_kind == "uniform01":
        rng = np.random.Generator(np.random.Philox(w.seed + 1_000_003))
        return rng.uniform(0.0, 1.0, size=pos.shape[1])
    if w.mass_kind == "ones":
        return np.ones(pos.shape[1], dtype=np.float64)
    raise ValueError(f"unknown mass kind {w.mass_kind!r}")


def masses_b(w: Workload, pos: np.ndarray) -> np.ndarray:
    """Species B of a reaction workload: the complement of A's Heaviside
    initial condition (A on the left of the split, B on the right)."""
    return 1.0 - masses(w, pos)


def initial_state(w: Workload):
    pos = positions(w)
    return pos, masses(w, pos)


def get(name: str, n: int | None = None) -> Workload:
    w = WORKLOADS[name]
    return w if n is None or n == w.n else w.scaled(n)


@dataclass
class Ensemble:
    """A batch of independent realisations: per-realisation workloads and
    their concatenated initial state."""
    name: str
    members: list
    steps: int

    @property
    def counts(self):
        return np.array([w.n for w in self.members], dtype=np.int64)


def ensemble(nreal: int = 512, n_min: int = 5_000, n_max: int = 200_000,
             seed: int = SEED_BASE + 4, steps: int = 200) -> Ensemble:
    """The ensemble workload: ``nreal`` 2-d realisations with log-uniform
    particle counts, uniform densities in [0.5, 2] and D uniform in [0.1, 2]."""
    rng = np.random.Generator(np.random.Philox(seed))
    logn = rng.uniform(np.log(n_min), np.log(n_max), size=nreal)
    counts = np.round(np.exp(logn)).astype(np.int64)
    rho = rng.uniform(0.5, 2.0, size=nreal)
    D = rng.uniform(0.1, 2.0, size=nreal)
    members = []
    for k in range(nreal):
        L = float(np.sqrt(counts[k] / rho[k]))
        members.append(Workload(f"ensemble_2d[{k}]", 2, int(counts[k]), (0.0, 0.0), (L, L),
                                float(D[k]), 0.5, 0.1, steps, "heaviside_left",
                                seed=seed + 1 + k, mass_param=0.5 * L))
    return Ensemble("ensemble_2d", members, steps)


def ensemble_state(e: Ensemble):
    """Concatenated initial positions (dim x total) and masses."""
    parts = [initial_state(w) for w in e.members]
    pos = np.concatenate([p for p, _ in parts], axis=1)
    mass = np.concatenate([m for _, m in parts])
    return pos, mass


def target_field(nbins, lo, hi, seed: int = SEED_BASE + 6) -> np.ndarray:
    """Seeded smooth target concentration on an nbins[0] x nbins[1] grid of
    bin centres over the box: 0.5 + 0.25 sin(2 pi (x/Lx + a)) cos(2 pi (y/Ly + b))
    with phases a, b drawn from the seed (the misfit target of the
    differentiable workload)."""
    rng = np.random.Generator(np.random.Philox(seed))
    a, b = rng.uniform(0.0, 1.0, size=2)
    Lx, Ly = hi[0] - lo[0], hi[1] - lo[1]
    xc = lo[0] + (np.arange(nbins[0]) + 0.5) * Lx / nbins[0]
    yc = lo[1] + (np.arange(nbins[1]) + 0.5) * Ly / nbins[1]
    X, Y = np.meshgrid(xc, yc, indexing="ij")
    return 0.5 + 0.25 * np.sin(2 * np.pi * (X / Lx + a)) * np.cos(2 * np.pi * (Y / Ly + b))
