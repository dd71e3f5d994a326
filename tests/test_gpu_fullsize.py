"""Parity at the workloads' full sizes, in the launch configuration bench.py
times: the 4e6-particle 2-d and 2e6-particle 3-d steps against the oracle
element by element (one step each: the oracle's K-D tree takes seconds at this
size), sampled realisations of the full 512-member ensemble (realisations are
independent, so the oracle runs each sampled one on its own), and the
adjoint's full-size gradient checked through properties that hold at any
size: linearity in the masses and a binary64 finite difference in D
(with the pair set and the bins checked unchanged across it); and the 2-d
workload run for its full 1000 steps in one call against 1000 single-step
calls."""
import numpy as np
import pytest

import oracle as O
from paper_2204_03756_gb300 import mtpt, workloads

from gpu_helpers import TOL, oracle_params, params_of, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


@pytest.mark.parametrize("name", ["gaussian_2d", "heaviside_3d"])
@pytest.mark.parametrize("form", [mtpt.MTPT_FP32W, mtpt.MTPT_FP64])
def test_full_size_step_equals_the_oracle(name, form):
    w = workloads.get(name)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(1)
        x, m, info = sim.positions(), sim.masses(), sim.info()
    xr, mr, npairs = O.run(oracle_params(p), pos, mass, 1)
    assert np.array_equal(x, xr)
    assert info["pair_count"] == npairs
    assert rel_err(m, mr) <= TOL[form]


def test_full_ensemble_sampled_realisations_equal_the_oracle():
    e = workloads.ensemble()
    pos, mass = workloads.ensemble_state(e)
    params = [params_of(w, precision=mtpt.MTPT_FP32W) for w in e.members]
    with mtpt.Batch(params, e.counts, pos, mass) as b:
        b.autotune(2)
        b.step(2)
        bm, bx = b.split(b.masses()), b.split(b.positions())
    rng = np.random.default_rng(0)
    for k in sorted(rng.choice(len(e.members), size=4, replace=False)):
        w = e.members[k]
        p0, m0 = workloads.initial_state(w)
        xr, mr, _ = O.run(oracle_params(params[k]), p0, m0, 2)
        assert np.array_equal(bx[k], xr), k
        assert rel_err(bm[k], mr) <= TOL[mtpt.MTPT_FP32W], k


def _misfit_torch(w, x, m, target, nb):
    import torch
    from paper_2204_03756_gb300.autograd import binned_concentration
    C = binned_concentration(x, m, w.lo, w.hi, nb)
    return ((C - target) ** 2).sum()


def test_full_size_adjoint_linearity_and_D_difference():
    import torch
    from paper_2204_03756_gb300.autograd import mtpt_run
    w = workloads.get("uniform_mass_2d")
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=mtpt.MTPT_FP64)
    nb = (100, 100)
    target = torch.from_numpy(workloads.target_field(nb, w.lo, w.hi)).cuda()
    steps = 40
    x0 = torch.from_numpy(pos).cuda()
    m0 = torch.from_numpy(mass).cuda().requires_grad_(True)
    D = torch.tensor(p.D, dtype=torch.float64, requires_grad=True)
    mT, xT = mtpt_run(m0, D, p, x0, steps, checkpoint_every=20)
    loss = _misfit_torch(w, xT, mT, target, nb)
    loss.backward()

    def L(mass_vec, Dval):
        with torch.no_grad():
            mT2, xT2 = mtpt_run(mass_vec, torch.tensor(Dval, dtype=torch.float64), p, x0,
                                steps, checkpoint_every=20)
            return float(_misfit_torch(w, xT2, mT2, target, nb)), xT2
    # masses enter linearly and the misfit is quadratic: the central difference
    # along any direction is exact up to rounding
    v = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, w.n)).cuda()
    eps = 1e-3
    Lp, _ = L(m0.detach() + eps * v, p.D)
    Lm, _ = L(m0.detach() - eps * v, p.D)
    fd = (Lp - Lm) / (2 * eps)
    g = float((m0.grad * v).sum())
    assert abs(fd - g) <= 1e-8 * max(abs(g), 1.0), (fd, g)
    # D: binary64 central difference on the same random path.  The adjoint is
    # the derivative of the piecewise-smooth path (fixed pair set, fixed bins);
    # the cutoff radius and the steps both move with D, so the difference is
    # taken with h small enough that no pair and no bin changes between +-h,
    # and the test checks that
    hD = 1e-8 * p.D
    runs = []
    for sgn in (1, -1):
        pD = mtpt.Params(**{**p.__dict__, "D": p.D + sgn * hD})
        with mtpt.Simulation(pD, pos, mass) as sim:
            sim.step(steps)
            x2, m2, npairs = sim.positions(), sim.masses(), sim.info()["pair_count"]
        Lx = float(_misfit_torch(w, torch.from_numpy(x2), torch.from_numpy(m2),
                                 target.cpu(), nb))
        runs.append((Lx, _bins(w, x2, nb), npairs))
    assert np.array_equal(runs[0][1], runs[1][1]), "a particle changed bin between +-h"
    assert runs[0][2] == runs[1][2], "the pair set changed between +-h"
    fdD = (runs[0][0] - runs[1][0]) / (2 * hD)
    gD = float(D.grad)
    assert abs(fdD - gD) <= 1e-4 * abs(gD), (fdD, gD)


def _bins(w, x, nb):
    ix = np.clip(((x[0] - w.lo[0]) / (w.hi[0] - w.lo[0]) * nb[0]).astype(int), 0, nb[0] - 1)
    iy = np.clip(((x[1] - w.lo[1]) / (w.hi[1] - w.lo[1]) * nb[1]).astype(int), 0, nb[1] - 1)
    return ix * nb[1] + iy


def test_full_length_run_in_one_call_equals_single_steps():
    """The 4e6-particle 2-d workload for its full 1000 steps: one call (the
    walk-ahead path, its middle steps replayed from a graph) equals 1000
    calls of one step bit for bit, and the precision form's exactly
    antisymmetric fluxes keep the total mass to binary64 rounding."""
    w = workloads.get("gaussian_2d")
    assert w.steps == 1000
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=mtpt.MTPT_FP32W)
    with mtpt.Simulation(p, pos, mass) as a:
        a.step(w.steps)
        xa, ma, ia = a.positions(), a.masses(), a.info()
    with mtpt.Simulation(p, pos, mass) as b:
        for _ in range(w.steps):
            b.step(1)
        xb, mb, ib = b.positions(), b.masses(), b.info()
    assert np.array_equal(xa, xb) and np.array_equal(ma, mb)
    assert ia["step"] == ib["step"] == w.steps and ia["pair_count"] == ib["pair_count"]
    assert abs(ma.sum() - mass.sum()) <= 1e-12 * mass.sum()
