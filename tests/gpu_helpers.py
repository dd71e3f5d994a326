"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare."""
import numpy as np

import oracle as O
from paper_2204_03756_gb300 import mtpt, workloads

# Tolerances (relative to max |M_ref|): binary64 form 1e-12, precision form 1e-5.
TOL = {mtpt.MTPT_FP64: 1e-12, mtpt.MTPT_FP32W: 1e-5}


def params_of(w, precision=mtpt.MTPT_FP64, **over):
    kw = dict(dim=w.dim, D=w.D, kappa=w.kappa, dt=w.dt, beta=w.beta, lam=w.lam,
              lo=w.lo, hi=w.hi, seed=w.seed, precision=precision, v=w.v)
    kw.update(over)
    return mtpt.Params(**kw)


def oracle_params(p: mtpt.Params) -> O.OracleParams:
    lo = tuple(p.lo) + (0.0,) * (3 - len(p.lo))
    hi = tuple(p.hi) + (0.0,) * (3 - len(p.hi))
    v = tuple(p.v) + (0.0,) * (3 - len(p.v))
    return O.OracleParams(dim=p.dim, D=p.D, kappa=p.kappa, dt=p.dt, beta=p.beta, lam=p.lam,
                          lo=lo, hi=hi, seed=p.seed, v=v[:3])


def rel_err(got, ref) -> float:
    scale = np.abs(ref).max()
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / (scale if scale > 0 else 1.0))


def run_both(p: mtpt.Params, pos, mass, steps, method="kdtree"):
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(steps)
        out = dict(pos=sim.positions(), mass=sim.masses(), info=sim.info())
    xr, mr, npairs = O.run(oracle_params(p), pos, mass, steps, method=method)
    return out, dict(pos=xr, mass=mr, pairs=npairs)
