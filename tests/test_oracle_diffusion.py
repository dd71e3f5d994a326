"""Pins of the oracle's whole time step against the diffusion equation it
discretises (Sec. 2.1: a Heaviside initial condition has an erfc solution;
C = N M / L^d).  The effective diffusion coefficient fitted to the erfc
profile must be the D that was put in, for the pure random walk (kappa = 1),
pure mass transfer (kappa = 0) and the paper's 50/50 split; a dropped factor
of 2, a wrong kernel variance or a sign error moves it far outside the band.
Runs at the paper's density 10 (where dt satisfies the optimality condition of
Sec. 2.2)."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle as O
from oracle import analytic as A


def _fit_D(x, m, t, x0, lo, hi, nbins):
    c, mean, _ = A.binned_profile(x, m, lo, hi, nbins)
    f = lambda D: A.rmse(mean, A.erf_profile(c, t, D, x0, "left"))
    r = minimize_scalar(f, bounds=(0.05, 5.0), method="bounded")
    return r.x, f(r.x)


@pytest.mark.parametrize("kappa,band", [(1.0, (0.9, 1.1)), (0.0, (0.85, 1.05)),
                                        (0.5, (0.88, 1.08))])
def test_heaviside_diffuses_into_erfc(kappa, band):
    rng = np.random.default_rng(5)
    n, Lx, Ly = 8000, 80.0, 10.0                       # density 10
    pos = np.stack([rng.uniform(0, Lx, n), rng.uniform(0, Ly, n)])
    m = (pos[0] < 40.0).astype(np.float64)
    p = O.OracleParams(dim=2, D=1.0, kappa=kappa, dt=0.1, lo=(0, 0, 0), hi=(Lx, Ly, 0),
                       seed=11)
    pos2, m2, npairs = O.run(p, pos, m, 50)            # t = 5
    assert abs(m2.sum() - m.sum()) < 1e-9
    D_fit, err = _fit_D(pos2[0], m2, 5.0, 40.0, 0.0, Lx, 40)
    assert band[0] <= D_fit <= band[1], (kappa, D_fit)
    assert err < 0.02
    if kappa == 1.0:
        assert npairs == 0 and np.array_equal(np.sort(m2), np.sort(m))
    else:
        assert npairs > 0


def test_gaussian_point_source_spreads_by_2Dt():
    rng = np.random.default_rng(8)
    n, L = 16000, 40.0                                  # density 10
    pos = rng.uniform(0, L, size=(2, n))
    s0 = 2.0
    r2 = ((pos - L / 2) ** 2).sum(0)
    m = np.exp(-r2 / (2 * s0 * s0))
    p = O.OracleParams(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0, 0), hi=(L, L, 0), seed=3)
    pos2, m2, _ = O.run(p, pos, m, 30)                  # t = 3
    w = m2 / m2.sum()
    for a in range(2):
        mu = (w * pos2[a]).sum()
        var = (w * (pos2[a] - mu) ** 2).sum()
        expect = A.point_source_variance(s0, 1.0, 3.0)  # 4 + 6 = 10
        assert abs(var - expect) < 0.08 * expect, (a, var, expect)


def test_concentration_from_masses():
    # C = N M / L^d; at unit density the concentration is the particle mass
    assert np.allclose(A.concentration([0.5, 1.0], 10_000, 100.0, 2), [0.5, 1.0])
    assert np.allclose(A.concentration([1.0], 1000, 10.0, 3), [1.0])


def test_advected_heaviside_front_moves_by_v_t():
    """Advection-diffusion (model equation of Sec. 2 with a uniform v): the
    Heaviside front is the erfc profile translated by v t.  Fitting both the
    shift and D recovers v t and the D that was put in (walls far enough from
    the front that the depleted and crowded strips near them do not reach
    it)."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(6)
    n, Lx, Ly = 20000, 200.0, 10.0                      # density 10
    pos = np.stack([rng.uniform(0, Lx, n), rng.uniform(0, Ly, n)])
    m = (pos[0] < 100.0).astype(np.float64)
    v, steps, dt = 2.0, 100, 0.1                        # t = 10: front 100 -> 120
    p = O.OracleParams(dim=2, D=1.0, kappa=0.5, dt=dt, lo=(0, 0, 0), hi=(Lx, Ly, 0),
                       seed=12, v=(v, 0.0, 0.0))
    pos2, m2, _ = O.run(p, pos, m, steps)
    t = steps * dt
    c, mean, counts = A.binned_profile(pos2[0], m2, 0.0, Lx, 100)
    sel = (c > 100.0) & (c < 140.0)
    f = lambda q: A.rmse(mean[sel], A.erf_profile(c[sel], t, q[1], 100.0 + q[0], "left"))
    r = minimize(f, x0=[15.0, 0.8], bounds=[(0.0, 40.0), (0.1, 5.0)], method="L-BFGS-B")
    shift, D_fit = r.x
    assert abs(shift - v * t) < 0.6, shift
    assert 0.85 <= D_fit <= 1.1, D_fit
    assert f(r.x) < 0.03
