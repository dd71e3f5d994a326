"""Pins of the oracle's bimolecular reaction A + B -> 0 (the reading of the
extension the paper names in Sec. 8: both species exchange mass with the same
weights, then each particle reacts well mixed over dt, rate law
dC_A/dt = dC_B/dt = -k C_A C_B with C = N M / V).

The reaction substep is pinned to the closed-form solution of that rate law
evaluated in 50-digit arithmetic and to a stiff ODE integrator; the reactive
run is pinned to plain mass transfer (k = 0), to the well-mixed solution
(uniform masses, which mass transfer leaves exactly unchanged), to the
conservation of sum(M_A - M_B), and to positivity."""
import numpy as np
import pytest

import oracle as O


def _exact(a0, b0, kp, t):
    """a(t), b(t) of da/dt = db/dt = -kp a b in 50-digit arithmetic, from
    the textbook closed form a(t) = D a0 / (a0 - b0 E), b(t) = D b0 E /
    (a0 - b0 E), D = a0 - b0, E = exp(-kp D t) (both a0 / (1 + kp a0 t) when
    D = 0; species swapped when D < 0)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    a0, b0, kp, t = (mp.mpf(float(v)) for v in (a0, b0, kp, t))
    d = a0 - b0
    if d == 0:
        a = b = a0 / (1 + kp * a0 * t)
    elif d > 0:
        e = mp.exp(-kp * d * t)
        a, b = d * a0 / (a0 - b0 * e), d * b0 * e / (a0 - b0 * e)
    else:
        e = mp.exp(kp * d * t)
        b, a = -d * b0 / (b0 - a0 * e), -d * a0 * e / (b0 - a0 * e)
    return float(a), float(b)


CASES = [(1.0, 0.5), (0.5, 1.0), (1.0, 1.0), (2.0, 1e-9), (1e-9, 2.0), (0.3, 0.3 + 1e-12),
         (5.0, 4.999999), (0.0, 1.0), (1.0, 0.0), (1e-3, 7e-3), (123.0, 45.0)]


@pytest.mark.parametrize("a0,b0", CASES)
@pytest.mark.parametrize("kp_dt", [1e-6, 1e-2, 0.3, 5.0, 200.0])
def test_react_substep_is_the_exact_solution(a0, b0, kp_dt):
    kp, dt = kp_dt / 0.1, 0.1
    a, b = O.react([a0], [b0], kp, dt)
    ea, eb = _exact(a0, b0, kp, dt)
    # a few units in the last place of each species, the one in deficit too;
    # that one carries exp(-x), x = kp |a0 - b0| dt, whose relative condition
    # number is x (x itself is rounded)
    x = kp * abs(a0 - b0) * dt
    tol = 1e-15 + 4.5e-16 * x
    assert abs(a[0] - ea) <= tol * ea + 1e-300
    assert abs(b[0] - eb) <= tol * eb + 1e-300
    assert a[0] >= 0.0 and b[0] >= 0.0
    assert a[0] - b[0] == pytest.approx(a0 - b0, abs=1e-15 * max(a0, b0))


def test_react_substeps_compose_to_the_solution_at_the_total_time():
    """The exact flow composes: n substeps of dt equal one of n dt."""
    a0 = np.array([1.0, 0.2, 3.0, 0.5])
    b0 = np.array([0.4, 0.9, 3.0, 2.5])
    kp, dt, n = 2.0, 0.05, 40
    a, b = a0.copy(), b0.copy()
    for _ in range(n):
        a, b = O.react(a, b, kp, dt)
    for i in range(a0.size):
        ea, eb = _exact(a0[i], b0[i], kp, n * dt)
        assert a[i] == pytest.approx(ea, rel=2e-14, abs=1e-16)
        assert b[i] == pytest.approx(eb, rel=2e-14, abs=1e-16)


def test_react_matches_an_ode_integrator():
    integrate = pytest.importorskip("scipy.integrate")
    kp, t = 1.7, 0.8
    for a0, b0 in [(1.0, 0.6), (0.25, 2.0), (1.0, 1.0)]:
        sol = integrate.solve_ivp(lambda _, y: [-kp * y[0] * y[1]] * 2, (0.0, t), [a0, b0],
                                  method="Radau", rtol=1e-12, atol=1e-14)
        a, b = O.react([a0], [b0], kp, t)
        assert a[0] == pytest.approx(sol.y[0, -1], rel=1e-9)
        assert b[0] == pytest.approx(sol.y[1, -1], rel=1e-9, abs=1e-12)


def test_particle_rate_is_k_n_over_the_volume():
    p2 = O.OracleParams(dim=2, lo=(0.0, -5.0, 0.0), hi=(100.0, 5.0, 0.0))
    assert O.particle_rate(p2, 4000, 0.5) == 0.5 * 4000 / (100.0 * 10.0)
    p3 = O.OracleParams(dim=3, lo=(0.0, 0.0, 0.0), hi=(2.0, 3.0, 4.0))
    assert O.particle_rate(p3, 10, 3.0) == 3.0 * 10 / 24.0


def _state(n, L, seed, dim=2):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, size=(dim, n))
    ma = (pos[0] < L / 2).astype(np.float64)
    mb = 1.0 - ma
    return pos, ma, mb


def test_without_reaction_each_species_is_a_plain_transfer_run():
    p = O.OracleParams(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0.0, 0.0), hi=(40.0, 40.0), seed=3)
    pos, ma, mb = _state(1500, 40.0, 1)
    mb = np.random.default_rng(2).uniform(0.0, 2.0, mb.size)
    x, a, b, npairs = O.run_reactive(p, pos, ma, mb, 6, k=0.0)
    xa, ra, na = O.run(p, pos, ma, 6)
    xb, rb, nb = O.run(p, pos, mb, 6)
    assert np.array_equal(x, xa) and np.array_equal(x, xb)
    assert np.array_equal(a, ra) and np.array_equal(b, rb)
    assert npairs == na == nb


def test_uniform_species_react_as_the_well_mixed_solution():
    """Mass transfer leaves uniform masses unchanged exactly, so every
    particle follows the well-mixed solution at every step."""
    p = O.OracleParams(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0.0, 0.0), hi=(30.0, 30.0), seed=4)
    n = 900
    pos = np.random.default_rng(5).uniform(0.0, 30.0, size=(2, n))
    a0, b0, k, steps = 0.8, 0.3, 0.5, 10
    _, a, b, _ = O.run_reactive(p, pos, np.full(n, a0), np.full(n, b0), steps, k)
    kp = O.particle_rate(p, n, k)
    ea, eb = _exact(a0, b0, kp, steps * p.dt)
    assert np.all(a == a[0]) and np.all(b == b[0])
    assert a[0] == pytest.approx(ea, rel=1e-14)
    assert b[0] == pytest.approx(eb, rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_reactive_run_conserves_the_species_difference_and_positivity(dim):
    L = 20.0 if dim == 2 else 9.0
    p = O.OracleParams(dim=dim, D=1.0, kappa=0.5, dt=0.1, lo=(0.0,) * 3, hi=(L,) * 3, seed=6)
    pos, ma, mb = _state(1200, L, 7, dim)
    _, a, b, npairs = O.run_reactive(p, pos, ma, mb, 15, k=2.0)
    assert npairs > 0
    assert np.all(a >= 0.0) and np.all(b >= 0.0)
    # both species lose mass (they meet at the front) by the same amount
    assert a.sum() < ma.sum() and b.sum() < mb.sum()
    drift = abs((a - b).sum() - (ma - mb).sum())
    assert drift <= 1e-12 * ma.size
    # without the reaction nothing would be lost
    _, a0, b0, _ = O.run_reactive(p, pos, ma, mb, 15, k=0.0)
    assert a0.sum() == pytest.approx(ma.sum(), rel=1e-12)
    assert b0.sum() == pytest.approx(mb.sum(), rel=1e-12)


def test_negative_masses_do_not_react_and_zero_masses_change_nothing():
    a, b = O.react([-1.0, 0.5, 0.0, -0.0, 2.0], [0.5, -1.0, 0.7, 0.3, 0.0], 3.0, 0.1)
    assert a.tolist() == [-1.0, 0.5, 0.0, -0.0, 2.0]
    assert b.tolist() == [0.5, -1.0, 0.7, 0.3, 0.0]
