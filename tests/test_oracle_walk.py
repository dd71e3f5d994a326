"""Pins of the oracle's random walk and reflecting walls (Sec. 3:
X_i(t + dt) = X_i(t) + xi_i sqrt(2 D_RW dt), zero-flux walls by elastic
reflection)."""
import numpy as np

import oracle as O


def _params(**kw):
    base = dict(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0.0, 0.0, 0.0), hi=(100.0, 100.0, 0.0),
                seed=99)
    base.update(kw)
    return O.OracleParams(**base)


def test_reflection_is_the_mirror_image():
    assert O.reflect(-0.25, 0.0, 10.0) == 0.25
    assert O.reflect(10.5, 0.0, 10.0) == 9.5
    assert O.reflect(0.0, 0.0, 10.0) == 0.0          # walls are inside
    assert O.reflect(10.0, 0.0, 10.0) == 10.0
    assert O.reflect(3.0, 0.0, 10.0) == 3.0
    assert O.reflect(-3.0, -5.0, 5.0) == -3.0
    assert O.reflect(-5.5, -5.0, 5.0) == -4.5
    assert O.reflect(23.0, 0.0, 10.0) == 3.0         # two mirrors: 23 -> -3 -> 3
    assert O.reflect(1e9, 0.0, 10.0) == 10.0         # beyond 64 mirrors: nearest wall


def test_no_walk_when_kappa_is_zero():
    rng = np.random.default_rng(1)
    pos = rng.uniform(0, 100, size=(2, 1000))
    out = O.random_walk(_params(kappa=0.0), pos, np.arange(1000), 0)
    assert np.array_equal(out, pos)


def test_walk_displacement_is_sqrt_2_drw_dt_times_the_normals():
    n = 200_000
    p = _params(kappa=0.7, D=2.0, dt=0.05, lo=(-1e6, -1e6, 0), hi=(1e6, 1e6, 0))
    pos = np.zeros((2, n))
    ids = np.arange(n, dtype=np.uint32)
    out = O.random_walk(p, pos, ids, 5)
    sigma = np.sqrt(2.0 * 0.7 * 2.0 * 0.05)
    z = O.normals(p.seed, ids, 5)
    assert np.array_equal(out[0], sigma * z[:, 0].astype(np.float64))
    assert np.array_equal(out[1], sigma * z[:, 1].astype(np.float64))
    var = out.var(axis=1)
    assert np.all(np.abs(var - 2 * 0.7 * 2.0 * 0.05) < 5 * np.sqrt(2.0 / n) * sigma ** 2)
    assert np.all(np.abs(out.mean(axis=1)) < 5 * sigma / np.sqrt(n))


def test_walk_3d_uses_three_independent_normals():
    n = 100_000
    p = _params(dim=3, lo=(-1e3,) * 3, hi=(1e3,) * 3)
    out = O.random_walk(p, np.zeros((3, n)), np.arange(n), 0)
    cc = np.corrcoef(out)
    assert np.abs(cc - np.eye(3)).max() < 5 / np.sqrt(n)


def test_walls_are_never_crossed_and_reflection_gives_a_half_normal():
    n = 200_000
    p = _params(D=1.0, kappa=1.0, dt=0.1, hi=(10.0, 10.0, 0.0))
    pos = np.zeros((2, n))          # every particle starts on the lower walls
    out = O.random_walk(p, pos, np.arange(n), 0)
    assert out.min() >= 0.0 and out.max() <= 10.0
    sigma = np.sqrt(2.0 * 1.0 * 0.1)
    # |sigma xi| has mean sigma sqrt(2/pi)
    assert abs(out[0].mean() - sigma * np.sqrt(2.0 / np.pi)) < 5 * sigma / np.sqrt(n)
    z = O.normals(p.seed, np.arange(n), 0)
    assert np.array_equal(out[0], np.abs(sigma * z[:, 0].astype(np.float64)))


# --- advection: the velocity term of the model equation (Sec. 2) ---------------

def test_advection_without_random_walk_is_an_exact_translation():
    """kappa = 0 (no random walk): every step moves every particle by exactly
    the rounded v dt per axis, so T steps equal T binary64 additions of it."""
    rng = np.random.default_rng(31)
    n = 500
    pos = rng.uniform(300.0, 700.0, size=(2, n))
    v = (0.75, -1.3)
    p = O.OracleParams(dim=2, D=1.0, kappa=0.0, dt=0.1, lo=(0, 0, 0), hi=(1000, 1000, 0),
                       seed=4, v=v + (0.0,))
    ids = np.arange(n, dtype=np.uint32)
    x = pos.copy()
    want = pos.copy()
    for t in range(25):
        x = O.random_walk(p, x, ids, t)
        for a in range(2):
            want[a] = want[a] + v[a] * 0.1
    assert np.array_equal(x, want)


def test_advection_adds_v_t_to_the_mean_displacement():
    """With the random walk on, the mean displacement is v t and its variance
    per axis 2 D_RW t (far from the walls)."""
    rng = np.random.default_rng(32)
    n, steps, dt = 20000, 40, 0.1
    pos = rng.uniform(4000.0, 6000.0, size=(2, n))
    v = (0.5, -0.25)
    p = O.OracleParams(dim=2, D=1.0, kappa=1.0, dt=dt, lo=(0, 0, 0), hi=(10000, 10000, 0),
                       seed=8, v=v + (0.0,))
    ids = np.arange(n, dtype=np.uint32)
    x = pos.copy()
    for t in range(steps):
        x = O.random_walk(p, x, ids, t)
    T = steps * dt
    for a in range(2):
        d = x[a] - pos[a]
        assert abs(d.mean() - v[a] * T) < 4 * np.sqrt(2 * T / n), (a, d.mean())
        assert abs(d.var() - 2 * T) < 0.05 * 2 * T, (a, d.var())


def test_advection_into_a_wall_is_mirrored():
    """A particle carried past a wall by v dt lands on its mirror image, and no
    particle ever leaves the box."""
    p = O.OracleParams(dim=1, D=1.0, kappa=0.0, dt=0.5, lo=(0, 0, 0), hi=(10, 0, 0),
                       seed=1, v=(3.0, 0.0, 0.0))
    x = np.array([[9.0, 0.5, 5.0]])
    ids = np.arange(3, dtype=np.uint32)
    x1 = O.random_walk(p, x, ids, 0)
    assert np.array_equal(x1[0], [2 * 10.0 - (9.0 + 1.5), 0.5 + 1.5, 5.0 + 1.5])
    rng = np.random.default_rng(33)
    y = rng.uniform(0, 10, size=(1, 400))
    q = O.OracleParams(dim=1, D=2.0, kappa=1.0, dt=0.5, lo=(0, 0, 0), hi=(10, 0, 0),
                       seed=2, v=(7.0, 0.0, 0.0))
    for t in range(30):
        y = O.random_walk(q, y, np.arange(400, dtype=np.uint32), t)
        assert (y >= 0).all() and (y <= 10).all()
