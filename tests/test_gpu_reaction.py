"""The bimolecular reaction A + B -> 0 on the GPU (the reaction extension of
Sec. 8 as the library reads it; see the oracle's run_reactive): against the
oracle in both forms and in 1-, 2- and 3-d, equal to plain transfer runs of
each species when k = 0, graph replay equal to step-by-step launches, and the
calls' argument and state checks."""
import zlib

import numpy as np
import pytest

import oracle as O
from paper_2204_03756_gb300 import mtpt

from gpu_helpers import TOL, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


def _case(name, dim, n, L, form, kappa=0.5, seed=11):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    pos = rng.uniform(0.0, L, size=(dim, n))
    pos[:, :2] = 0.0                          # on the walls
    ma = (pos[0] < L / 2).astype(np.float64)
    mb = 1.0 - ma
    mb[rng.uniform(size=n) < 0.2] *= 0.5      # uneven species B
    p = mtpt.Params(dim=dim, D=1.0, kappa=kappa, dt=0.1, lo=(0.0,) * dim, hi=(L,) * dim,
                    seed=seed, precision=form)
    return p, pos, ma, mb


# name: (dim, n, box side, form, k, steps)
CASES = {
    "2d_fp64": (2, 20_000, 60.0, mtpt.MTPT_FP64, 2.0, 12),
    "2d_fp32w": (2, 20_000, 60.0, mtpt.MTPT_FP32W, 2.0, 12),
    "3d_fp64": (3, 12_000, 20.0, mtpt.MTPT_FP64, 5.0, 8),
    "3d_fp32w": (3, 12_000, 20.0, mtpt.MTPT_FP32W, 5.0, 8),
    "1d_fp64": (1, 3_000, 1_500.0, mtpt.MTPT_FP64, 0.5, 10),
    "2d_fast_fp64": (2, 8_000, 40.0, mtpt.MTPT_FP64, 400.0, 6),
}


@pytest.mark.parametrize("name", list(CASES))
def test_reaction_matches_the_oracle(name):
    dim, n, L, form, k, steps = CASES[name]
    p, pos, ma, mb = _case(name, dim, n, L, form)
    with mtpt.Simulation(p, pos, ma) as sim:
        sim.set_reaction(k, mb)
        sim.step(steps)
        x, a, b, info = sim.positions(), sim.masses(), sim.masses_b(), sim.info()
    xr, ar, br, npairs = O.run_reactive(oracle_params(p), pos, ma, mb, steps, k)
    assert np.array_equal(x, xr)
    assert info["pair_count"] == npairs
    scale = max(np.abs(ar).max(), np.abs(br).max())
    assert np.abs(a - ar).max() / scale <= TOL[form]
    assert np.abs(b - br).max() / scale <= TOL[form]
    # the reaction consumed mass (at the front only, so little in 1-d), and
    # A - B is conserved
    assert a.sum() < ma.sum() and b.sum() < mb.sum()
    assert abs((a - b).sum() - (ma - mb).sum()) <= 1e-9 * n


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
def test_no_reaction_leaves_each_species_a_plain_transfer_run(form):
    p, pos, ma, mb = _case("k0", 2, 15_000, 50.0, form)
    with mtpt.Simulation(p, pos, ma) as sim:
        sim.set_reaction(0.0, mb)
        sim.step(7)
        a, b = sim.masses(), sim.masses_b()
    with mtpt.Simulation(p, pos, ma) as s1:
        s1.step(7)
        assert np.array_equal(a, s1.masses())
    with mtpt.Simulation(p, pos, mb) as s2:
        s2.step(7)
        assert np.array_equal(b, s2.masses())


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
def test_graph_replay_and_reloads(form):
    p, pos, ma, mb = _case("graph", 2, 15_000, 50.0, form)
    with mtpt.Simulation(p, pos, ma) as g, mtpt.Simulation(p, pos, ma) as s:
        for sim in (g, s):
            sim.set_reaction(3.0, mb)
        g.step(10)                              # captured two-step graph, replayed
        for _ in range(10):
            s.step(1)
        assert np.array_equal(g.masses(), s.masses())
        assert np.array_equal(g.masses_b(), s.masses_b())
        # a reload clears species B
        g.set_particles(pos, ma)
        assert np.array_equal(g.masses_b(), np.zeros(ma.size))
        mtpt.mtpt_set_masses_b(g.h, mb)
        assert np.array_equal(g.masses_b(), mb)


def test_reaction_calls_check_their_arguments_and_state():
    p, pos, ma, mb = _case("args", 2, 2_000, 30.0, mtpt.MTPT_FP64)
    with mtpt.Simulation(p, pos, ma) as sim:
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_set_masses_b(sim.h, mb)             # before set_reaction
        assert e.value.code == mtpt.MTPT_ERR_STATE
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(mtpt.MtptError) as e:
                mtpt.mtpt_set_reaction(sim.h, bad)
            assert e.value.code == mtpt.MTPT_ERR_INVALID_ARG
        sim.set_reaction(1.0)
        assert np.array_equal(sim.masses_b(), np.zeros(ma.size))
        neg = mb.copy()
        neg[5] = -0.1
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_set_masses_b(sim.h, neg)
        assert e.value.code == mtpt.MTPT_ERR_INVALID_ARG
        assert np.array_equal(sim.masses_b(), np.zeros(ma.size))   # unchanged
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_adjoint_forward(sim.h, 4, 2)
        assert e.value.code == mtpt.MTPT_ERR_STATE
    with mtpt.Batch([p, p], np.array([1000, 1000]), pos, ma) as b:
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_set_reaction(b.h, 1.0)
        assert e.value.code == mtpt.MTPT_ERR_STATE


def test_reaction_front_at_scale_keeps_its_invariants():
    """Species A on the left half, B on the right, 1e6 particles, 20 steps:
    masses stay non-negative, sum(A - B) is conserved, mass is lost only near
    the front, and far from it neither species ever meets the other."""
    n, L = 1_000_000, 1000.0
    p, pos, ma, mb = _case("scale", 2, n, L, mtpt.MTPT_FP32W, seed=5)
    mb = 1.0 - ma
    with mtpt.Simulation(p, pos, ma) as sim:
        sim.set_reaction(1.0, mb)
        sim.step(20)
        a, b = sim.masses(), sim.masses_b()
    assert np.all(a >= 0.0) and np.all(b >= 0.0)
    assert abs((a - b).sum() - (ma - mb).sum()) <= 1e-8 * n
    lost = ma.sum() - a.sum()
    assert 0.0 < lost < 0.05 * ma.sum()
    far = np.abs(pos[0] - L / 2) > 100.0
    assert np.all((a[far] == 0.0) | (b[far] == 0.0))
