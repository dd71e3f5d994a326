"""The batched (ensemble) form: many independent realisations with uneven
particle counts and their own D, density, box and seed, stepped by one launch
per kernel.  Realisation k must evolve bit for bit as a single handle with its
own parameters, and both must match the oracle; multi-step calls that replay a
captured CUDA graph must equal step-by-step launches."""
import numpy as np
import pytest

import oracle as O
from paper_2204_03756_gb300 import mtpt, workloads

from gpu_helpers import TOL, oracle_params, params_of, rel_err

pytestmark = pytest.mark.gpu

FORMS = [mtpt.MTPT_FP64, mtpt.MTPT_FP32W]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


def _small_ensemble(form, kappas=(0.5, 0.5, 1.0, 0.0, 0.5)):
    e = workloads.ensemble(nreal=len(kappas), n_min=300, n_max=6000, steps=10)
    params = []
    for w, kappa in zip(e.members, kappas):
        params.append(params_of(w, precision=form, kappa=kappa))
    return e, params


@pytest.mark.parametrize("form", FORMS)
def test_batch_equals_single_handles_bit_for_bit(form):
    e, params = _small_ensemble(form)
    pos, mass = workloads.ensemble_state(e)
    with mtpt.Batch(params, e.counts, pos, mass) as b:
        b.step(7)
        bm, bx = b.split(b.masses()), b.split(b.positions())
        total_pairs = b.info()["pair_count"]
    pair_sum = 0
    for k, w in enumerate(e.members):
        p0, m0 = workloads.initial_state(w)
        with mtpt.Simulation(params[k], p0, m0) as s:
            s.step(7)
            assert np.array_equal(bx[k], s.positions()), k
            assert np.array_equal(bm[k], s.masses()), k
            pair_sum += s.info()["pair_count"]
    assert total_pairs == pair_sum


@pytest.mark.parametrize("form", FORMS)
def test_batch_matches_the_oracle(form):
    e, params = _small_ensemble(form, kappas=(0.5, 0.3, 0.5))
    pos, mass = workloads.ensemble_state(e)
    with mtpt.Batch(params, e.counts, pos, mass) as b:
        b.step(6)
        bm, bx = b.split(b.masses()), b.split(b.positions())
        for k in range(len(params)):
            info = b.realisation_info(k)
            assert info["n"] == e.counts[k]
    for k, w in enumerate(e.members):
        p0, m0 = workloads.initial_state(w)
        xr, mr, _ = O.run(oracle_params(params[k]), p0, m0, 6)
        assert np.array_equal(bx[k], xr)
        assert rel_err(bm[k], mr) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_graph_replay_equals_step_by_step(form):
    w = workloads.get("gaussian_2d", 30_000)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    with mtpt.Simulation(p, pos, mass) as a:
        a.step(9)                       # graph of two steps x4 + one direct step
        ma, xa, ia = a.masses(), a.positions(), a.info()
    with mtpt.Simulation(p, pos, mass) as b:
        for _ in range(9):
            b.step(1)
        mb, xb, ib = b.masses(), b.positions(), b.info()
    assert np.array_equal(xa, xb) and np.array_equal(ma, mb)
    assert ia["step"] == ib["step"] == 9 and ia["pair_count"] == ib["pair_count"]
    # the graph is reused across calls and after an odd step count
    with mtpt.Simulation(p, pos, mass) as c:
        c.step(4)
        c.step(1)
        c.step(4)
        assert np.array_equal(c.masses(), ma)


def test_batch_rejects_mixed_dims_and_single_set_call():
    a = mtpt.Params(dim=2, lo=(0, 0), hi=(5, 5))
    b = mtpt.Params(dim=3, lo=(0, 0, 0), hi=(5, 5, 5))
    with pytest.raises(mtpt.MtptError):
        mtpt.mtpt_create_batch([a, b])
    h = mtpt.mtpt_create_batch([a, a])
    try:
        with pytest.raises(mtpt.MtptError):
            mtpt.mtpt_set_particles(h, 2, np.ones((2, 3)), np.ones(3))
    finally:
        mtpt.mtpt_destroy(h)


@pytest.mark.parametrize("form", FORMS)
def test_tuned_grids_keep_parity_and_autotune_restores_state(form):
    w = workloads.get("uniform_mass_2d", 20_000)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    xr, mr, npairs = O.run(oracle_params(p), pos, mass, 5)
    for scale, block in ((2.0, 128), (1.25, 256), (0.5, 256)):
        with mtpt.Simulation(p, pos, mass) as s:
            s.set_tuning(scale, block)
            s.step(5)
            assert np.array_equal(s.positions(), xr)
            assert s.info()["pair_count"] == npairs
            assert rel_err(s.masses(), mr) <= TOL[form]
    with mtpt.Simulation(p, pos, mass) as s:
        s.step(2)
        m2, x2, i2 = s.masses(), s.positions(), s.info()
        t = s.autotune(trial_steps=4)
        assert t["cell_scale"] in (0.5, 1.0, 1.25, 1.5, 2.0) and t["pair_block"] in (128, 256)
        assert np.array_equal(s.masses(), m2) and np.array_equal(s.positions(), x2)
        i3 = s.info()
        assert i3["step"] == i2["step"] and i3["pair_count"] == i2["pair_count"]
        s.step(3)
        xr5, mr5, _ = O.run(oracle_params(p), pos, mass, 5)
        assert np.array_equal(s.positions(), xr5)
        assert rel_err(s.masses(), mr5) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_batch_with_per_realisation_velocities_equals_single_runs(form):
    e = workloads.ensemble(nreal=3, n_min=500, n_max=4000, steps=5)
    vs = [(0.0, 0.0), (1.0, -0.5), (-2.0, 3.0)]
    params = [params_of(w, precision=form, v=v) for w, v in zip(e.members, vs)]
    pos, mass = workloads.ensemble_state(e)
    with mtpt.Batch(params, e.counts, pos, mass) as b:
        b.step(5)
        bx, bm = b.split(b.positions()), b.split(b.masses())
    for k, w in enumerate(e.members):
        p0, m0 = workloads.initial_state(w)
        with mtpt.Simulation(params[k], p0, m0) as sim:
            sim.step(5)
            assert np.array_equal(sim.positions(), bx[k])
            assert np.array_equal(sim.masses(), bm[k])
