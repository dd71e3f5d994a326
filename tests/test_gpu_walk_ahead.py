"""Walk-ahead in multi-step calls of a plain handle or a batch: the pass 2 of
every step but a call's last also does the next step's walk (the walk of
Sec. 3, with the advection term of Sec. 8 when there is a velocity, then the
next counting sort's keys), writing into the other buffer pair, in both
forms.  A call of n steps must equal n calls of one step, which never walk
ahead, bit for bit -- positions, masses, pair count and step counter --
through the first step's record sort after a host load, the one-step graph
replayed for the middle steps (one per buffer parity, so consecutive calls
alternate), reloads between calls, list overflow and batches, in 1-, 2- and
3-d; and the oracle still agrees."""
import numpy as np
import pytest

import oracle as O
from paper_2204_03756_gb300 import mtpt

from gpu_helpers import TOL, oracle_params, rel_err

pytestmark = pytest.mark.gpu

FP32W = mtpt.MTPT_FP32W
CALLS = [2, 3, 7, 1, 12, 5, 6]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


def _state(sim):
    info = sim.info()
    return sim.positions(), sim.masses(), info["pair_count"], info["step"]


def _same(a, b):
    return (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
            and a[3] == b[3])


def _case(dim, n, L, seed=21, form=FP32W, v=None):
    rng = np.random.default_rng(100 + dim)
    pos = rng.uniform(0.0, L, size=(dim, n))
    mass = (pos[0] < L / 2).astype(np.float64) + 0.25 * rng.uniform(size=n)
    extra = {} if v is None else {"v": v}
    p = mtpt.Params(dim=dim, D=1.0, kappa=0.5, dt=0.1, lo=(0.0,) * dim, hi=(L,) * dim,
                    seed=seed, precision=form, **extra)
    return p, pos, mass


CASES = [(1, 3000, 1500.0, FP32W, None), (2, 40000, 150.0, FP32W, None),
         (3, 30000, 30.0, FP32W, None), (2, 30000, 130.0, mtpt.MTPT_FP64, None),
         (3, 20000, 26.0, mtpt.MTPT_FP64, None), (2, 30000, 130.0, FP32W, (0.7, -0.4)),
         (2, 20000, 110.0, mtpt.MTPT_FP64, (0.0, 1.3))]


@pytest.mark.parametrize("dim,n,L,form,v", CASES)
def test_calls_of_many_steps_equal_single_steps(dim, n, L, form, v):
    p, pos, mass = _case(dim, n, L, form=form, v=v)
    with mtpt.Simulation(p, pos, mass) as a, mtpt.Simulation(p, pos, mass) as b:
        for k in CALLS:
            a.step(k)
            for _ in range(k):
                b.step(1)
            assert _same(_state(a), _state(b)), k
        # a host load between calls: the next call's first step sorts the
        # input-order particles through records, then walks ahead
        a.set_particles(pos, mass)
        b.set_particles(pos, mass)
        for k in (9, 4):
            a.step(k)
            for _ in range(k):
                b.step(1)
            assert _same(_state(a), _state(b)), k


def test_walk_ahead_with_list_overflow_and_the_oracle():
    # a dense clump (lists over capacity: pass 2 searches, reading the
    # positions the walk-ahead must leave alone) inside a sparse box
    rng = np.random.default_rng(12)
    sparse = rng.uniform(0, 60.0, size=(2, 3000))
    clump = 30.0 + rng.uniform(-0.4, 0.4, size=(2, 150))
    pos = np.concatenate([sparse, clump], axis=1)
    mass = rng.uniform(0, 1, pos.shape[1])
    p = mtpt.Params(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0), hi=(60, 60), seed=8,
                    precision=FP32W)
    steps = 9
    with mtpt.Simulation(p, pos, mass) as a, mtpt.Simulation(p, pos, mass) as b:
        a.step(steps)
        for _ in range(steps):
            b.step(1)
        sa = _state(a)
        assert _same(sa, _state(b))
    xr, mr, npairs = O.run(oracle_params(p), pos, mass, steps)
    assert np.array_equal(sa[0], xr)
    assert sa[2] == npairs
    assert rel_err(sa[1], mr) <= TOL[FP32W]


def test_pipelined_loads_between_walk_ahead_calls():
    p, pos, mass = _case(2, 20000, 100.0, seed=5)
    pos2 = np.ascontiguousarray(pos[:, ::-1])        # the same particles, reversed
    mass2 = np.ascontiguousarray(mass[::-1])
    with mtpt.Simulation(p, pos, mass) as a, mtpt.Simulation(p, pos, mass) as b:
        for src_pos, src_mass in ((pos2, mass2), (pos, mass), (pos2, mass2)):
            mtpt.mtpt_set_particles_async(a.h, 2, src_pos, src_mass)
            a.step(6)
            mtpt.mtpt_sync(a.h)
            b.set_particles(src_pos, src_mass)
            for _ in range(6):
                b.step(1)
            assert _same(_state(a), _state(b))


@pytest.mark.parametrize("form", [FP32W, mtpt.MTPT_FP64])
def test_batch_calls_of_many_steps_equal_single_steps(form):
    from paper_2204_03756_gb300 import workloads
    from gpu_helpers import params_of
    e = workloads.ensemble(nreal=4, n_min=400, n_max=8000, steps=10)
    params = [params_of(w, precision=form, kappa=kappa)
              for w, kappa in zip(e.members, (0.5, 0.2, 0.5, 1.0))]
    pos, mass = workloads.ensemble_state(e)
    with mtpt.Batch(params, e.counts, pos, mass) as a, \
            mtpt.Batch(params, e.counts, pos, mass) as b:
        for k in (5, 2, 8, 1, 6):
            a.step(k)
            for _ in range(k):
                b.step(1)
            assert np.array_equal(a.positions(), b.positions()), k
            assert np.array_equal(a.masses(), b.masses()), k
            assert a.info()["pair_count"] == b.info()["pair_count"], k
