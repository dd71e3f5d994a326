"""Allocation failures on the host side (failure detection without a GPU
fault): the library's device allocations are made to fail one at a time, at
every point a call can meet one, and the handle must report
MTPT_ERR_NO_MEMORY and keep its particles, counters and tuning; afterwards it
steps on exactly as a handle that never saw the failure."""
import numpy as np
import pytest

from paper_2204_03756_gb300 import mtpt, workloads

from gpu_helpers import params_of

pytestmark = pytest.mark.gpu

FORMS = [mtpt.MTPT_FP64, mtpt.MTPT_FP32W]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()
    yield
    mtpt.mtpt_debug_fail_alloc(0)


def _state(sim):
    info = sim.info()
    return sim.positions(), sim.masses(), (info["step"], info["pair_count"])


def _same(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def _case(form, n):
    w = workloads.get("uniform_mass_2d", n)
    pos, mass = workloads.initial_state(w)
    return params_of(w, precision=form), pos, mass


def _every_failure_point(call, max_points=80):
    """Runs `call(nth)`, which arms the nth allocation to fail right before
    the operation it tests, for nth = 1, 2, ... until a run meets no failure;
    returns how many failure points it met."""
    for nth in range(1, max_points + 1):
        hit = call(nth)
        left = mtpt.mtpt_debug_fail_alloc(0)
        if not hit:
            assert left > 0            # the armed failure was never reached
            return nth - 1
    raise AssertionError("more allocation points than expected")


@pytest.mark.parametrize("form", FORMS)
def test_load_that_cannot_allocate_keeps_the_old_state(form):
    p, pos, mass = _case(form, 3000)
    rng = np.random.default_rng(9)               # a larger load in the same box: every buffer grows
    pos2 = np.vstack([rng.uniform(p.lo[a], p.hi[a], 40000) for a in range(2)])
    mass2 = rng.uniform(0.0, 1.0, 40000)
    with mtpt.Simulation(p, pos, mass) as ref:
        ref.step(5)
        want = _state(ref)

    def attempt(nth):
        with mtpt.Simulation(p, pos, mass) as sim:
            sim.step(2)
            before = _state(sim)
            mtpt.mtpt_debug_fail_alloc(nth)
            try:
                mtpt.mtpt_set_particles(sim.h, 2, pos2, mass2)
                hit = False
            except mtpt.MtptError as e:
                assert e.code == mtpt.MTPT_ERR_NO_MEMORY
                hit = True
                mtpt.mtpt_debug_fail_alloc(0)
                assert _same(_state(sim), before)
                sim.step(3)                       # steps on as if nothing happened
                assert _same(_state(sim), want)
            return hit

    assert _every_failure_point(attempt) >= 10


@pytest.mark.parametrize("form", FORMS)
def test_steps_allocate_nothing(form):
    p, pos, mass = _case(form, 20000)
    with mtpt.Simulation(p, pos, mass) as sim:
        mtpt.mtpt_debug_fail_alloc(1)
        sim.step(1)                              # the first sort after the load
        sim.step(6)                              # a captured two-step graph, replayed
        assert mtpt.mtpt_debug_fail_alloc(0) == 1


@pytest.mark.parametrize("form", FORMS)
def test_autotune_that_cannot_allocate_keeps_state_and_tuning(form):
    p, pos, mass = _case(form, 20000)

    def attempt(nth):
        with mtpt.Simulation(p, pos, mass) as sim:
            sim.set_tuning(1.5, 128)
            sim.step(2)
            before = _state(sim)
            mtpt.mtpt_debug_fail_alloc(nth)
            try:
                sim.autotune(trial_steps=1)
                return False
            except mtpt.MtptError as e:
                assert e.code == mtpt.MTPT_ERR_NO_MEMORY
                mtpt.mtpt_debug_fail_alloc(0)
                assert _same(_state(sim), before)
                assert mtpt.mtpt_get_tuning(sim.h) == {"cell_scale": 1.5, "pair_block": 128}
                sim.step(2)
                with mtpt.Simulation(p, pos, mass) as ref:
                    ref.set_tuning(1.5, 128)
                    ref.step(4)
                    assert _same(_state(sim), _state(ref))
                return True

    assert _every_failure_point(attempt) >= 2


def test_adjoint_recording_that_cannot_allocate_keeps_state():
    p, pos, mass = _case(mtpt.MTPT_FP64, 5000)

    def attempt(nth):
        with mtpt.Simulation(p, pos, mass) as sim:
            sim.step(1)
            before = _state(sim)
            mtpt.mtpt_debug_fail_alloc(nth)
            try:
                mtpt.mtpt_adjoint_forward(sim.h, 6, 3)
                return False
            except mtpt.MtptError as e:
                assert e.code == mtpt.MTPT_ERR_NO_MEMORY
                mtpt.mtpt_debug_fail_alloc(0)
                assert _same(_state(sim), before)
                mtpt.mtpt_adjoint_forward(sim.h, 6, 3)   # now it records
                with mtpt.Simulation(p, pos, mass) as ref:
                    ref.step(7)
                    assert _same(_state(sim), _state(ref))
                return True

    assert _every_failure_point(attempt) >= 5
