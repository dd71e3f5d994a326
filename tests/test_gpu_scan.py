"""The one-launch cell-count scan (the counting sort's prefix sum: every tile
publishes its total, then adds those of the tiles before it): its bounded
waits.  A test hook makes one scan tile never publish, so every tile after it
runs out of polls and sums the held tile's counts directly; every step must
come out bit for bit as without the hook, and the library's count of waits
given up must rise by exactly the tiles after the held one, per scan."""
import numpy as np
import pytest

from paper_2204_03756_gb300 import mtpt, workloads

from gpu_helpers import params_of

pytestmark = pytest.mark.gpu

SCAN_TILE = 16384   # cells per scan tile
STEPS = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()
    yield
    mtpt.mtpt_debug_scan_hold(-1)


def _run(p, pos, mass, steps):
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(steps)
        info = sim.info()
        return sim.positions(), sim.masses(), info["pair_count"], info["cells"]


def _tiles(cells):
    n_cells = int(np.prod(cells))
    return (n_cells + 1 + SCAN_TILE - 1) // SCAN_TILE


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
def test_a_held_tile_changes_nothing_but_the_wait_count(form):
    w = workloads.get("uniform_mass_2d", 400_000)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    x0, m0, pairs0, cells = _run(p, pos, mass, STEPS)
    ntiles = _tiles(cells)
    assert ntiles >= 8, "the case must span several scan tiles"
    seen = mtpt.mtpt_debug_scan_hold(-1)
    try:
        # the first tile, one in the middle and the last
        for hold in sorted({0, ntiles // 2, ntiles - 1}):
            mtpt.mtpt_debug_scan_hold(hold)
            x, m, pairs, _ = _run(p, pos, mass, STEPS)
            now = mtpt.mtpt_debug_scan_hold(hold)
            assert np.array_equal(x, x0) and np.array_equal(m, m0) and pairs == pairs0, hold
            # one scan per step (the load's sort has no scan of its own)
            assert now - seen == (ntiles - 1 - hold) * STEPS, hold
            seen = now
    finally:
        mtpt.mtpt_debug_scan_hold(-1)
    # and without the hook no tile stops waiting
    x, m, pairs, _ = _run(p, pos, mass, STEPS)
    assert np.array_equal(x, x0) and np.array_equal(m, m0) and pairs == pairs0
    assert mtpt.mtpt_debug_scan_hold(-1) == seen


def test_the_hook_checks_its_argument():
    with pytest.raises(mtpt.MtptError) as e:
        mtpt.mtpt_debug_scan_hold(-2)
    assert e.value.code == mtpt.MTPT_ERR_INVALID_ARG


def test_a_scan_of_several_block_waves_keeps_parity():
    """A sparse box whose cell grid hits its cap (4 n + 64 cells): about 300
    scan tiles, nearly two waves of the one-block-per-SM scan, so tiles of the
    second wave read totals published by blocks that have already finished.  Two
    steps against the oracle: positions and pair count exact, masses within
    tolerance."""
    import oracle as O
    from gpu_helpers import TOL, oracle_params, rel_err
    n, L = 1_200_000, 12_000.0
    rng = np.random.default_rng(77)
    pos = rng.uniform(0.0, L, size=(2, n))
    mass = rng.uniform(0.0, 1.0, n)
    p = mtpt.Params(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0.0, 0.0), hi=(L, L), seed=9,
                    precision=mtpt.MTPT_FP32W)
    with mtpt.Simulation(p, pos, mass) as sim:
        cells = sim.info()["cells"]
        assert _tiles(cells) > 152        # more tiles than one scan block per SM
        sim.step(2)
        x, m, info = sim.positions(), sim.masses(), sim.info()
    xr, mr, npairs = O.run(oracle_params(p), pos, mass, 2)
    assert np.array_equal(x, xr)
    assert info["pair_count"] == npairs and npairs > 0
    assert rel_err(m, mr) <= TOL[mtpt.MTPT_FP32W]
