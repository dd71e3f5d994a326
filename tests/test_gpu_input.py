"""Host-loaded input is checked on the device (positions inside their
realisation's box, masses finite and, in the precision form, at most 1e30 in
magnitude) before the handle's state is touched: a rejected load keeps the old
particles, masses and step counter."""
import numpy as np
import pytest

from paper_2204_03756_gb300 import mtpt, workloads

from gpu_helpers import params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
def test_rejected_host_loads_keep_the_old_state(form):
    w = workloads.get("heaviside_2d", 3000)
    pos, mass = workloads.initial_state(w)
    with mtpt.Simulation(params_of(w, precision=form), pos, mass) as sim:
        sim.step(3)
        x0, m0, info0 = sim.positions(), sim.masses(), sim.info()
        bad_cases = []
        p = pos.copy(); p[0, 17] = w.hi[0] + 1e-9; bad_cases.append((p, mass, mtpt.MTPT_ERR_OUT_OF_DOMAIN))
        p = pos.copy(); p[1, -1] = np.nan; bad_cases.append((p, mass, mtpt.MTPT_ERR_OUT_OF_DOMAIN))
        p = pos.copy(); p[1, 5] = -np.inf; bad_cases.append((p, mass, mtpt.MTPT_ERR_OUT_OF_DOMAIN))
        m = mass.copy(); m[9] = np.inf; bad_cases.append((pos, m, mtpt.MTPT_ERR_INVALID_ARG))
        m = mass.copy(); m[0] = np.nan; bad_cases.append((pos, m, mtpt.MTPT_ERR_INVALID_ARG))
        if form == mtpt.MTPT_FP32W:
            m = mass.copy(); m[3] = -2e30; bad_cases.append((pos, m, mtpt.MTPT_ERR_INVALID_ARG))
        for bp, bm, code in bad_cases:
            with pytest.raises(mtpt.MtptError) as e:
                mtpt.mtpt_set_particles(sim.h, 2, bp, bm)
            assert e.value.code == code
            assert np.array_equal(sim.positions(), x0)
            assert np.array_equal(sim.masses(), m0)
            assert sim.info()["step"] == info0["step"]
        # the walls themselves are inside, -0 as well as +0 at a wall at 0
        p = pos.copy(); p[0, 0] = w.lo[0]; p[1, 1] = w.hi[1]; p[0, 2] = -0.0; p[1, 3] = 0.0
        mtpt.mtpt_set_particles(sim.h, 2, p, mass)
        assert sim.info()["step"] == 0
        assert np.array_equal(sim.positions(), p)


def test_batch_load_checks_each_realisation_against_its_own_box():
    members = [workloads.get("heaviside_2d", 800), workloads.get("heaviside_2d", 3000)]
    states = [workloads.initial_state(w) for w in members]
    counts = [w.n for w in members]
    pos = np.concatenate([s[0] for s in states], axis=1)
    mass = np.concatenate([s[1] for s in states])
    params = [params_of(w) for w in members]
    with mtpt.Batch(params, counts, pos, mass) as b:
        x0 = b.positions()
        # inside the larger box of realisation 1, outside realisation 0's box
        bad = pos.copy()
        bad[0, 5] = 0.5 * (members[0].hi[0] + members[1].hi[0])
        assert members[0].hi[0] < bad[0, 5] < members[1].hi[0]
        with pytest.raises(mtpt.MtptError) as e:
            b.set_particles_batch(counts, bad, mass)
        assert e.value.code == mtpt.MTPT_ERR_OUT_OF_DOMAIN
        assert np.array_equal(b.positions(), x0)
        # the same coordinate is fine for a particle of realisation 1
        ok = pos.copy()
        ok[0, counts[0] + 5] = bad[0, 5]
        b.set_particles_batch(counts, ok, mass)
        assert np.array_equal(b.positions(), ok)
