"""Pipelined host I/O (mtpt_set_particles_async / mtpt_get_masses_async):
the loop load -> step -> read with the copies overlapped gives, step for step,
the masses of the synchronous calls bit for bit; a rejected load keeps the
old state and step counter and is reported once by the next sync."""
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


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _inputs(w, count, seed):
    """`count` distinct seeded inputs of the workload's size and box."""
    rng = np.random.default_rng(seed)
    pos0, mass0 = workloads.initial_state(w)
    out = [(pos0, mass0)]
    for _ in range(count - 1):
        pos = np.stack([rng.uniform(w.lo[a], w.hi[a], w.n) for a in range(w.dim)])
        out.append((pos, rng.uniform(0.0, 1.0, w.n)))
    return out


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
@pytest.mark.parametrize("name,n", [("heaviside_2d", 10000), ("heaviside_3d", 6001)])
def test_pipeline_equals_synchronous_calls(form, name, n):
    w = workloads.get(name, n)
    p = params_of(w, precision=form)
    inputs = _inputs(w, 3, 11)
    plan = [0, 1, 1, 2, 0, 2, 1]                      # input of each pipelined step
    ref = []
    with mtpt.Simulation(p, *inputs[0]) as sim:
        for k in plan:
            sim.set_particles(*inputs[k])
            sim.step(1)
            ref.append(sim.masses())
    pinned = [(_pinned(x), _pinned(m)) for x, m in inputs]
    import torch
    outs = [torch.empty(w.n, dtype=torch.float64).pin_memory() for _ in plan]
    with mtpt.Simulation(p, *inputs[0]) as sim:
        for k, out in zip(plan, outs):
            sim.set_particles_async(*pinned[k])
            sim.step(1)
            sim.masses_async(out)
        sim.sync()
        assert sim.info()["step"] == 1
    for t, (r, o) in enumerate(zip(ref, outs)):
        assert np.array_equal(o.numpy(), r), f"step {t}"


def test_pipeline_with_multi_step_runs_and_numpy_buffers():
    """Graph-replayed runs (four steps and more) between pipelined loads, host
    buffers plain numpy (pageable)."""
    w = workloads.get("heaviside_2d", 8000)
    p = params_of(w, precision=mtpt.MTPT_FP32W)
    inputs = _inputs(w, 2, 5)
    ref = []
    with mtpt.Simulation(p, *inputs[0]) as sim:
        for k, steps in [(1, 4), (0, 5), (1, 6)]:
            sim.set_particles(*inputs[k])
            sim.step(steps)
            ref.append((sim.masses(), sim.positions()))
    outs = [np.empty(w.n) for _ in ref]
    with mtpt.Simulation(p, *inputs[0]) as sim:
        for (k, steps), out in zip([(1, 4), (0, 5), (1, 6)], outs):
            sim.set_particles_async(*inputs[k])
            sim.step(steps)
            sim.masses_async(out)
        sim.sync()
        assert sim.info()["step"] == 6
        assert np.array_equal(sim.positions(), ref[-1][1])
    for (m, _), out in zip(ref, outs):
        assert np.array_equal(out, m)


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
def test_rejected_pipelined_load_keeps_state_and_is_reported_once(form):
    w = workloads.get("heaviside_2d", 3000)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    with mtpt.Simulation(p, pos, mass) as ref:
        ref.step(5)
        m_ref, x_ref = ref.masses(), ref.positions()
    bad = []
    b = pos.copy(); b[0, 17] = w.hi[0] + 1e-9; bad.append((b, mass, mtpt.MTPT_ERR_OUT_OF_DOMAIN))
    b = pos.copy(); b[1, 4] = np.nan; bad.append((b, mass, mtpt.MTPT_ERR_OUT_OF_DOMAIN))
    m = mass.copy(); m[9] = np.inf; bad.append((pos, m, mtpt.MTPT_ERR_INVALID_ARG))
    if form == mtpt.MTPT_FP32W:
        m = mass.copy(); m[3] = -2e30; bad.append((pos, m, mtpt.MTPT_ERR_INVALID_ARG))
    for bp, bm, code in bad:
        with mtpt.Simulation(p, pos, mass) as sim:
            sim.step(2)
            sim.set_particles_async(bp, bm)           # rejected on the device
            sim.step(3)                               # runs on the kept state
            out = np.empty(w.n)
            sim.masses_async(out)
            with pytest.raises(mtpt.MtptError) as e:
                sim.sync()
            assert e.value.code == code
            sim.sync()                                # reported once
            assert np.array_equal(out, m_ref)
            assert np.array_equal(sim.positions(), x_ref)
            assert sim.info()["step"] == 5
            # an accepted load after the rejected one
            sim.set_particles_async(pos, mass)
            sim.step(5)
            sim.masses_async(out)
            sim.sync()
            assert np.array_equal(out, m_ref)


def test_argument_errors():
    w = workloads.get("heaviside_2d", 1000)
    pos, mass = workloads.initial_state(w)
    with mtpt.Simulation(params_of(w), pos, mass) as sim:
        with pytest.raises(mtpt.MtptError) as e:
            sim.set_particles_async(pos[:, :999].copy(), mass[:999].copy())
        assert e.value.code == mtpt.MTPT_ERR_INVALID_ARG
        with pytest.raises(ValueError):
            sim.set_particles_async(pos[:, ::1].T, mass)          # not C-contiguous
        with pytest.raises(ValueError):
            sim.set_particles_async(pos.astype(np.float32), mass)
        with pytest.raises(ValueError):
            sim.masses_async(np.empty(w.n, dtype=np.float32))
    members = [workloads.get("heaviside_2d", 500), workloads.get("heaviside_2d", 700)]
    states = [workloads.initial_state(m) for m in members]
    counts = [m.n for m in members]
    bpos = np.concatenate([s[0] for s in states], axis=1)
    bmass = np.concatenate([s[1] for s in states])
    with mtpt.Batch([params_of(m) for m in members], counts, bpos, bmass) as b:
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_set_particles_async(b.h, 2, bpos, bmass)
        assert e.value.code == mtpt.MTPT_ERR_INVALID_ARG


def test_pipeline_on_a_user_stream_with_timing_and_a_one_member_batch():
    """The pipelined calls on a caller's stream with per-kernel timing on, and
    on a batch handle of one realisation, give the single handle's masses."""
    import torch
    w = workloads.get("heaviside_2d", 6000)
    p = params_of(w, precision=mtpt.MTPT_FP32W)
    inputs = _inputs(w, 2, 9)
    ref = []
    with mtpt.Simulation(p, *inputs[0]) as sim:
        for k in (1, 0, 1):
            sim.set_particles(*inputs[k])
            sim.step(2)
            ref.append(sim.masses())
    pinned = [(_pinned(x), _pinned(m)) for x, m in inputs]
    stream = torch.cuda.Stream()
    outs = [torch.empty(w.n, dtype=torch.float64).pin_memory() for _ in ref]
    with mtpt.Simulation(p, *inputs[0]) as sim:
        mtpt.mtpt_set_stream(sim.h, stream.cuda_stream)
        mtpt.mtpt_timing_enable(sim.h, True)
        for k, out in zip((1, 0, 1), outs):
            sim.set_particles_async(*pinned[k])
            sim.step(2)
            sim.masses_async(out)
        sim.sync()
        stats = mtpt.mtpt_timing_read(sim.h)
        # six pass-2 launches: each call's first step walks ahead for its second
        assert stats["load_input"][0] == 3
        assert stats["exchange_f32"][0] == 3 and stats["exchange_walk_f32"][0] == 3
        assert stats["walk_key"][0] == 3
    for r, o in zip(ref, outs):
        assert np.array_equal(o.numpy(), r)
    outs_b = [np.empty(w.n) for _ in ref]
    with mtpt.Batch([p], [w.n], *inputs[0]) as b:
        for k, out in zip((1, 0, 1), outs_b):
            mtpt.mtpt_set_particles_async(b.h, 2, *inputs[k])
            b.step(2)
            mtpt.mtpt_get_masses_async(b.h, out)
        b.sync()
    for r, o in zip(ref, outs_b):
        assert np.array_equal(o, r)
