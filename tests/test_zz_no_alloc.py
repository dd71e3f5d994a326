"""mtpt_step_noalloc: the time step for callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or their loop cannot
afford cudaMalloc/cudaFree).  Called through the C ABI on torch-owned device
buffers, two calls in a row, and checked against the handle-based entry points
on the same state.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

from paper_2204_03756_gb300 import mtpt, workloads

pytestmark = pytest.mark.gpu

TOL = {mtpt.MTPT_FP64: 1e-12, mtpt.MTPT_FP32W: 1e-5}


def _lib():
    from paper_2204_03756_gb300 import build
    build.build()
    lib = mtpt.load()
    lib.mtpt_step_noalloc.argtypes = [ctypes.POINTER(mtpt._Params), ctypes.c_int64,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
    lib.mtpt_step_noalloc.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
@pytest.mark.parametrize("name,n", [("heaviside_2d", 10_000), ("heaviside_3d", 30_001)])
def test_noalloc_step_matches_the_handle_path_on_two_calls(form, name, n):
    import torch
    lib = _lib()
    w = workloads.get(name, n)
    pos, mass = workloads.initial_state(w)
    p = mtpt.Params(dim=w.dim, D=w.D, kappa=w.kappa, dt=w.dt, beta=w.beta, lam=w.lam,
                    lo=w.lo, hi=w.hi, seed=w.seed, precision=form)
    cp = p.c()
    stream = torch.cuda.Stream()
    pos_t = torch.from_numpy(pos.copy()).cuda()
    mass_t = torch.from_numpy(mass.copy()).cuda()
    torch.cuda.synchronize()
    with mtpt.Simulation(p, pos, mass) as ref:
        for call in range(2):
            rc = lib.mtpt_step_noalloc(ctypes.byref(cp), w.n, call, pos_t.data_ptr(),
                                       mass_t.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == mtpt.MTPT_OK, mtpt.status_string(rc)
            stream.synchronize()
            ref.step(1)
            got_m = mass_t.cpu().numpy()
            got_x = pos_t.cpu().numpy()
            want_m, want_x = ref.masses(), ref.positions()
            assert np.array_equal(got_x, want_x)
            # the handle sorts its freshly loaded state with payload records,
            # this call with sort keys: the same cell order, the same masses
            assert np.array_equal(got_m, want_m), call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    lib = _lib()
    p = mtpt.Params(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0), hi=(300, 300), seed=1)
    cp = p.c()
    n = 65_537
    pos = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    mass = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc = lib.mtpt_step_noalloc(ctypes.byref(cp), n, 0, pos.data_ptr(), mass.data_ptr(), None)
    assert rc == mtpt.MTPT_ERR_TOO_LARGE
    assert "scratch" in mtpt.status_string(rc)
    assert lib.mtpt_step_noalloc(ctypes.byref(cp), -1, 0, None, None, None) == \
        mtpt.MTPT_ERR_INVALID_ARG


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
def test_noalloc_runs_at_its_documented_limit(form):
    """MTPT_NOALLOC_MAX_PARTICLES particles in 3-d fit the scratch even when
    the box is so sparse that the cell count reaches its cap (the largest
    layout the call can need), and match the handle path."""
    import torch
    lib = _lib()
    n = mtpt.NOALLOC_MAX_PARTICLES
    rng = np.random.default_rng(31)
    L = 1000.0
    pos = rng.uniform(0.0, L, size=(3, n))
    mass = rng.uniform(0.0, 1.0, n)
    p = mtpt.Params(dim=3, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0, 0), hi=(L, L, L), seed=4,
                    precision=form)
    cp = p.c()
    pos_t = torch.from_numpy(pos.copy()).cuda()
    mass_t = torch.from_numpy(mass.copy()).cuda()
    rc = lib.mtpt_step_noalloc(ctypes.byref(cp), n, 0, pos_t.data_ptr(), mass_t.data_ptr(), None)
    assert rc == mtpt.MTPT_OK, mtpt.status_string(rc)
    torch.cuda.synchronize()
    with mtpt.Simulation(p, pos, mass) as ref:
        ref.step(1)
        assert np.array_equal(pos_t.cpu().numpy(), ref.positions())
        want = ref.masses()
    # the same kernels on the same cell order: the masses agree bit for bit
    # here too (the tolerance of the method's forms is far looser)
    got = mass_t.cpu().numpy()
    assert np.abs(got - want).max() <= TOL[form] * np.abs(want).max()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("form", [mtpt.MTPT_FP64, mtpt.MTPT_FP32W])
def test_noalloc_allocates_nothing_and_runs_through_the_binding(form):
    """The entry point's defining property: after a first call (which loads
    the kernels it launches and sets up the scratch), further calls leave the
    device's free memory and torch's caching allocator untouched.  The calls
    here go through the Python binding, on torch's current stream, and match
    the handle path on the same state."""
    import torch
    _lib()
    w = workloads.get("heaviside_2d", 20_000)
    pos, mass = workloads.initial_state(w)
    p = mtpt.Params(dim=w.dim, D=w.D, kappa=w.kappa, dt=w.dt, beta=w.beta, lam=w.lam,
                    lo=w.lo, hi=w.hi, seed=w.seed, precision=form)
    warm_x = torch.from_numpy(pos.copy()).cuda()
    warm_m = torch.from_numpy(mass.copy()).cuda()
    pos_t = torch.from_numpy(pos.copy()).cuda()
    mass_t = torch.from_numpy(mass.copy()).cuda()
    mtpt.mtpt_step_noalloc(p, 0, warm_x, warm_m)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for step in range(3):
        mtpt.mtpt_step_noalloc(p, step, pos_t, mass_t)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    with mtpt.Simulation(p, pos, mass) as ref:
        ref.step(3)
        assert np.array_equal(pos_t.cpu().numpy(), ref.positions())
        assert np.array_equal(mass_t.cpu().numpy(), ref.masses())
