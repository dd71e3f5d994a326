"""Workloads run twice by tests/test_gpu_checked.py: once on the normal
library and once, in a child process, on the bounds-checked build
(MTPT_LIBRARY=checked).  run() returns every result array by name; main()
(the child) saves them and the check word to an .npz file."""
import ctypes
import sys

import numpy as np

from paper_2204_03756_gb300 import mtpt, workloads


def _params(w, form, **over):
    kw = dict(dim=w.dim, D=w.D, kappa=w.kappa, dt=w.dt, beta=w.beta, lam=w.lam,
              lo=w.lo, hi=w.hi, seed=w.seed, precision=form)
    kw.update(over)
    return mtpt.Params(**kw)


def run() -> dict:
    import torch
    out = {}
    forms = {"fp64": mtpt.MTPT_FP64, "fp32w": mtpt.MTPT_FP32W}
    # single runs, 2-d and 3-d, both forms; host loads twice (in-place path)
    for name, n, steps in (("gaussian_2d", 100_000, 3), ("heaviside_3d", 50_000, 2)):
        w = workloads.get(name, n)
        pos, mass = workloads.initial_state(w)
        for fk, form in forms.items():
            with mtpt.Simulation(_params(w, form), pos, mass) as sim:
                sim.step(steps)
                mtpt.mtpt_set_particles(sim.h, w.dim, pos, mass)
                sim.step(steps)
                out[f"{name}_{fk}_m"] = sim.masses()
                out[f"{name}_{fk}_x"] = sim.positions()
                out[f"{name}_{fk}_r"] = sim.row_sums()
                gi, gj = sim.pairs()
                out[f"{name}_{fk}_pairs"] = np.stack([gi, gj])
    # advection (uniform velocity), both forms
    w = workloads.get("advection_2d", 30_000)
    pos, mass = workloads.initial_state(w)
    for fk, form in forms.items():
        with mtpt.Simulation(_params(w, form, v=w.v), pos, mass) as sim:
            sim.step(4)
            out[f"advection_{fk}_m"] = sim.masses()
            out[f"advection_{fk}_x"] = sim.positions()
    # pipelined host loads and reads, one of them rejected on the device
    w = workloads.get("heaviside_2d", 20_000)
    pos, mass = workloads.initial_state(w)
    bad = pos.copy()
    bad[0, 7] = w.hi[0] + 1.0
    outs = [np.empty(w.n) for _ in range(3)]
    with mtpt.Simulation(_params(w, mtpt.MTPT_FP32W), pos, mass) as sim:
        for inp, o in zip(((pos, mass), (bad, mass), (pos, mass)), outs):
            sim.set_particles_async(*inp)
            sim.step(2)
            sim.masses_async(o)
        try:
            sim.sync()
        except mtpt.MtptError as e:
            assert e.code == mtpt.MTPT_ERR_OUT_OF_DOMAIN
        else:
            raise AssertionError("the rejected load was not reported")
    for k, o in enumerate(outs):
        out[f"async_{k}_m"] = o
    # a batch of uneven realisations, both forms
    e = workloads.ensemble(nreal=16)
    members = sorted(e.members, key=lambda m: m.n)[:5]
    states = [workloads.initial_state(m) for m in members]
    pos = np.concatenate([s[0] for s in states], axis=1)
    mass = np.concatenate([s[1] for s in states])
    for fk, form in forms.items():
        with mtpt.Batch([_params(m, form) for m in members], [m.n for m in members],
                        pos, mass) as b:
            b.step(5)                       # graph replay included
            out[f"batch_{fk}_m"] = b.masses()
            out[f"batch_{fk}_x"] = b.positions()
    # boxes far from the origin (binary32 and binary64 cell indices)
    rng = np.random.default_rng(5)
    for tag, lo in (("f32cells", (4800.0, -5000.0)), ("f64cells", (2.0e6, -3.5e6))):
        L = np.array([45.0, 38.0])
        p = rng.uniform(0, 1, size=(2, 3000)) * L[:, None] + np.array(lo)[:, None]
        prm = mtpt.Params(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=lo, hi=tuple(np.array(lo) + L),
                          seed=9, precision=mtpt.MTPT_FP32W)
        with mtpt.Simulation(prm, p, rng.uniform(0, 1, 3000)) as sim:
            sim.step(3)
            out[f"far_{tag}_m"] = sim.masses()
    # adjoint
    w = workloads.get("uniform_mass_2d", 3000)
    pos, mass = workloads.initial_state(w)
    h = mtpt.mtpt_create(_params(w, mtpt.MTPT_FP64))
    try:
        mtpt.mtpt_set_particles(h, 2, pos, mass)
        mtpt.mtpt_adjoint_forward(h, 6, 3)
        g = torch.ones(w.n, dtype=torch.float64, device="cuda")
        g0 = torch.empty_like(g)
        out["adjoint_dldD"] = np.array([mtpt.mtpt_adjoint_backward(h, g, g0)])
        out["adjoint_g0"] = g0.cpu().numpy()
    finally:
        mtpt.mtpt_destroy(h)
    # the no-allocation step
    lib = mtpt.load()
    lib.mtpt_step_noalloc.argtypes = [ctypes.POINTER(mtpt._Params), ctypes.c_int64,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
    w = workloads.get("heaviside_2d", 10_000)
    pos, mass = workloads.initial_state(w)
    cp = _params(w, mtpt.MTPT_FP32W).c()
    pt = torch.from_numpy(pos.copy()).cuda()
    mt = torch.from_numpy(mass.copy()).cuda()
    for call in range(2):
        rc = lib.mtpt_step_noalloc(ctypes.byref(cp), w.n, call, pt.data_ptr(), mt.data_ptr(),
                                   None)
        assert rc == mtpt.MTPT_OK, mtpt.status_string(rc)
    torch.cuda.synchronize()
    out["noalloc_m"] = mt.cpu().numpy()
    out["noalloc_x"] = pt.cpu().numpy()
    return out


def main(path: str) -> None:
    import torch
    torch.cuda.set_device(0)
    mtpt.load()
    mtpt.mtpt_check_word(reset=True)
    res = run()
    res["check_word"] = np.array([mtpt.mtpt_check_word()], dtype=np.uint32)
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
