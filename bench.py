#!/usr/bin/env python
"""Throughput of the MTPT time step on GB300: particle-steps/s and
pair-interactions/s, binary64 form and precision form.

Workload (default): the 2-d diffusion at scale -- N = 4,000,000 particles
uniform in [0,2000]^2 (density 1), Gaussian point-source mass (sigma 5 at the
centre), D = 1, kappa = 0.5, dt = 0.1, lambda = 3.  A "step" is one full time
step of the hot path (walk, cell-list build, row sums, exchange) over every
particle.  Inputs are resident in HBM when the timed region starts; the
per-step working set (state double buffer, cell list, row sums) is several
times the 129 MB L2.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent realisation (seed + rank) on its
own GPU: no data-path collective ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2204_03756_gb300 import mtpt, workloads  # noqa: E402

FORMS = {"fp64": mtpt.MTPT_FP64, "fp32w": mtpt.MTPT_FP32W}
# arithmetic of each form: binary64 throughout; or binary32 kernel and
# weights with compensated binary32 row and flux sums and a binary64 mass update
DTYPE = {"fp64": "f64", "fp32w": "f32 weights, compensated f32 sums, f64 update"}
# timed single-run forms: precision form on the --workload workload, or on
# the 3-d workload for the "_3d" forms
FORM_WORKLOAD = {"fp32w": None, "fp64": None, "fp32w_3d": "heaviside_3d", "fp64_3d": "heaviside_3d",
                 "fp32w_adv": "advection_2d", "fp64_adv": "advection_2d",
                 "fp32w_react": "reaction_2d", "fp64_react": "reaction_2d"}


def _base(form: str) -> str:
    return form.split("_")[0]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def _algo_bytes_per_particle(kernel: str, dim: int, form: str) -> float:
    """Bytes the kernel's own arithmetic must read and write once per particle
    (its inputs and outputs; cell-list traffic excluded)."""
    x = 8 * dim
    r = 8 if _base(form) == "fp64" else 4
    table = {
        "walk_key": 2 * x,                 # positions read + written
        "rowsum_f64": x + r, "rowsum_f32": x + r,          # positions in, r out
        "exchange_f64": x + 8 + r + 8, "exchange_f32": x + 8 + r + 8,  # X, M, r in; M out
        # pass 2 and the next step's walk (walk-ahead): both kernels' bytes
        "exchange_walk_f32": x + 8 + r + 8 + 2 * x,
        "gather": 2 * (x + 8 + 4),         # state copied into cell order
        "scatter": 8, "scan": 0,
    }
    return float(table.get(kernel, 0))


# DRAM bytes per particle of each kernel from one-kernel ncu captures of the
# bench's own launch (profiles/step_kernels_gaussian_2d_4M.md: gaussian_2d,
# 4e6 particles, precision form, one launch per capture after three steps).
# Valid only for the library source it was measured on: a different hash of
# the CUDA sources and the header reports traffic as null.
TRAFFIC_DIM = 2
TRAFFIC_SOURCE_SHA1 = "fd2803d8f07e"
TRAFFIC_BYTES_PER_PARTICLE = {
    "walk_key": (88933632 + 31892736) / 4e6,
    "scatter": (81824512 + 34699776) / 4e6,
    "gather": (152929792 + 124269312) / 4e6,
    "rowsum_f32": (238171904 + 292427776) / 4e6,
    "exchange_f32": (389639424 + 26841344) / 4e6,
    "exchange_walk_f32": (478508544 + 117244416) / 4e6,
}


# Warp instructions per particle of the same captures
# (smsp__inst_executed.sum / 4e6): with the live launch time they give the
# issue rate, against the issue peak of 4 warp instructions per clock per SM
# (one per scheduler).
INSTR_PER_PARTICLE = {
    "walk_key": 43906125 / 4e6,
    "scatter": 4125000 / 4e6,
    "gather": 38024198 / 4e6,
    "rowsum_f32": 178884629 / 4e6,
    "exchange_f32": 49384081 / 4e6,
    "exchange_walk_f32": 93525743 / 4e6,
}
SMS, SCHEDULERS_PER_SM = 152, 4


# What bounds each kernel in those captures (ncu counters; see
# profiles/step_kernels_gaussian_2d_4M.md), reported beside the roofline
# while the kernel source hash matches.
BINDING = {
    "exchange_f32": ("DRAM 58 % with long-scoreboard stalls on the list reads and the "
                     "neighbour-record gathers; issue 46 % at 21 of 32 active lanes"),
    "exchange_walk_f32": ("DRAM 59 % and binary64 pipe 52 % (pass 2's update and the next "
                          "step's x + sigma xi); issue 61 % at 26 of 32 active lanes"),
    "rowsum_f32": "instruction issue: 72 % of issue slots at 18 of 32 active lanes; DRAM 32 %",
    "rowsum_f64": "binary64 pipe 86 % busy",
    "exchange_f64": "binary64 pipe 86 % busy",
    "gather": "DRAM 62 % (payload reads through the permutation, cell-ordered writes)",
    "scatter": "DRAM 42 % at 10 % issue (slot atomics, permutation and sort-key stores)",
    "walk_key": "binary64 pipe 80 % busy (x + sigma xi)",
}


def _kernel_source_sha1() -> str:
    """Hash of everything that shapes a kernel launch: every file of the CUDA
    sources (kernels and the host code that configures their launches) and
    the C header."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2204_03756_gb300", "csrc")
    paths = [os.path.join(csrc, f) for f in sorted(os.listdir(csrc))]
    paths.append(os.path.join(ROOT, "include", "mtpt.h"))
    h = hashlib.sha1()
    for path in paths:
        with open(path, "rb") as f:
            h.update(os.path.basename(path).encode() + b"\0" + f.read())
    return h.hexdigest()[:12]


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _params(w, form: str, rank: int) -> mtpt.Params:
    return mtpt.Params(dim=w.dim, D=w.D, kappa=w.kappa, dt=w.dt, beta=w.beta, lam=w.lam,
                       lo=w.lo, hi=w.hi, seed=w.seed + rank, precision=FORMS[_base(form)],
                       v=w.v)


def workload_config(w, form: str, world: int) -> dict:
    """The `config` object of both arms' JSON lines."""
    return {"workload": w.name, "n": w.n, "dim": w.dim, "box": list(w.hi),
            "D": w.D, "kappa": w.kappa, "dt": w.dt, "lambda": w.lam,
            "form": form, "steps_in_config": w.steps,
            "l2": "inputs larger than L2 (per-step working set > 300 MB)",
            "parallelism": f"replicas{world}" if world > 1 else "single"}


def reduce_over_ranks(ms: float, pairs: float, dist, device: str = "cuda"):
    """Whole-job timing of replicas: the slowest rank's time and the sum of
    every rank's neighbour pairs (each rank steps its own realisation)."""
    if dist is None:
        return ms, pairs
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    pt = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(pt, op=dist.ReduceOp.SUM)
    return float(t.item()), float(pt.item())


def job_throughput(n_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Particle-steps per second of the whole job (all ranks' particles over
    the slowest rank's time)."""
    return n_per_rank * steps * world / (max_ms / 1e3)


def _conserved(h, w) -> float:
    """The total the step conserves: the mass, or with A + B -> 0 the
    difference of the species' masses."""
    m = mtpt.mtpt_get_masses(h, w.n)
    if w.react_k > 0.0:
        return float((m - mtpt.mtpt_get_masses_b(h, w.n)).sum())
    return float(m.sum())


def time_form(w, pos, mass, form, steps, warmup, rank, world, dist, autotune_steps=4):
    import torch
    p = _params(w, form, rank)
    stream = torch.cuda.Stream()
    h = mtpt.mtpt_create(p)
    try:
        mtpt.mtpt_set_stream(h, stream.cuda_stream)
        mtpt.mtpt_set_particles(h, w.dim, pos, mass)
        if w.react_k > 0.0:                 # A + B -> 0: species B from the workload
            mtpt.mtpt_set_reaction(h, w.react_k)
            mtpt.mtpt_set_masses_b(h, workloads.masses_b(w, pos))
        # the autotuner's pick (cell width x pair block), restored state after
        # it; without trial steps the default tuning
        tuning = (mtpt.mtpt_autotune(h, autotune_steps) if autotune_steps > 0
                  else mtpt.mtpt_get_tuning(h))
        mtpt.mtpt_step(h, warmup)
        mtpt.mtpt_sync(h)
        m_before = _conserved(h, w)
        pairs0 = mtpt.mtpt_get_info(h)["pair_count"]
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        time.sleep(0.3)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mtpt.mtpt_step(h, steps)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        info = mtpt.mtpt_get_info(h)
        pairs = info["pair_count"] - pairs0
        m_after = _conserved(h, w)
        # second pass with per-kernel events (same stream, same workload)
        mtpt.mtpt_timing_reset(h)
        mtpt.mtpt_timing_enable(h, True)
        mtpt.mtpt_step(h, steps)
        kstats = mtpt.mtpt_timing_read(h)
        mtpt.mtpt_timing_enable(h, False)
    finally:
        mtpt.mtpt_destroy(h)
    max_ms, pairs = reduce_over_ranks(ms, pairs, dist)
    sec = max_ms / 1e3
    return {
        "form": form, "workload": w.name, "n": w.n, "ms": max_ms, "ms_per_step": max_ms / steps,
        "particle_steps_per_s": job_throughput(w.n, steps, world, max_ms),
        "pair_interactions_per_s": pairs / sec,
        "pairs_per_particle_step": pairs / (w.n * steps * world),
        "mass_drift_rel": abs(m_after - m_before) / abs(m_before),
        "clocks": clocks, "kernels": kstats, "launches_per_step":
            sum(v[0] for v in kstats.values()) / steps, "tuning": tuning,
    }


def time_split(w, pos, mass, form, steps, warmup, rank, world, dist, e2e_steps):
    """One domain cut into a checkerboard of `world` tiles (Secs. 4-5), one
    tile per rank: every step walks each tile's natives, exchanges the
    migrating particles and the 2 psi ghost pads with one all-to-all (NCCL
    on device buffers) and runs the mass transfer.  The whole job processes
    the workload's n particles per step whatever the number of ranks
    ("scaling": "strong").  `e2e` loads the tile's natives from pinned host
    memory before every step and reads its masses back after it."""
    import torch
    from paper_2204_03756_gb300 import ddc
    p = _params(w, form, 0)
    tiles = mtpt.mtpt_tiling_factors(w.dim, w.lo, w.hi, world)
    mine = ddc.tile_of(pos, w.lo, w.hi, tiles) == rank
    ids = np.flatnonzero(mine).astype(np.uint32)
    my_pos, my_mass = np.ascontiguousarray(pos[:, mine]), np.ascontiguousarray(mass[mine])

    class _One:                            # a single rank: no exchange partner
        def get_rank(self): return 0
        def get_world_size(self): return 1
        def get_backend(self): return "nccl"
        def all_to_all_single(self, out, inp, out_split=None, in_split=None): out.copy_(inp)
    group = dist if dist is not None else _One()
    sd = ddc.Subdomain(p, w.n, my_pos, my_mass, ids, group, tiles)
    stream = torch.cuda.current_stream()
    try:
        sd.step(warmup)
        torch.cuda.synchronize()
        pairs0 = sd.info()["pair_count"]
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        time.sleep(0.3)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sd.step(steps)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        pairs = sd.info()["pair_count"] - pairs0
        # second pass with per-kernel events: the launches of a step
        mtpt.mtpt_timing_reset(sd.h)
        mtpt.mtpt_timing_enable(sd.h, True)
        sd.step(steps)
        kstats = mtpt.mtpt_timing_read(sd.h)
        mtpt.mtpt_timing_enable(sd.h, False)
        # end to end: natives in from pinned host memory, one step, masses out
        lib = mtpt.load()
        pin_pos = torch.from_numpy(my_pos).pin_memory()
        pin_mass = torch.from_numpy(my_mass).pin_memory()
        pin_ids = torch.from_numpy(ids.view(np.int32)).pin_memory()
        out = torch.empty(max(1, 2 * len(ids)), dtype=torch.float64).pin_memory()
        h2d = d2h = 0

        def e2e_step():
            nonlocal h2d, d2h
            rc = lib.mtpt_set_particles_tile(sd.h, len(ids), pin_pos.data_ptr(),
                                             pin_mass.data_ptr(), pin_ids.data_ptr())
            if rc:
                raise mtpt.MtptError(rc, "mtpt_set_particles_tile")
            sd.step(1)
            n_now = sd.info()["n"]
            if n_now > out.numel():
                raise RuntimeError("e2e output buffer too small")
            rc = lib.mtpt_get_masses(sd.h, out.data_ptr())
            if rc:
                raise mtpt.MtptError(rc, "mtpt_get_masses")
            h2d += pin_pos.numel() * 8 + pin_mass.numel() * 8 + pin_ids.numel() * 4
            d2h += n_now * 8

        for _ in range(3):
            e2e_step()
        h2d = d2h = 0
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3
    finally:
        sd.close()
    max_ms, pairs_all = reduce_over_ranks(ms, pairs, dist)
    e2e_max, _ = reduce_over_ranks(e2e_ms, 0.0, dist)
    io, _ = reduce_over_ranks(0.0, float(h2d + d2h), dist)
    sec = max_ms / 1e3
    return {
        "form": form, "workload": w.name, "n": w.n, "ms": max_ms, "ms_per_step": max_ms / steps,
        "particle_steps_per_s": w.n * steps / sec,
        "pair_interactions_per_s": pairs_all / sec,
        "pairs_per_particle_step": pairs_all / (w.n * steps), "clocks": clocks,
        "tiles": list(tiles), "kernels": kstats,
        "launches_per_step": sum(v[0] for v in kstats.values()) / steps,
        "e2e": {"value": w.n * e2e_steps / (e2e_max / 1e3), "unit": "particle-steps/s",
                "ms_per_step": e2e_max / e2e_steps, "steps": e2e_steps,
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "api": "mtpt_set_particles_tile + tile step + mtpt_get_masses per step"},
    }


def time_batched(steps, warmup, rank, world, dist, nreal=512, autotune_steps=4):
    """The ensemble workload (independent 2-d realisations with uneven counts,
    densities and D) in the precision form, one launch per kernel per step
    over all realisations, autotuned, multi-step calls replayed as a CUDA
    graph."""
    import torch
    e = workloads.ensemble(nreal=nreal)
    pos, mass = workloads.ensemble_state(e)
    params = [mtpt.Params(dim=w.dim, D=w.D, kappa=w.kappa, dt=w.dt, beta=w.beta, lam=w.lam,
                          lo=w.lo, hi=w.hi, seed=w.seed + 7919 * rank,
                          precision=mtpt.MTPT_FP32W) for w in e.members]
    stream = torch.cuda.Stream()
    h = mtpt.mtpt_create_batch(params)
    total = int(e.counts.sum())
    try:
        mtpt.mtpt_set_stream(h, stream.cuda_stream)
        mtpt.mtpt_set_particles_batch(h, 2, e.counts, pos, mass)
        tuning = (mtpt.mtpt_autotune(h, autotune_steps) if autotune_steps > 0
                  else mtpt.mtpt_get_tuning(h))
        mtpt.mtpt_step(h, warmup)
        mtpt.mtpt_sync(h)
        pairs0 = mtpt.mtpt_get_info(h)["pair_count"]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mtpt.mtpt_step(h, steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pairs = mtpt.mtpt_get_info(h)["pair_count"] - pairs0
        mtpt.mtpt_timing_reset(h)
        mtpt.mtpt_timing_enable(h, True)
        mtpt.mtpt_step(h, steps)
        kstats = mtpt.mtpt_timing_read(h)
        mtpt.mtpt_timing_enable(h, False)
    finally:
        mtpt.mtpt_destroy(h)
    max_ms, pairs_all = reduce_over_ranks(ms, pairs, dist)
    sec = max_ms / 1e3
    return {"form": "batched", "precision": "fp32w", "realisations": nreal,
            "particles": total, "ms": max_ms, "ms_per_step": max_ms / steps,
            "particle_steps_per_s": job_throughput(total, steps, world, max_ms),
            "pair_interactions_per_s": pairs_all / sec,
            "pairs_per_particle_step": pairs / (total * steps),
            "tuning": tuning, "kernels": kstats,
            "launches_per_step": sum(v[0] for v in kstats.values()) / steps,
            "graph": "two-step CUDA graph replayed for the timed steps"}


def time_adjoint(rank, nbins=(100, 100), checkpoint_every=20):
    """The differentiable workload (250,000 particles in [0,500]^2, masses
    U(0,1), D = 0.5, dt = 0.1, 200 steps): forward run with checkpoints every
    20 steps in the precision form, then the adjoint sweep (binary64 adjoint
    passes) for the gradient of the 100 x 100 binned-concentration misfit
    against a seeded target with respect to the initial masses and D.  One
    gradient evaluation warms the handle up (its first forward run allocates
    the checkpoint store); the second is timed."""
    import torch
    from paper_2204_03756_gb300.autograd import binned_concentration
    w = workloads.get("uniform_mass_2d")
    pos, mass = workloads.initial_state(w)
    p = mtpt.Params(dim=w.dim, D=w.D, kappa=w.kappa, dt=w.dt, beta=w.beta, lam=w.lam,
                    lo=w.lo, hi=w.hi, seed=w.seed + rank, precision=mtpt.MTPT_FP32W)
    target = torch.from_numpy(workloads.target_field(nbins, w.lo, w.hi)).cuda()
    h = mtpt.mtpt_create(p)

    def gradient():
        mtpt.mtpt_set_particles(h, w.dim, pos, mass)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mtpt.mtpt_adjoint_forward(h, w.steps, checkpoint_every)
        t1 = time.perf_counter()
        mT = torch.empty(w.n, dtype=torch.float64, device="cuda")
        xT = torch.empty(w.dim * w.n, dtype=torch.float64, device="cuda")
        mtpt.mtpt_get_masses_device(h, mT)
        mtpt.mtpt_get_positions_device(h, xT)
        mtpt.mtpt_sync(h)
        mT.requires_grad_(True)
        C = binned_concentration(xT.view(w.dim, w.n), mT, w.lo, w.hi, nbins)
        loss = ((C - target) ** 2).sum()
        loss.backward()
        g = mT.grad.contiguous()
        g0 = torch.empty_like(g)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        dldD = mtpt.mtpt_adjoint_backward(h, g, g0)
        t3 = time.perf_counter()
        return t1 - t0, t3 - t2, loss, dldD, g0

    try:
        gradient()
        fwd, bwd, loss, dldD, g0 = gradient()
    finally:
        mtpt.mtpt_destroy(h)
    return {"form": "adjoint", "workload": "uniform_mass_2d", "n": w.n, "steps": w.steps,
            "checkpoint_every": checkpoint_every, "forward_s": fwd, "backward_s": bwd,
            "gradient_particle_steps_per_s": w.n * w.steps / (fwd + bwd),
            "loss": float(loss.item()), "dL_dD": dldD,
            "dL_dM0_norm": float(g0.norm().item()), "warmup_gradients": 1,
            "precision": "forward fp32w, adjoint passes f64"}


# binary64 instructions per accepted ordered pair of the binary64 pair passes:
# rowsum -- squared distance 2d (a difference and a multiply or fma per axis),
# the kernel exponential 7 (2 fma reduction, 4 fma polynomial, 1 table
# multiply; the reduction index and the 2^-q scaling are integer/binary32),
# the row-sum add 1; exchange (kernel values read back from the neighbour
# lists) -- r_i + r_j 1, the quotient 5 (Newton step 2, product 1,
# correction 2), the mass difference, the product and the flux add 3.
def _f64_ops_per_pair(kernel: str, dim: int) -> float:
    return {"rowsum_f64": 2 * dim + 7 + 1, "exchange_f64": 1 + 5 + 3}[kernel]


# GB300 binary64 issue rate: 2 binary64 operations per clock per SM (recipe's
# 1.25 TFLOP/s counts an fma as two) x 152 SMs x 2.07 GHz
F64_PEAK_OPS = 2 * 152 * 2.07e9


def issue_rate(name, w, per_launch_s, clocks):
    """Warp instructions issued per second by one launch of `name` (from the
    captured count per particle) against the issue peak at the SM clock the
    timed region ran at; None when the capture does not apply."""
    if name not in INSTR_PER_PARTICLE or w.dim != TRAFFIC_DIM or \
            _kernel_source_sha1() != TRAFFIC_SOURCE_SHA1:
        return None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    achieved = INSTR_PER_PARTICLE[name] * w.n / per_launch_s
    peak = SMS * SCHEDULERS_PER_SM * mhz * 1e6
    return {"achieved": achieved, "peak": peak, "unit": "warp instr/s", "frac": achieved / peak,
            "instr_per_launch": INSTR_PER_PARTICLE[name] * w.n,
            "peak_source": f"{SMS} SMs x {SCHEDULERS_PER_SM} schedulers x {mhz:.0f} MHz"}


def roofline(w, res, peaks):
    kst = res["kernels"]
    name, (launches, total_ms) = max(kst.items(), key=lambda kv: kv[1][1])
    per_launch_s = total_ms / launches / 1e3
    share = total_ms / sum(v[1] for v in kst.values())
    current = w.dim == TRAFFIC_DIM and _kernel_source_sha1() == TRAFFIC_SOURCE_SHA1
    binding = BINDING.get(name) if current else None
    if name in ("rowsum_f64", "exchange_f64"):
        pairs = res["pairs_per_particle_step"] * w.n
        ops = _f64_ops_per_pair(name, w.dim) * pairs
        achieved = ops / per_launch_s / 1e9
        return {"bound": "alu", "kernel": name, "achieved": achieved,
                "peak": F64_PEAK_OPS / 1e9, "unit": "G binary64 op/s",
                "frac": achieved / (F64_PEAK_OPS / 1e9), "traffic": None,
                "algorithmic_ops_per_launch": ops, "launch_ms": per_launch_s * 1e3,
                "share_of_step": share, "binding_ncu": binding,
                "peak_source": "derived: 2 binary64 ops/clk/SM x 152 SMs x 2.07 GHz"}
    algo = _algo_bytes_per_particle(name, w.dim, res["form"]) * w.n
    achieved = algo / per_launch_s / 1e9
    traffic = None
    if name in TRAFFIC_BYTES_PER_PARTICLE and current:
        traffic = TRAFFIC_BYTES_PER_PARTICLE[name] * w.n
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "algorithmic_bytes_per_launch": algo, "launch_ms": per_launch_s * 1e3,
            "share_of_step": share, "binding_ncu": binding, "peak_source": peaks["source"],
            "issue": issue_rate(name, w, per_launch_s, res.get("clocks"))}


def e2e_form(w, pos, mass, form, steps, rank, world=1, dist=None):
    """Through the C ABI with HOST buffers: every step uploads the state from
    pinned host memory, advances one time step and reads the masses back into
    pinned host memory.  `value` uses the pipelined calls
    (mtpt_set_particles_async / mtpt_get_masses_async: the copies of one step
    overlap the device work of another; one mtpt_sync after the last step);
    `sync_calls` the synchronous mtpt_set_particles / mtpt_get_masses, which
    wait for each copy.  Each is the median of three timed runs."""
    import torch
    p = _params(w, form, rank)
    pin_pos = torch.from_numpy(np.ascontiguousarray(pos)).pin_memory()
    pin_mass = torch.from_numpy(np.ascontiguousarray(mass)).pin_memory()
    out = torch.empty(w.n, dtype=torch.float64).pin_memory()
    h = mtpt.mtpt_create(p)
    lib = mtpt.load()

    def pipelined(k):
        for _ in range(k):
            rc = lib.mtpt_set_particles_async(h, w.n, pin_pos.data_ptr(), pin_mass.data_ptr())
            rc = rc or lib.mtpt_step(h, 1)
            rc = rc or lib.mtpt_get_masses_async(h, out.data_ptr())
            if rc:
                raise mtpt.MtptError(rc, "e2e pipelined step")
        rc = lib.mtpt_sync(h)
        if rc:
            raise mtpt.MtptError(rc, "e2e sync")

    def synchronous(k):
        for _ in range(k):
            rc = lib.mtpt_set_particles(h, w.n, pin_pos.data_ptr(), pin_mass.data_ptr())
            rc = rc or lib.mtpt_step(h, 1)
            rc = rc or lib.mtpt_get_masses(h, out.data_ptr())
            if rc:
                raise mtpt.MtptError(rc, "e2e step")

    def timed(fn):
        fn(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn(steps)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # three timed runs of `steps` steps each, the median reported: the
    # pipelined loop issues some twenty host calls per step, so a stall of the
    # host thread shows in one run rather than in the figure
    try:
        synchronous(1)
        secs_sync = [timed(synchronous) for _ in range(3)]
        secs = [timed(pipelined) for _ in range(3)]
    finally:
        mtpt.mtpt_destroy(h)
    sec, sec_sync = statistics.median(secs), statistics.median(secs_sync)
    # whole job: every rank's particles over the slowest rank's time
    ms, _ = reduce_over_ranks(sec * 1e3, 0.0, dist)
    ms_sync, _ = reduce_over_ranks(sec_sync * 1e3, 0.0, dist)
    return {"value": job_throughput(w.n, steps, world, ms), "unit": "particle-steps/s",
            "h2d_bytes_per_step": int(pos.nbytes + mass.nbytes) * world,
            "d2h_bytes_per_step": int(w.n * 8) * world, "steps": steps,
            "ms_per_step": ms / steps, "api": "pipelined",
            "runs_ms_per_step": [t * 1e3 / steps for t in secs],
            "sync_calls": {"value": job_throughput(w.n, steps, world, ms_sync),
                           "ms_per_step": ms_sync / steps,
                           "runs_ms_per_step": [t * 1e3 / steps for t in secs_sync]}}


def _step_errors(p, pos, mass, steps, x_ref, m_ref, npairs):
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(steps)
        x, m, info = sim.positions(), sim.masses(), sim.info()
    return {"max_rel_err_vs_oracle": float(np.abs(m - m_ref).max() / np.abs(m_ref).max()),
            "positions_bit_exact": bool(np.array_equal(x, x_ref)),
            "pair_count_equal": bool(info["pair_count"] == npairs)}


def _reactive_errors(p, k, pos, ma, mb, x_ref, a_ref, b_ref, npairs):
    """One reactive step against the oracle: both species, error relative to
    the largest reference mass of either."""
    with mtpt.Simulation(p, pos, ma) as sim:
        sim.set_reaction(k, mb)
        sim.step(1)
        x, a, b, info = sim.positions(), sim.masses(), sim.masses_b(), sim.info()
    scale = max(np.abs(a_ref).max(), np.abs(b_ref).max())
    err = max(np.abs(a - a_ref).max(), np.abs(b - b_ref).max()) / scale
    return {"max_rel_err_vs_oracle": float(err),
            "positions_bit_exact": bool(np.array_equal(x, x_ref)),
            "pair_count_equal": bool(info["pair_count"] == npairs)}


def _oracle_params(O, p):
    return O.OracleParams(dim=p.dim, D=p.D, kappa=p.kappa, dt=p.dt, beta=p.beta, lam=p.lam,
                          lo=tuple(p.lo) + (0.0,) * (3 - p.dim),
                          hi=tuple(p.hi) + (0.0,) * (3 - p.dim), seed=p.seed,
                          v=tuple(p.v)[:3] + (0.0,) * (3 - len(tuple(p.v)[:3])))


def cpu_baseline(w, pos, mass, forms, batched=False, adjoint=False):
    """The CPU oracle timed on one core over one full time step of the whole
    workload.  The same leg reports every form's error against the oracle:
    the forms on that workload on that full step, the forms on other
    workloads (3-d, advection) on one step of theirs at 200,000 particles, the batched kernels on two steps of four
    ensemble realisations spanning the count range (batched together, each
    compared with its own oracle run), and the adjoint's dL/dM_0 against the
    oracle's reverse sweep on 20,000 particles over 10 steps."""
    import oracle as O
    t0 = time.perf_counter()
    op = _oracle_params(O, _params(w, forms[0], 0))
    x_ref, m_ref, npairs = O.run(op, pos, mass, 1)
    sec = time.perf_counter() - t0
    parity = {}
    for f in forms:
        if FORM_WORKLOAD.get(f) is None:
            parity[f] = dict(_step_errors(_params(w, f, 0), pos, mass, 1, x_ref, m_ref, npairs),
                             case=f"{w.name}, n={w.n}, 1 step")
    others = sorted({FORM_WORKLOAD[f] for f in forms if FORM_WORKLOAD.get(f) is not None})
    for name in others:
        fs = [f for f in forms if FORM_WORKLOAD.get(f) == name]
        wk = workloads.get(name, 200_000)
        pk, mk = workloads.initial_state(wk)
        if wk.react_k > 0.0:
            mb = workloads.masses_b(wk, pk)
            xr, ar, br, nr = O.run_reactive(_oracle_params(O, _params(wk, fs[0], 0)), pk, mk, mb,
                                            1, wk.react_k)
            for f in fs:
                parity[f] = dict(_reactive_errors(_params(wk, f, 0), wk.react_k, pk, mk, mb,
                                                  xr, ar, br, nr),
                                 case=f"{name}, n={wk.n}, 1 step, both species")
            continue
        xr, mr, nr = O.run(_oracle_params(O, _params(wk, fs[0], 0)), pk, mk, 1)
        for f in fs:
            parity[f] = dict(_step_errors(_params(wk, f, 0), pk, mk, 1, xr, mr, nr),
                             case=f"{name}, n={wk.n}, 1 step")
    if batched:
        e = workloads.ensemble()
        order = np.argsort(e.counts)
        pick = [int(order[k]) for k in (0, len(order) // 3, 2 * len(order) // 3, len(order) - 1)]
        members = [e.members[k] for k in pick]
        states = [workloads.initial_state(m) for m in members]
        params = [_params(m, "fp32w", 0) for m in members]
        with mtpt.Batch(params, [m.n for m in members],
                        np.concatenate([st[0] for st in states], axis=1),
                        np.concatenate([st[1] for st in states])) as bt:
            bt.step(2)
            bx, bm = bt.split(bt.positions()), bt.split(bt.masses())
        errs, exact = [], True
        for k, (m, st) in enumerate(zip(members, states)):
            xr, mr, _ = O.run(_oracle_params(O, params[k]), st[0], st[1], 2)
            errs.append(float(np.abs(bm[k] - mr).max() / np.abs(mr).max()))
            exact &= bool(np.array_equal(bx[k], xr))
        parity["batched"] = {"max_rel_err_vs_oracle": max(errs), "positions_bit_exact": exact,
                             "case": "2 steps of ensemble realisations with "
                                     f"{[m.n for m in members]} particles, batched together"}
    if adjoint:
        parity["adjoint"] = _adjoint_parity(O)
    return {"value": w.n / sec, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"one full time step of all {w.n} particles (serial C oracle, K-D tree)",
            "seconds": sec, "pair_interactions_per_s": npairs / sec, "parity": parity,
            "erf_check": _erf_check(O), "host": _host_info()}


# Arm CPU part numbers (MIDR) of the server cores this may run on
ARM_PARTS = {"0xd0c": "Neoverse-N1", "0xd40": "Neoverse-V1", "0xd49": "Neoverse-N2",
             "0xd4f": "Neoverse-V2", "0xd84": "Neoverse-V3"}


def _host_info():
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                key, val = key.strip().lower(), val.strip()
                if key == "model name":
                    model = val
                    break
                if key == "cpu part":
                    model = f"{ARM_PARTS.get(val, 'Arm')} (CPU part {val})"
                    break
    except OSError:
        pass
    return {"cpu_count": os.cpu_count(), "cpu": model, "machine": platform.machine()}


def _erf_check(O):
    """The small 2-d Heaviside case (1e4 particles, 100 steps, binary64): GPU
    and oracle runs against the closed-form erfc profile of pure diffusion
    (RMSE of the mean particle mass in 50 slabs of x), and against each
    other."""
    from oracle import analytic as A
    w = workloads.get("heaviside_2d")
    pos, mass = workloads.initial_state(w)
    p = _params(w, "fp64", 0)
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(w.steps)
        xg, mg = sim.positions(), sim.masses()
    xr, mr, _ = O.run(_oracle_params(O, p), pos, mass, w.steps)
    t = w.steps * w.dt
    out = {"workload": w.name, "n": w.n, "steps": w.steps}
    for name, (x, m) in (("gpu", (xg, mg)), ("oracle", (xr, mr))):
        c, mean, _ = A.binned_profile(x[0], m, w.lo[0], w.hi[0], 50)
        out[f"rmse_{name}_vs_erf"] = A.rmse(mean, A.erf_profile(c, t, w.D, w.mass_param, "left"))
    out["max_rel_err_gpu_vs_oracle"] = float(np.abs(mg - mr).max() / np.abs(mr).max())
    out["positions_bit_exact"] = bool(np.array_equal(xg, xr))
    return out


def _adjoint_parity(O, n=20_000, steps=10, nbins=(20, 20)):
    """dL/dM_0 of the binned misfit: GPU adjoint vs the oracle's transfer
    operator applied in reverse (it is symmetric) along the oracle's walk."""
    import torch
    w = workloads.get("uniform_mass_2d", n)
    pos, mass = workloads.initial_state(w)
    p = _params(w, "fp64", 0)
    op = _oracle_params(O, p)
    ids = np.arange(n, dtype=np.uint32)
    xs, x, m = [], pos, mass
    for t in range(steps):
        x = O.random_walk(op, x, ids, t)
        m = O.mass_transfer(op, x, m)[0]
        xs.append(x)
    target = workloads.target_field(nbins, w.lo, w.hi).ravel()
    ix = np.clip(((x[0] - w.lo[0]) / (w.hi[0] - w.lo[0]) * nbins[0]).astype(int), 0, nbins[0] - 1)
    iy = np.clip(((x[1] - w.lo[1]) / (w.hi[1] - w.lo[1]) * nbins[1]).astype(int), 0, nbins[1] - 1)
    b = ix * nbins[1] + iy
    area = (w.hi[0] - w.lo[0]) / nbins[0] * (w.hi[1] - w.lo[1]) / nbins[1]
    C = np.bincount(b, weights=m, minlength=nbins[0] * nbins[1]) / area
    g = 2.0 * (C - target)[b] / area
    lam = g.copy()
    for t in reversed(range(steps)):
        lam = O.mass_transfer(op, xs[t], lam)[0]
    h = mtpt.mtpt_create(p)
    try:
        mtpt.mtpt_set_particles(h, 2, pos, mass)
        mtpt.mtpt_adjoint_forward(h, steps, 4)
        gt = torch.from_numpy(g).cuda()
        g0 = torch.empty_like(gt)
        mtpt.mtpt_adjoint_backward(h, gt, g0)
    finally:
        mtpt.mtpt_destroy(h)
    got = g0.cpu().numpy()
    return {"max_rel_err_vs_oracle": float(np.abs(got - lam).max() / np.abs(lam).max()),
            "quantity": "dL/dM_0", "case": f"uniform_mass_2d, n={n}, {steps} steps"}


def reference_arm(args, w, pos, mass):
    """The oracle as the reference implementation: each step is one oracle
    time step of a bounded sample of the workload (a corner sub-box at the same
    density)."""
    import oracle as O
    n_sample = int(args.ref_sample)
    ws = w.scaled(n_sample)
    ps, ms = workloads.initial_state(ws)
    op = O.OracleParams(dim=ws.dim, D=ws.D, kappa=ws.kappa, dt=ws.dt, beta=ws.beta, lam=ws.lam,
                        lo=tuple(ws.lo) + (0.0,) * (3 - ws.dim),
                        hi=tuple(ws.hi) + (0.0,) * (3 - ws.dim), seed=ws.seed)
    x, m = ps, ms
    for s in range(args.warmup):
        x, m, _ = O.run(op, x, m, 1, step0=s)
    t0 = time.perf_counter()
    pairs = 0
    for s in range(args.steps):
        x, m, np_ = O.run(op, x, m, 1, step0=args.warmup + s)
        pairs += np_
    sec = time.perf_counter() - t0
    value = n_sample * args.steps / sec
    sample = (f"{n_sample} particles of the workload at its density (box "
              f"{ws.hi[0] - ws.lo[0]:.1f}^{ws.dim}), one oracle step per bench step")
    return {"impl": "reference", "metric": "particle-steps/s", "value": value,
            "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(w, args.forms.split(",")[0], 1),
            "pair_interactions_per_s": pairs / sec,
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def forms_summary(forms: dict) -> dict:
    """One compact entry per timed form (binary64, precision form, 3-d,
    advection, batched, adjoint): step time, throughput, error against the
    oracle and the dominant kernel's roofline fraction."""
    out = {}
    for f, r in forms.items():
        e = {}
        for k in ("ms_per_step", "particle_steps_per_s", "pair_interactions_per_s",
                  "gradient_particle_steps_per_s", "forward_s", "backward_s", "mass_drift_rel"):
            if r.get(k) is not None:
                e[k] = float(f"{r[k]:.4g}")
        err = (r.get("err_vs_oracle") or {}).get("max_rel_err_vs_oracle")
        if err is not None:
            e["err_vs_oracle"] = float(f"{err:.3g}")
        if r.get("tuning"):
            e["tuning"] = r["tuning"]
        rf = r.get("roofline")
        if rf:
            e["roofline"] = {"kernel": rf["kernel"], "bound": rf["bound"],
                             "frac": float(f"{rf['frac']:.3g}")}
        if f in FORMS or _base(f) in FORMS:
            e["dtype"] = DTYPE[_base(f)]
        out[f] = e
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gaussian_2d", choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--forms", default="fp32w,fp64,fp32w_3d,fp32w_adv,fp32w_react,batched,adjoint",
                    help="comma list; the first is the headline value")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--autotune-steps", type=int, default=4,
                    help="trial steps per tuning of the autotuner (0: default tuning, no trials)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=200_000)
    ap.add_argument("--n", type=int, default=None,
                    help="scale the workload to n particles at the same density "
                         "(profiling runs; the default is the workload's own size)")
    ap.add_argument("--split", default="auto", choices=["auto", "on", "off"],
                    help="one domain cut into one tile per rank (auto: with more than "
                         "one rank); off: independent replicas per rank")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world, rank, local = _dist()
    w = workloads.get(args.workload, args.n)

    if args.impl == "reference":
        if rank != 0:
            return 0
        pos, mass = workloads.initial_state(w)
        print(json.dumps(reference_arm(args, w, pos, mass)))
        return 0

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    mtpt.load()
    pos, mass = workloads.initial_state(w)
    forms = [f for f in args.forms.split(",") if f and f not in ("batched", "adjoint")]
    for f in forms:
        if f not in FORM_WORKLOAD:
            ap.error(f"unknown form {f!r}")
    if forms and FORM_WORKLOAD[forms[0]] is not None:
        ap.error("the first form (the headline) must run on --workload")
    states = {}

    def state_of(f):
        name = FORM_WORKLOAD[f]
        if name is None:
            return w, pos, mass
        if name not in states:
            wf = workloads.get(name)
            states[name] = (wf,) + tuple(workloads.initial_state(wf))
        return states[name]

    split = args.split == "on" or (args.split == "auto" and world > 1)
    if split:
        f = forms[0] if forms else "fp32w"
        r = time_split(w, pos, mass, f, args.steps, args.warmup, rank, world, dist,
                       args.e2e_steps)
        e2e = dict(r.pop("e2e"))
        line = {
            "metric": "particle-steps/s", "value": r["particle_steps_per_s"],
            "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": DTYPE[_base(f)], "data": "synthetic",
            "config": dict(workload_config(w, f, world),
                           parallelism=f"checkerboard {'x'.join(map(str, r['tiles']))}"),
            "pair_interactions_per_s": r["pair_interactions_per_s"],
            "gpu_launches": int(round(r["launches_per_step"] * args.steps)),
            "clocks": r.pop("clocks"), "e2e": e2e, "split": r,
        }
        # host copies per step of the whole job: every rank's natives in, masses out
        e2e["h2d_bytes_per_step"] = int(pos.nbytes + mass.nbytes + 4 * w.n)
        e2e["d2h_bytes_per_step"] = int(mass.nbytes)
        if rank == 0:
            print(json.dumps(line))
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    results = {}
    for f in forms:
        wf, pf, mf = state_of(f)
        results[f] = time_form(wf, pf, mf, f, args.steps, args.warmup, rank, world, dist,
                               args.autotune_steps)
    batched = None
    if "batched" in args.forms.split(","):
        batched = time_batched(args.steps, args.warmup, rank, world, dist,
                               autotune_steps=args.autotune_steps)
    adjoint = time_adjoint(rank) if "adjoint" in args.forms.split(",") else None
    peaks = _peaks()
    if not forms:                        # only batched / adjoint requested
        line = {"metric": "particle-steps/s", "unit": "particle-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE["fp32w"],
                "data": "synthetic", "forms": {}}
        if batched is not None:
            line.update(value=batched["particle_steps_per_s"], ms_per_step=batched["ms_per_step"],
                        config={"workload": "ensemble_2d", "realisations": batched["realisations"],
                                "n": batched["particles"]},
                        gpu_launches=int(round(batched["launches_per_step"] * args.steps)))
            line["forms"]["batched"] = batched
        if adjoint is not None:
            line["forms"]["adjoint"] = adjoint
        if rank == 0:
            print(json.dumps(line))
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    head = results[forms[0]]
    e2e = e2e_form(w, pos, mass, forms[0], args.e2e_steps, rank, world, dist)
    line = {
        "metric": "particle-steps/s", "value": head["particle_steps_per_s"],
        "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[_base(forms[0])], "data": "synthetic",
        "config": workload_config(w, forms[0], world),
        "pair_interactions_per_s": head["pair_interactions_per_s"],
        "pairs_per_particle_step": head["pairs_per_particle_step"],
        "mass_drift_rel": head["mass_drift_rel"],
        "gpu_launches": int(round(head["launches_per_step"] * args.steps)),
        "clocks": head["clocks"],
        "roofline": roofline(w, head, peaks),
        "e2e": e2e,
        "forms": {f: {k: v for k, v in r.items() if k not in ("clocks",)}
                  for f, r in results.items()},
    }
    for f, r in results.items():
        line["forms"][f]["roofline"] = roofline(state_of(f)[0], r, peaks)
    if batched is not None:
        line["forms"]["batched"] = batched
    if adjoint is not None:
        line["forms"]["adjoint"] = adjoint
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, pos, mass, forms, batched=batched is not None,
                                            adjoint=adjoint is not None)
        for f, err in line["cpu_baseline"]["parity"].items():
            line["forms"][f]["err_vs_oracle"] = err
    line["forms_summary"] = forms_summary(line["forms"])   # last key: the line's tail
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
