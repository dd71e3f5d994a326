"""Python binding of the C ABI in ``include/mtpt.h`` (argument marshalling only).

Every function keeps the C name.  Host arrays are numpy; device arrays are
torch CUDA tensors (PyTorch supplies device memory and the stream: the
``*_device`` calls run on ``torch.cuda.current_stream()``).  The binding
loads the in-tree ``_lib/libmtpt.so`` and raises if it is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MTPT_OK = 0
MTPT_ERR_INVALID_ARG = 1
MTPT_ERR_OUT_OF_DOMAIN = 2
MTPT_ERR_CUDA = 3
MTPT_ERR_NO_MEMORY = 4
MTPT_ERR_STATE = 5
MTPT_ERR_CAPACITY = 6
MTPT_ERR_TOO_LARGE = 7
NOALLOC_MAX_PARTICLES = 65536

MTPT_FP64 = 0
MTPT_FP32W = 1

MTPT_DO_WALK = 1
MTPT_DO_TRANSFER = 2

EXPORTED = [
    "mtpt_create", "mtpt_destroy", "mtpt_set_stream", "mtpt_set_particles",
    "mtpt_set_particles_device", "mtpt_step", "mtpt_step_ex", "mtpt_get_masses",
    "mtpt_get_masses_device", "mtpt_get_positions", "mtpt_get_positions_device",
    "mtpt_get_row_sums", "mtpt_get_pairs", "mtpt_get_info", "mtpt_set_step", "mtpt_sync",
    "mtpt_timing_enable", "mtpt_timing_read", "mtpt_timing_reset", "mtpt_step_noalloc",
    "mtpt_create_batch", "mtpt_set_particles_batch", "mtpt_get_realisation_info",
    "mtpt_set_tuning", "mtpt_get_tuning", "mtpt_autotune", "mtpt_adjoint_forward",
    "mtpt_adjoint_backward", "mtpt_status_string", "mtpt_check_word",
    "mtpt_set_particles_async", "mtpt_get_masses_async", "mtpt_tiling_factors",
    "mtpt_set_tiling", "mtpt_set_particles_tile", "mtpt_tile_pack", "mtpt_tile_transfer",
    "mtpt_get_ids", "mtpt_debug_fail_alloc", "mtpt_set_reaction", "mtpt_set_masses_b",
    "mtpt_get_masses_b", "mtpt_debug_scan_hold",
]


class MtptError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("D", ctypes.c_double), ("kappa", ctypes.c_double),
                ("dt", ctypes.c_double), ("beta", ctypes.c_double),
                ("lam", ctypes.c_double),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("seed", ctypes.c_uint64), ("v", ctypes.c_double * 3)]


class _KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class _Tuning(ctypes.Structure):
    _fields_ = [("cell_scale", ctypes.c_double), ("pair_block", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class _Tiling(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int32 * 3), ("tile", ctypes.c_int32),
                ("n_global", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("step", ctypes.c_uint64),
                ("pair_count", ctypes.c_uint64),
                ("D_RW", ctypes.c_double), ("D_MT", ctypes.c_double),
                ("sigma", ctypes.c_double), ("h2", ctypes.c_double),
                ("psi", ctypes.c_double), ("psi2", ctypes.c_double),
                ("kernel_norm", ctypes.c_double),
                ("cells", ctypes.c_int32 * 3), ("cell_width", ctypes.c_double * 3)]


@dataclass
class Params:
    """Sec. 2-3 parameters: dimension, D, kappa = D_RW / D, dt, beta, lambda
    (psi = lambda sqrt(4 D_MT dt / beta)), box [lo, hi] with reflecting walls,
    walk seed, precision form (MTPT_FP64 or MTPT_FP32W) and a uniform velocity
    v (advection; 0 in the paper's runs)."""
    dim: int = 2
    D: float = 1.0
    kappa: float = 0.5
    dt: float = 0.1
    beta: float = 1.0
    lam: float = 3.0
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    seed: int = 0
    precision: int = MTPT_FP64
    v: tuple = (0.0, 0.0, 0.0)

    def c(self) -> _Params:
        lo = list(self.lo)[:3] + [0.0] * (3 - min(3, len(self.lo)))
        hi = list(self.hi)[:3] + [0.0] * (3 - min(3, len(self.hi)))
        v = list(self.v)[:3] + [0.0] * (3 - min(3, len(self.v)))
        return _Params(self.dim, self.precision, self.D, self.kappa, self.dt, self.beta,
                       self.lam, (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi),
                       self.seed, (ctypes.c_double * 3)(*v))


_lib = None


def lib_path() -> str:
    """The library this process loads: the normal build, or the bounds-checked
    build when the environment sets MTPT_LIBRARY=checked."""
    if os.environ.get("MTPT_LIBRARY", "") == "checked":
        return _build.LIB_CHECKED_PATH
    return _build.LIB_PATH


def load():
    """Load the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.mtpt_create.argtypes = [P(_Params), P(vp)]
    lib.mtpt_destroy.argtypes = [vp]
    lib.mtpt_set_stream.argtypes = [vp, vp]
    lib.mtpt_set_particles.argtypes = [vp, ctypes.c_int64, vp, vp]
    lib.mtpt_set_particles_device.argtypes = [vp, ctypes.c_int64, vp, vp]
    lib.mtpt_set_particles_async.argtypes = [vp, ctypes.c_int64, vp, vp]
    lib.mtpt_get_masses_async.argtypes = [vp, vp]
    lib.mtpt_step.argtypes = [vp, ctypes.c_int64]
    lib.mtpt_step_ex.argtypes = [vp, ctypes.c_int64, ctypes.c_int32]
    for name in ("mtpt_get_masses", "mtpt_get_masses_device", "mtpt_get_positions",
                 "mtpt_get_positions_device", "mtpt_get_row_sums"):
        getattr(lib, name).argtypes = [vp, vp]
    lib.mtpt_get_pairs.argtypes = [vp, ctypes.c_int64, P(ctypes.c_int64), vp, vp]
    lib.mtpt_get_info.argtypes = [vp, P(_Info)]
    lib.mtpt_set_step.argtypes = [vp, ctypes.c_uint64]
    lib.mtpt_check_word.argtypes = [P(ctypes.c_uint32), ctypes.c_int32]
    lib.mtpt_sync.argtypes = [vp]
    lib.mtpt_timing_enable.argtypes = [vp, ctypes.c_int32]
    lib.mtpt_timing_read.argtypes = [vp, ctypes.c_int32, P(_KernelStat), P(ctypes.c_int32)]
    lib.mtpt_timing_reset.argtypes = [vp]
    lib.mtpt_adjoint_forward.argtypes = [vp, ctypes.c_int64, ctypes.c_int64]
    lib.mtpt_adjoint_backward.argtypes = [vp, vp, vp, P(ctypes.c_double)]
    lib.mtpt_set_tuning.argtypes = [vp, P(_Tuning)]
    lib.mtpt_get_tuning.argtypes = [vp, P(_Tuning)]
    lib.mtpt_autotune.argtypes = [vp, ctypes.c_int32, P(_Tuning)]
    lib.mtpt_create_batch.argtypes = [P(_Params), ctypes.c_int32, P(vp)]
    lib.mtpt_set_particles_batch.argtypes = [vp, P(ctypes.c_int64), vp, vp]
    lib.mtpt_get_realisation_info.argtypes = [vp, ctypes.c_int32, P(_Info)]
    lib.mtpt_step_noalloc.argtypes = [P(_Params), ctypes.c_int64, ctypes.c_uint64, vp, vp, vp]
    lib.mtpt_tiling_factors.argtypes = [ctypes.c_int32, vp, vp, ctypes.c_int32,
                                        P(ctypes.c_int32)]
    lib.mtpt_set_tiling.argtypes = [vp, P(_Tiling)]
    lib.mtpt_set_particles_tile.argtypes = [vp, ctypes.c_int64, vp, vp, vp]
    lib.mtpt_tile_pack.argtypes = [vp, ctypes.c_int64, vp, P(ctypes.c_int64)]
    lib.mtpt_tile_transfer.argtypes = [vp, ctypes.c_int64, vp]
    lib.mtpt_get_ids.argtypes = [vp, vp]
    lib.mtpt_debug_fail_alloc.argtypes = [ctypes.c_int64, P(ctypes.c_int64)]
    lib.mtpt_debug_scan_hold.argtypes = [ctypes.c_int32, P(ctypes.c_uint64)]
    lib.mtpt_set_reaction.argtypes = [vp, ctypes.c_double]
    lib.mtpt_set_masses_b.argtypes = [vp, vp]
    lib.mtpt_get_masses_b.argtypes = [vp, vp]
    lib.mtpt_status_string.argtypes = [ctypes.c_int]
    lib.mtpt_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "mtpt_status_string":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().mtpt_status_string(code).decode()


def _check(code: int, where: str):
    if code != MTPT_OK:
        raise MtptError(code, where)


def _host_f64(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _dev_ptr(t, dtype_name: str, numel: int) -> int:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}" or t.numel() != numel:
        raise ValueError(f"expected {numel} elements of {dtype_name}")
    return t.data_ptr()


def _torch_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


# --- the C entry points ------------------------------------------------------

def mtpt_create(params: Params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    cp = params.c()
    _check(load().mtpt_create(ctypes.byref(cp), ctypes.byref(h)), "mtpt_create")
    return h


def mtpt_create_batch(params_list) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    arr = (_Params * len(params_list))(*[p.c() for p in params_list])
    _check(load().mtpt_create_batch(arr, len(params_list), ctypes.byref(h)), "mtpt_create_batch")
    return h


def mtpt_set_particles_batch(h, dim: int, counts, pos, mass) -> None:
    counts = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
    mass = np.ascontiguousarray(np.asarray(mass, dtype=np.float64)).ravel()
    total = int(counts.sum())
    if mass.size != total:
        raise ValueError(f"expected {total} masses, got {mass.size}")
    pos = _host_f64(pos, (dim, total))
    _check(load().mtpt_set_particles_batch(h, counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           pos.ctypes.data, mass.ctypes.data),
           "mtpt_set_particles_batch")


def _info_dict(info) -> dict:
    return {"n": info.n, "step": info.step, "pair_count": info.pair_count,
            "D_RW": info.D_RW, "D_MT": info.D_MT, "sigma": info.sigma, "h2": info.h2,
            "psi": info.psi, "psi2": info.psi2, "kernel_norm": info.kernel_norm,
            "cells": tuple(info.cells), "cell_width": tuple(info.cell_width)}


def mtpt_get_realisation_info(h, k: int) -> dict:
    info = _Info()
    _check(load().mtpt_get_realisation_info(h, k, ctypes.byref(info)), "mtpt_get_realisation_info")
    return _info_dict(info)


def mtpt_set_tuning(h, cell_scale: float = 1.0, pair_block: int = 256) -> None:
    t = _Tuning(cell_scale, pair_block, 0)
    _check(load().mtpt_set_tuning(h, ctypes.byref(t)), "mtpt_set_tuning")


def mtpt_get_tuning(h) -> dict:
    t = _Tuning()
    _check(load().mtpt_get_tuning(h, ctypes.byref(t)), "mtpt_get_tuning")
    return {"cell_scale": t.cell_scale, "pair_block": t.pair_block}


def mtpt_autotune(h, trial_steps: int = 4) -> dict:
    t = _Tuning()
    _check(load().mtpt_autotune(h, trial_steps, ctypes.byref(t)), "mtpt_autotune")
    return {"cell_scale": t.cell_scale, "pair_block": t.pair_block}


def mtpt_check_word(reset: bool = False) -> int:
    """Bounds-check word of the checked build (see include/mtpt.h); raises
    MtptError(MTPT_ERR_STATE) in the normal build."""
    out = ctypes.c_uint32()
    _check(load().mtpt_check_word(ctypes.byref(out), 1 if reset else 0), "mtpt_check_word")
    return int(out.value)


def mtpt_adjoint_forward(h, nsteps: int, checkpoint_every: int) -> None:
    _check(load().mtpt_adjoint_forward(h, nsteps, checkpoint_every), "mtpt_adjoint_forward")


def mtpt_adjoint_backward(h, gmass, gmass0) -> float:
    """gmass: dL/dM_T, gmass0: output dL/dM_0 (CUDA float64 tensors, input
    order).  Returns dL/dD."""
    out = ctypes.c_double()
    n = gmass.numel()
    _check(load().mtpt_adjoint_backward(h, _dev_ptr(gmass, "float64", n),
                                        _dev_ptr(gmass0, "float64", n), ctypes.byref(out)),
           "mtpt_adjoint_backward")
    return float(out.value)


def mtpt_destroy(h) -> None:
    try:
        _check(load().mtpt_destroy(h), "mtpt_destroy")
    finally:
        _ASYNC_HOLD.pop(_handle_key(h), None)


def mtpt_set_stream(h, stream: int | None) -> None:
    _check(load().mtpt_set_stream(h, ctypes.c_void_p(stream or 0)), "mtpt_set_stream")


def mtpt_set_particles(h, dim: int, pos, mass) -> None:
    mass = np.ascontiguousarray(np.asarray(mass, dtype=np.float64)).ravel()
    n = mass.size
    pos = _host_f64(pos, (dim, n))
    _check(load().mtpt_set_particles(h, n, pos.ctypes.data, mass.ctypes.data),
           "mtpt_set_particles")


def mtpt_set_particles_device(h, dim: int, pos, mass) -> None:
    n = mass.numel()
    mtpt_set_stream(h, _torch_stream())
    _check(load().mtpt_set_particles_device(h, n, _dev_ptr(pos, "float64", dim * n),
                                            _dev_ptr(mass, "float64", n)),
           "mtpt_set_particles_device")


def mtpt_step(h, nsteps: int) -> None:
    _check(load().mtpt_step(h, nsteps), "mtpt_step")


def mtpt_step_ex(h, nsteps: int, flags: int) -> None:
    _check(load().mtpt_step_ex(h, nsteps, flags), "mtpt_step_ex")


def mtpt_get_info(h) -> dict:
    info = _Info()
    _check(load().mtpt_get_info(h, ctypes.byref(info)), "mtpt_get_info")
    return _info_dict(info)


def mtpt_get_masses(h, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _check(load().mtpt_get_masses(h, out.ctypes.data), "mtpt_get_masses")
    return out


def mtpt_get_masses_device(h, out) -> None:
    _check(load().mtpt_get_masses_device(h, _dev_ptr(out, "float64", out.numel())),
           "mtpt_get_masses_device")


def mtpt_get_positions(h, dim: int, n: int) -> np.ndarray:
    out = np.empty((dim, n), dtype=np.float64)
    _check(load().mtpt_get_positions(h, out.ctypes.data), "mtpt_get_positions")
    return out


def mtpt_get_positions_device(h, out) -> None:
    _check(load().mtpt_get_positions_device(h, _dev_ptr(out, "float64", out.numel())),
           "mtpt_get_positions_device")


def mtpt_get_row_sums(h, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _check(load().mtpt_get_row_sums(h, out.ctypes.data), "mtpt_get_row_sums")
    return out


def mtpt_get_pairs(h, cap: int):
    """Ordered neighbour pairs of the current positions as input-order index
    arrays (i, j), sorted by (i, j)."""
    pi = np.empty(max(cap, 1), dtype=np.uint32)
    pj = np.empty(max(cap, 1), dtype=np.uint32)
    count = ctypes.c_int64()
    rc = load().mtpt_get_pairs(h, cap, ctypes.byref(count), pi.ctypes.data, pj.ctypes.data)
    _check(rc, "mtpt_get_pairs")
    m = count.value
    i, j = pi[:m].astype(np.int64), pj[:m].astype(np.int64)
    order = np.lexsort((j, i))
    return i[order], j[order]


def mtpt_set_step(h, step: int) -> None:
    _check(load().mtpt_set_step(h, step), "mtpt_set_step")


def mtpt_sync(h) -> None:
    try:
        _check(load().mtpt_sync(h), "mtpt_sync")
    finally:
        _ASYNC_HOLD.pop(_handle_key(h), None)


# Host arrays handed to the *_async calls stay referenced here until the
# handle's next mtpt_sync (or mtpt_destroy), so the copies never read or
# write freed memory.
_ASYNC_HOLD: dict = {}


def _handle_key(h) -> int:
    return int(ctypes.cast(h, ctypes.c_void_p).value or 0)


def _host_in_place(a, numel: int, what: str) -> int:
    """Address of a float64, C-contiguous host array of `numel` elements (numpy
    or CPU torch tensor), used in place: a converted copy would be a
    temporary that the pending copy outlives."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != numel:
                raise ValueError(f"{what}: expected a contiguous float64 CPU tensor of {numel}")
            return a.data_ptr()
    except ImportError:
        pass
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
            and a.size == numel):
        raise ValueError(f"{what}: expected a C-contiguous float64 array of {numel}")
    return a.ctypes.data


def mtpt_set_particles_async(h, dim: int, pos, mass) -> None:
    """Enqueue a host load (include/mtpt.h); pos (dim x n) and mass (n) are
    read in place until mtpt_sync: pinned torch tensors give the overlap."""
    n = mass.numel() if hasattr(mass, "numel") else np.asarray(mass).size
    pp = _host_in_place(pos, dim * n, "pos")
    pm = _host_in_place(mass, n, "mass")
    _check(load().mtpt_set_particles_async(h, n, pp, pm), "mtpt_set_particles_async")
    _ASYNC_HOLD.setdefault(_handle_key(h), []).extend((pos, mass))


def mtpt_get_masses_async(h, out) -> None:
    """Enqueue the read of the masses into `out` (n float64, host), filled
    once mtpt_sync returns."""
    n = out.numel() if hasattr(out, "numel") else np.asarray(out).size
    po = _host_in_place(out, n, "out")
    _check(load().mtpt_get_masses_async(h, po), "mtpt_get_masses_async")
    _ASYNC_HOLD.setdefault(_handle_key(h), []).append(out)


def mtpt_timing_enable(h, on: bool) -> None:
    _check(load().mtpt_timing_enable(h, 1 if on else 0), "mtpt_timing_enable")


def mtpt_timing_read(h) -> dict:
    """{kernel name: (launches, total milliseconds)} since the last reset."""
    cap = 64
    arr = (_KernelStat * cap)()
    count = ctypes.c_int32()
    _check(load().mtpt_timing_read(h, cap, arr, ctypes.byref(count)), "mtpt_timing_read")
    return {arr[k].name.decode(): (int(arr[k].launches), float(arr[k].total_ms))
            for k in range(min(cap, count.value))}


def mtpt_timing_reset(h) -> None:
    _check(load().mtpt_timing_reset(h), "mtpt_timing_reset")


def mtpt_step_noalloc(params: Params, step: int, pos, mass) -> None:
    """One time step on torch CUDA buffers (pos: dim*n float64 SoA, mass: n
    float64, updated in place) with no device allocation, for callers whose
    device memory is owned by another allocator.  Enqueued on torch's current
    stream; n is limited to NOALLOC_MAX_PARTICLES."""
    n = mass.numel()
    cp = params.c()
    _check(load().mtpt_step_noalloc(ctypes.byref(cp), n, step,
                                    _dev_ptr(pos, "float64", params.dim * n),
                                    _dev_ptr(mass, "float64", n), _torch_stream()),
           "mtpt_step_noalloc")


def mtpt_tiling_factors(dim: int, lo, hi, ntiles: int) -> tuple:
    """Tiles per axis of a checkerboard of `ntiles` tiles (Eq. "minimization")."""
    lo = np.ascontiguousarray(np.asarray(lo, dtype=np.float64))
    hi = np.ascontiguousarray(np.asarray(hi, dtype=np.float64))
    out = (ctypes.c_int32 * 3)()
    _check(load().mtpt_tiling_factors(dim, lo.ctypes.data, hi.ctypes.data, ntiles, out),
           "mtpt_tiling_factors")
    return tuple(int(v) for v in out)


def mtpt_set_tiling(h, tiles, tile: int, n_global: int) -> None:
    t = _Tiling((ctypes.c_int32 * 3)(*(list(tiles) + [1] * (3 - len(tiles)))), tile, n_global)
    _check(load().mtpt_set_tiling(h, ctypes.byref(t)), "mtpt_set_tiling")


def mtpt_set_particles_tile(h, dim: int, pos, mass, ids) -> None:
    mass = np.ascontiguousarray(np.asarray(mass, dtype=np.float64)).ravel()
    n = mass.size
    pos = _host_f64(pos, (dim, n))
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32)).ravel()
    if ids.size != n:
        raise ValueError(f"expected {n} ids, got {ids.size}")
    _check(load().mtpt_set_particles_tile(h, n, pos.ctypes.data, mass.ctypes.data,
                                          ids.ctypes.data), "mtpt_set_particles_tile")


def mtpt_tile_pack(h, send, ntiles: int):
    """Packs into the CUDA float64 tensor `send` (records of dim + 2 values,
    capacity send.numel() // (dim + 2) records).  Returns (status, counts),
    counts an int64 array of 2 x ntiles; status MTPT_ERR_CAPACITY asks for a
    larger buffer, anything else but MTPT_OK raises."""
    import torch
    if not (isinstance(send, torch.Tensor) and send.is_cuda and send.is_contiguous()
            and send.dtype == torch.float64 and send.dim() == 2):
        raise ValueError("expected a contiguous 2-d CUDA float64 tensor of records")
    counts = np.zeros(2 * ntiles, dtype=np.int64)
    rc = load().mtpt_tile_pack(h, send.shape[0], ctypes.c_void_p(send.data_ptr()),
                               counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc not in (MTPT_OK, MTPT_ERR_CAPACITY):
        raise MtptError(rc, "mtpt_tile_pack")
    return rc, counts


def mtpt_tile_transfer(h, recv) -> None:
    """recv: contiguous 2-d CUDA float64 tensor of received records."""
    _check(load().mtpt_tile_transfer(h, recv.shape[0], ctypes.c_void_p(recv.data_ptr())
                                     if recv.numel() else None), "mtpt_tile_transfer")


def mtpt_get_ids(h, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    _check(load().mtpt_get_ids(h, out.ctypes.data), "mtpt_get_ids")
    return out


def mtpt_set_reaction(h, k: float) -> None:
    _check(load().mtpt_set_reaction(h, float(k)), "mtpt_set_reaction")


def mtpt_set_masses_b(h, mass_b) -> None:
    mass_b = np.ascontiguousarray(np.asarray(mass_b, dtype=np.float64).ravel())
    _check(load().mtpt_set_masses_b(h, mass_b.ctypes.data), "mtpt_set_masses_b")


def mtpt_get_masses_b(h, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _check(load().mtpt_get_masses_b(h, out.ctypes.data), "mtpt_get_masses_b")
    return out


def mtpt_debug_fail_alloc(nth: int) -> int:
    """Make the nth device allocation from now fail (0: off); returns how many
    the previous setting still had to go."""
    left = ctypes.c_int64()
    _check(load().mtpt_debug_fail_alloc(nth, ctypes.byref(left)), "mtpt_debug_fail_alloc")
    return int(left.value)


def mtpt_debug_scan_hold(tile: int) -> int:
    """Make the scans launched from now never publish scan tile `tile` (-1:
    off); returns how many scan tiles on the current device have stopped
    waiting for a tile before them so far (syncs the device)."""
    gave_up = ctypes.c_uint64()
    _check(load().mtpt_debug_scan_hold(tile, ctypes.byref(gave_up)), "mtpt_debug_scan_hold")
    return int(gave_up.value)


def mtpt_status_string(code: int) -> str:
    return status_string(code)


class Simulation:
    """Owning wrapper over one handle (host numpy in, host numpy out)."""

    def __init__(self, params: Params, pos=None, mass=None):
        self.params = params
        self.h = mtpt_create(params)
        self.n = 0
        if pos is not None:
            self.set_particles(pos, mass)

    def set_particles(self, pos, mass):
        mass = np.asarray(mass, dtype=np.float64).ravel()
        mtpt_set_particles(self.h, self.params.dim, pos, mass)
        self.n = mass.size

    def step(self, nsteps: int = 1, flags: int = MTPT_DO_WALK | MTPT_DO_TRANSFER):
        mtpt_step_ex(self.h, nsteps, flags)

    def masses(self) -> np.ndarray:
        return mtpt_get_masses(self.h, self.n)

    def set_particles_async(self, pos, mass):
        """Pipelined load (same n); pos, mass are read in place until sync()."""
        mtpt_set_particles_async(self.h, self.params.dim, pos, mass)

    def masses_async(self, out):
        """Pipelined read into `out` (n float64, host), valid after sync()."""
        mtpt_get_masses_async(self.h, out)

    def sync(self):
        mtpt_sync(self.h)

    def positions(self) -> np.ndarray:
        return mtpt_get_positions(self.h, self.params.dim, self.n)

    def row_sums(self) -> np.ndarray:
        return mtpt_get_row_sums(self.h, self.n)

    def pairs(self, cap: int | None = None):
        if cap is None:
            cap = max(1024, 64 * self.n)
        return mtpt_get_pairs(self.h, cap)

    def info(self) -> dict:
        return mtpt_get_info(self.h)

    def autotune(self, trial_steps: int = 4) -> dict:
        return mtpt_autotune(self.h, trial_steps)

    def set_reaction(self, k: float, mass_b=None):
        """Bimolecular reaction A + B -> 0 with rate constant k; species B's
        masses (input order) when given, else zero."""
        mtpt_set_reaction(self.h, k)
        if mass_b is not None:
            mtpt_set_masses_b(self.h, mass_b)

    def masses_b(self) -> np.ndarray:
        return mtpt_get_masses_b(self.h, self.n)

    def set_tuning(self, cell_scale: float = 1.0, pair_block: int = 256):
        mtpt_set_tuning(self.h, cell_scale, pair_block)

    def set_step(self, step: int):
        mtpt_set_step(self.h, step)

    def close(self):
        if self.h is not None:
            mtpt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(Simulation):
    """Owning wrapper over a batch handle: realisation k uses params_list[k]
    and the k-th block of the concatenated particle arrays."""

    def __init__(self, params_list, counts=None, pos=None, mass=None):
        self.params_list = list(params_list)
        self.params = self.params_list[0]
        self.h = mtpt_create_batch(self.params_list)
        self.n = 0
        self.counts = None
        if counts is not None:
            self.set_particles_batch(counts, pos, mass)

    def set_particles_batch(self, counts, pos, mass):
        mtpt_set_particles_batch(self.h, self.params.dim, counts, pos, mass)
        self.counts = np.asarray(counts, dtype=np.int64)
        self.n = int(self.counts.sum())

    def realisation_info(self, k: int) -> dict:
        return mtpt_get_realisation_info(self.h, k)

    def split(self, arr):
        """Split a concatenated per-particle array into per-realisation views
        (the last axis is the particle axis)."""
        edges = np.concatenate([[0], np.cumsum(self.counts)])
        return [arr[..., edges[k]:edges[k + 1]] for k in range(len(self.counts))]
