"""ctypes binding of the serial FP64 C oracle (TEST INFRASTRUCTURE ONLY).

Builds ``mtpt_oracle.c`` with gcc on first use (``-O2 -ffp-contract=off``,
no fast-math) into ``oracle/_build/`` and exposes numpy-level wrappers.
Positions are structure-of-arrays, shape ``(dim, n)`` float64; masses shape
``(n,)`` float64; particle ids ``uint32``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mtpt_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lib = None

__all__ = [
    "OracleParams", "build", "load", "derived", "philox4x32_10", "log_f32",
    "sincos_2pi_f32", "box_muller", "normals", "reflect", "random_walk", "pairs",
    "mass_transfer", "run", "react", "particle_rate", "run_reactive",
]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, plain C, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int),
                ("D", ctypes.c_double), ("kappa", ctypes.c_double),
                ("dt", ctypes.c_double), ("beta", ctypes.c_double),
                ("lam", ctypes.c_double),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("seed", ctypes.c_uint64), ("v", ctypes.c_double * 3)]


@dataclass
class OracleParams:
    """Parameters of Sec. 2-3: dimension, D, kappa = D_RW / D, dt, beta,
    lambda (psi = lambda sqrt(4 D_MT dt / beta)), box [lo, hi] with
    reflecting walls, the random-walk seed, and a uniform velocity v (the
    advection term of the model equation of Sec. 2; the paper's runs take
    v = 0)."""
    dim: int = 2
    D: float = 1.0
    kappa: float = 0.5
    dt: float = 0.1
    beta: float = 1.0
    lam: float = 3.0
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (100.0, 100.0, 100.0)
    seed: int = 0
    v: tuple = (0.0, 0.0, 0.0)

    def c(self) -> _CParams:
        lo = list(self.lo) + [0.0] * (3 - len(self.lo))
        hi = list(self.hi) + [0.0] * (3 - len(self.hi))
        v = list(self.v) + [0.0] * (3 - len(self.v))
        return _CParams(self.dim, self.D, self.kappa, self.dt, self.beta, self.lam,
                        (ctypes.c_double * 3)(*lo[:3]), (ctypes.c_double * 3)(*hi[:3]),
                        self.seed, (ctypes.c_double * 3)(*v[:3]))


def load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    u32p, f32p, f64p, i64p = (P(ctypes.c_uint32), P(ctypes.c_float),
                              P(ctypes.c_double), P(ctypes.c_int64))
    lib.orc_philox_many.argtypes = [ctypes.c_int64, u32p, u32p, u32p]
    lib.orc_log_f32_many.argtypes = [ctypes.c_int64, f32p, f32p]
    lib.orc_sincos_2pi_many.argtypes = [ctypes.c_int64, u32p, f32p, f32p]
    lib.orc_box_muller_many.argtypes = [ctypes.c_int64, u32p, f32p]
    lib.orc_normals_many.argtypes = [ctypes.c_uint64, ctypes.c_int64, u32p,
                                     ctypes.c_uint64, f32p]
    lib.orc_reflect.argtypes = [ctypes.c_double] * 3
    lib.orc_reflect.restype = ctypes.c_double
    lib.orc_random_walk.argtypes = [P(_CParams), ctypes.c_int64, f64p, u32p, ctypes.c_uint64]
    lib.orc_pairs.argtypes = [ctypes.c_int, ctypes.c_int64, f64p, ctypes.c_double,
                              ctypes.c_int, P(i64p), P(i64p)]
    lib.orc_pairs.restype = ctypes.c_int64
    lib.orc_free.argtypes = [ctypes.c_void_p]
    lib.orc_mass_transfer.argtypes = [P(_CParams), ctypes.c_int64, f64p, f64p, f64p,
                                      ctypes.c_int, f64p, f64p]
    lib.orc_mass_transfer.restype = ctypes.c_int64
    lib.orc_run.argtypes = [P(_CParams), ctypes.c_int64, f64p, f64p, u32p,
                            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int]
    lib.orc_run.restype = ctypes.c_int64
    lib.orc_derived_values.argtypes = [P(_CParams), f64p]
    lib.orc_react.argtypes = [ctypes.c_int64, f64p, f64p, ctypes.c_double, ctypes.c_double]
    lib.orc_particle_rate.argtypes = [P(_CParams), ctypes.c_int64, ctypes.c_double]
    lib.orc_particle_rate.restype = ctypes.c_double
    lib.orc_run_reactive.argtypes = [P(_CParams), ctypes.c_int64, f64p, f64p, f64p, u32p,
                                     ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_double]
    lib.orc_run_reactive.restype = ctypes.c_int64
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def derived(p: OracleParams) -> dict:
    """D_RW, D_MT, walk scale sigma, h^2, psi, psi^2 and (2 pi h^2)^(-d/2)."""
    lib = load()
    out = np.zeros(7, dtype=np.float64)
    cp = p.c()
    lib.orc_derived_values(ctypes.byref(cp), _ptr(out, ctypes.c_double))
    keys = ["D_RW", "D_MT", "sigma", "h2", "psi", "psi2", "kernel_norm"]
    return dict(zip(keys, out.tolist()))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` (n x 4 uint32) under ``key`` (2 uint32)."""
    lib = load()
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib.orc_philox_many(ctr.shape[0], _ptr(ctr, ctypes.c_uint32),
                        _ptr(key, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def log_f32(u) -> np.ndarray:
    lib = load()
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float32).ravel())
    out = np.empty_like(u)
    lib.orc_log_f32_many(u.size, _ptr(u, ctypes.c_float), _ptr(out, ctypes.c_float))
    return out


def sincos_2pi_f32(k):
    """(sin, cos) of 2 pi k / 2^24 for integers k in [0, 2^24]."""
    lib = load()
    k = np.ascontiguousarray(np.asarray(k, dtype=np.uint32).ravel())
    s = np.empty(k.size, dtype=np.float32)
    c = np.empty(k.size, dtype=np.float32)
    lib.orc_sincos_2pi_many(k.size, _ptr(k, ctypes.c_uint32), _ptr(s, ctypes.c_float),
                            _ptr(c, ctypes.c_float))
    return s, c


def box_muller(words) -> np.ndarray:
    """The four N(0,1) draws (n x 4 float32) the walk takes from each block
    of four generator words (n x 4 uint32)."""
    lib = load()
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(-1, 4))
    out = np.empty(w.shape, dtype=np.float32)
    lib.orc_box_muller_many(w.shape[0], _ptr(w, ctypes.c_uint32), _ptr(out, ctypes.c_float))
    return out


def normals(seed: int, ids, step: int) -> np.ndarray:
    """The four N(0,1) draws (n x 4 float32) of each particle id at ``step``."""
    lib = load()
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32).ravel())
    out = np.empty((ids.size, 4), dtype=np.float32)
    lib.orc_normals_many(seed, ids.size, _ptr(ids, ctypes.c_uint32), step,
                         _ptr(out, ctypes.c_float))
    return out


def reflect(x: float, lo: float, hi: float) -> float:
    return load().orc_reflect(x, lo, hi)


def random_walk(p: OracleParams, pos, ids, step: int) -> np.ndarray:
    """One random-walk move (with reflection) of every particle; returns new
    positions (dim x n), leaving ``pos`` untouched."""
    lib = load()
    out = np.ascontiguousarray(np.array(pos, dtype=np.float64, copy=True))
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    cp = p.c()
    lib.orc_random_walk(ctypes.byref(cp), out.shape[1], _ptr(out, ctypes.c_double),
                        _ptr(ids, ctypes.c_uint32), step)
    return out


def pairs(pos, psi2: float, method: str = "kdtree"):
    """All ordered neighbour pairs (i, j), i != j, ||x_i - x_j||^2 <= psi2,
    sorted by (i, j).  ``method`` is "brute" or "kdtree"."""
    lib = load()
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
    dim, n = pos.shape
    pi = ctypes.POINTER(ctypes.c_int64)()
    pj = ctypes.POINTER(ctypes.c_int64)()
    m = lib.orc_pairs(dim, n, _ptr(pos, ctypes.c_double), psi2,
                      0 if method == "brute" else 1, ctypes.byref(pi), ctypes.byref(pj))
    if m < 0:
        raise MemoryError("oracle pair search: allocation failed")
    if m == 0:
        if pi:
            lib.orc_free(pi)
            lib.orc_free(pj)
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    i = np.ctypeslib.as_array(pi, shape=(m,)).copy()
    j = np.ctypeslib.as_array(pj, shape=(m,)).copy()
    lib.orc_free(pi)
    lib.orc_free(pj)
    order = np.lexsort((j, i))
    return i[order], j[order]


def mass_transfer(p: OracleParams, pos, mass, method: str = "kdtree"):
    """One mass-transfer update on fixed positions.  Returns
    (new_mass, row_sums, col_sums, n_pairs)."""
    lib = load()
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
    mass = np.ascontiguousarray(np.asarray(mass, dtype=np.float64))
    n = mass.size
    out = np.empty_like(mass)
    rs = np.empty_like(mass)
    cs = np.empty_like(mass)
    cp = p.c()
    m = lib.orc_mass_transfer(ctypes.byref(cp), n, _ptr(pos, ctypes.c_double),
                              _ptr(mass, ctypes.c_double), _ptr(out, ctypes.c_double),
                              0 if method == "brute" else 1,
                              _ptr(rs, ctypes.c_double), _ptr(cs, ctypes.c_double))
    if m < 0:
        raise MemoryError("oracle mass transfer: allocation failed")
    return out, rs, cs, int(m)


def run(p: OracleParams, pos, mass, nsteps: int, step0: int = 0, ids=None,
        method: str = "kdtree"):
    """``nsteps`` full steps (walk, then mass transfer) from step counter
    ``step0``.  Returns (pos, mass, total ordered pairs over all steps)."""
    lib = load()
    pos = np.ascontiguousarray(np.array(pos, dtype=np.float64, copy=True))
    mass = np.ascontiguousarray(np.array(mass, dtype=np.float64, copy=True))
    n = mass.size
    if ids is None:
        ids = np.arange(n, dtype=np.uint32)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    cp = p.c()
    total = lib.orc_run(ctypes.byref(cp), n, _ptr(pos, ctypes.c_double),
                        _ptr(mass, ctypes.c_double), _ptr(ids, ctypes.c_uint32),
                        step0, nsteps, 0 if method == "brute" else 1)
    if total < 0:
        raise MemoryError("oracle run: allocation failed")
    return pos, mass, int(total)


def react(a, b, kp: float, dt: float):
    """One well-mixed reaction substep A + B -> 0 of length dt on particle
    masses a, b >= 0 with the particle rate kp (see ``particle_rate``).
    Returns the new (a, b)."""
    lib = load()
    a = np.ascontiguousarray(np.array(a, dtype=np.float64, copy=True))
    b = np.ascontiguousarray(np.array(b, dtype=np.float64, copy=True))
    lib.orc_react(a.size, _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double), kp, dt)
    return a, b


def particle_rate(p: OracleParams, n: int, k: float) -> float:
    """k_p = k N / V: the rate constant k of the concentration rate law
    applied to particle masses (C = N M / V)."""
    cp = p.c()
    return float(load().orc_particle_rate(ctypes.byref(cp), n, k))


def run_reactive(p: OracleParams, pos, ma, mb, nsteps: int, k: float, step0: int = 0,
                 ids=None, method: str = "kdtree"):
    """``nsteps`` reactive steps A + B -> 0 (walk; transfer of both species
    with the same weights; well-mixed reaction per particle with rate
    constant k).  Returns (pos, ma, mb, total ordered pairs)."""
    lib = load()
    pos = np.ascontiguousarray(np.array(pos, dtype=np.float64, copy=True))
    ma = np.ascontiguousarray(np.array(ma, dtype=np.float64, copy=True))
    mb = np.ascontiguousarray(np.array(mb, dtype=np.float64, copy=True))
    n = ma.size
    if ids is None:
        ids = np.arange(n, dtype=np.uint32)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    cp = p.c()
    total = lib.orc_run_reactive(ctypes.byref(cp), n, _ptr(pos, ctypes.c_double),
                                 _ptr(ma, ctypes.c_double), _ptr(mb, ctypes.c_double),
                                 _ptr(ids, ctypes.c_uint32), step0, nsteps,
                                 0 if method == "brute" else 1, k)
    if total < 0:
        raise MemoryError("oracle reactive run: allocation failed")
    return pos, ma, mb, int(total)
