"""The C-ABI library loads and exports every entry point that include/mtpt.h
declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2204_03756_gb300 import build as cuda_build
from paper_2204_03756_gb300 import mtpt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "mtpt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mtpt_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return mtpt.load()


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for name in ("mtpt_create", "mtpt_set_particles", "mtpt_step", "mtpt_get_masses",
                 "mtpt_destroy"):
        assert name in syms
    assert set(syms) == set(mtpt.EXPORTED)


def _declaration_comments():
    """The comment block right before each declaration, whitespace and the
    comment's leading asterisks folded."""
    text = open(os.path.join(ROOT, "include", "mtpt.h")).read()
    pat = re.compile(r"(/\*(?:(?!\*/).)*\*/)\s*(?:#define[^\n]*\n\s*)*"
                     r"(?:int|const char\*)\s+(mtpt_[a-z_]+)\s*\(", re.S)
    out = {}
    for m in pat.finditer(text):
        body = re.sub(r"\s*\n\s*\*?", " ", m.group(1))
        out[m.group(2)] = re.sub(r"\s+", " ", body)
    return out


def test_every_boundary_call_cites_its_passage():
    """The calls of the method itself name the section or equation of the
    paper that defines them; every other declaration either cites one, says
    that it has no counterpart in the paper, or defers to the call it varies
    ("As mtpt_...")."""
    com = _declaration_comments()
    assert set(com) == set(_declared_symbols())
    for name in ("mtpt_create", "mtpt_set_particles", "mtpt_step", "mtpt_get_masses",
                 "mtpt_get_positions", "mtpt_create_batch", "mtpt_get_row_sums",
                 "mtpt_get_pairs", "mtpt_get_info"):
        assert "Sec." in com[name] or "Eq." in com[name], name
    for name, c in com.items():
        cites = "Sec." in c or "Eq." in c
        other = "no counterpart in the paper" in c.lower() or re.match(r"/\* As mtpt_", c)
        assert cites or other, name


def test_binding_declares_every_signature(lib):
    """ctypes passes undeclared arguments as C int: every entry point the
    binding exports has its argument types declared."""
    for name in mtpt.EXPORTED:
        assert getattr(lib, name).argtypes is not None, name


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_parameter_validation_without_gpu(lib):
    good = dict(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0), hi=(10, 10))
    for ok in (good, dict(good, D=0.0), dict(good, kappa=1.0), dict(good, D=1e-31, dt=1e-3)):
        mtpt.mtpt_destroy(mtpt.mtpt_create(mtpt.Params(**ok)))   # h^2 = 0 or >= 1e-35
    bad = [dict(dim=0), dict(dim=4), dict(kappa=1.5), dict(dt=0.0), dict(D=-1.0),
           dict(lo=(5, 0), hi=(1, 10)), dict(beta=0.0), dict(lam=0.0), dict(precision=7),
           dict(D=float("nan")), dict(lam=20.5), dict(lo=(-2e15, 0)),
           dict(D=1e-33, dt=1e-3),          # h^2 = 1e-36: below the kernel range
           dict(v=(float("nan"), 0.0)), dict(v=(0.0, float("inf"))), dict(v=(1e17, 0.0))]
    for b in bad:
        kw = dict(good)
        kw.update(b)
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_create(mtpt.Params(**kw))
        assert e.value.code == mtpt.MTPT_ERR_INVALID_ARG
    assert lib.mtpt_create(None, None) == mtpt.MTPT_ERR_INVALID_ARG
    assert lib.mtpt_destroy(None) == mtpt.MTPT_OK
    assert lib.mtpt_step(None, 1) == mtpt.MTPT_ERR_INVALID_ARG


def test_calls_before_particles_are_rejected(lib):
    h = mtpt.mtpt_create(mtpt.Params(dim=2, lo=(0, 0), hi=(10, 10)))
    try:
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_step(h, 1)
        assert e.value.code == mtpt.MTPT_ERR_STATE
        assert lib.mtpt_step(h, -1) == mtpt.MTPT_ERR_INVALID_ARG
        buf = (ctypes.c_double * 2)()
        assert lib.mtpt_set_particles_async(h, 1, buf, buf) == mtpt.MTPT_ERR_STATE
        assert lib.mtpt_get_masses_async(h, buf) == mtpt.MTPT_ERR_STATE
        assert lib.mtpt_set_particles_async(None, 1, buf, buf) == mtpt.MTPT_ERR_INVALID_ARG
    finally:
        mtpt.mtpt_destroy(h)


def test_status_strings(lib):
    for code in range(7):
        assert mtpt.mtpt_status_string(code)
    assert mtpt.mtpt_status_string(99) == "unknown status"


def test_checked_library_exports_every_declared_symbol():
    from paper_2204_03756_gb300 import build
    build.build()
    lib = ctypes.CDLL(build.LIB_CHECKED_PATH)
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_normal_build_has_no_check_word(lib):
    out = ctypes.c_uint32(7)
    assert lib.mtpt_check_word(ctypes.byref(out), 0) == mtpt.MTPT_ERR_STATE
    assert out.value == 0


@pytest.mark.parametrize("variant", ["normal", "checked"])
def test_c_client_compiles_links_and_runs_without_a_gpu(tmp_path, variant):
    """The header is valid C99 and a C program links every entry point from
    the shipped library and gets the documented answers from the calls that
    need no GPU."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    cuda_build.build()
    lib = cuda_build.LIB_PATH if variant == "normal" else cuda_build.LIB_CHECKED_PATH
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "abi_check")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-o", exe,
           os.path.join(here, "c", "abi_check.c"), "-I", cuda_build.INCLUDE_DIR, lib,
           "-Wl,-rpath," + os.path.dirname(lib)]
    out = subprocess.run(cmd, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
