"""The C-ABI library builds, loads and exports what include/vct.h declares.

No GPU needed: only calls that touch no device are made (struct sizes,
version, argument validation that fails before any CUDA call).
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "vct.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(vct_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_13927_gb300 import vct
    return vct.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("vct_create_population", "vct_simulate", "vct_stats", "vct_last_error",
                     "vct_destroy_population", "vct_sync", "vct_state_bytes"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2202_13927_gb300 import vct
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in vct.SIGNATURES, f"binding lacks {name}"


def test_struct_mirrors_match_the_library(lib):
    from paper_2202_13927_gb300 import vct
    assert lib.vct_struct_size(b"vct_patient_stats") == vct.PATIENT_STATS_DTYPE.itemsize == 96
    assert lib.vct_struct_size(b"nope") == 0
    assert b"sm_103a" in lib.vct_version()


def test_state_bytes(lib):
    assert lib.vct_state_bytes(2, 1000) == 2 * 1000 * (27 * 8 + 8 * 4)
    assert lib.vct_state_bytes(0, 5) == 0


def test_argument_errors_are_reported_not_raised(lib):
    from paper_2202_13927_gb300 import vct, workloads as W
    h = C.c_void_p()
    assert lib.vct_create_population(None, None, C.byref(h)) == -1
    assert b"NULL" in lib.vct_last_error()
    d = vct.population_desc(W.population(10, 1))
    d.max_attempts = 0
    assert lib.vct_create_population(C.byref(d), None, C.byref(h)) == -1
    assert b"max_attempts" in lib.vct_last_error()
    d = vct.population_desc(W.population(10, 1))
    d.first_patient = (1 << 32) - 5
    assert lib.vct_create_population(C.byref(d), None, C.byref(h)) == -1
    d = vct.population_desc(W.population(10, 1))
    d.p_mean[11] = float("nan")
    assert lib.vct_create_population(C.byref(d), None, C.byref(h)) == -1
    assert lib.vct_simulate(None, None, 0, None, None, None) == -1
    assert lib.vct_stats(None, 1, 5, None, 0, None, None) == -1
    assert lib.vct_philox_fill(None, -1, 0, None, None, 0, None) == -1


def test_scenario_and_option_marshalling():
    from paper_2202_13927_gb300 import vct, workloads as W
    sc = W.scenario(7, meal_minute=(420, 720, 1080), kp_mult=2.0)
    s = vct.scenario_struct(sc)
    assert s.n_meals == 3 and s.horizon_periods == 7 * 288 and s.kp_mult == 2.0
    assert list(s.meal_minute)[:3] == [420.0, 720.0, 1080.0]
    o = vct.sim_opts({"precision": "fp64", "trace_dtype": "f32", "trace_kind": "bg"})
    assert o.precision == vct.FP64 and o.trace_dtype == vct.TRACE_F32 and o.trace_kind == vct.TRACE_BG
    arr = vct.scenario_array([sc, sc])
    assert len(arr) == 2
    with pytest.raises(ValueError):
        vct.scenario_struct(W.scenario(1, meal_minute=tuple(range(0, 900, 100))))


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without libvct.so the binding raises instead of running
    anything else."""
    from paper_2202_13927_gb300 import vct
    monkeypatch.setattr(vct, "_lib", None)
    monkeypatch.setattr(vct._build, "LIB", str(tmp_path / "libvct.so"))
    with pytest.raises(RuntimeError, match="libvct.so not found"):
        vct.load(build_if_missing=False)


def test_no_gpu_means_an_error_not_a_fallback():
    """On a host without a GPU the product path raises at its first call."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2202_13927_gb300 import vct, workloads as W
    with pytest.raises(Exception):
        vct.Population.create(W.population(4, 1))


def test_every_declared_call_is_documented():
    """Each entry point of the header follows a comment (a group of
    declarations in a row shares the comment above the group)."""
    lines = open(os.path.join(ROOT, "include", "vct.h")).read().splitlines()
    documented, in_decl, undocumented = False, False, []
    decl = re.compile(r"^(vct_status|const char \*|size_t)\s*\**\s*(vct_\w+)\(")
    for line in lines:
        s = line.strip()
        if s.endswith("*/"):
            documented = True
            continue
        m = decl.match(s)
        if m:
            in_decl = True
            if not documented:
                undocumented.append(m.group(2))
        if in_decl and s.endswith(";"):
            in_decl = False
            continue
        if not in_decl and not s:
            documented = False
    assert undocumented == []
