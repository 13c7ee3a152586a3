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


def test_stats_scratch_sizes_follow_the_documented_formula(lib):
    """vct_stats_noalloc_bytes / vct_stats_workspace_bytes against the layout the
    header states: five regions rounded up to 256 bytes, then 16 B per
    scenario of offset table."""
    from paper_2202_13927_gb300 import vct
    up = lambda x: (x + 255) // 256 * 256
    for S, n, hz in ((1, 1000, [2016]), (3, 4099, [1, 17, 300]), (2, 1_000_000, [104832, 288]),
                     (1, 0, [5])):
        nblk = min(max((max(n, 1) + 1023) // 1024, 1), 1024)
        want = (up(104 * S) + up(32 * S * nblk) + up(8 * S * nblk)
                + up(C.sizeof(vct.PopulationStats) * S) + up(4 * 5 * sum(h + 1 for h in hz)) + 16 * S)
        assert vct.stats_noalloc_bytes(S, n, hz) == want, (S, n, hz)
        assert vct.stats_workspace_bytes(S, n, hz) == want
    # a 52-week scenario fits the fixed array, four of them do not
    assert vct.stats_noalloc_bytes(1, 1_000_000, [104832]) <= (8 << 20)
    assert vct.stats_noalloc_bytes(4, 1_000_000, [104832] * 4) > (8 << 20)
    assert vct.stats_noalloc_bytes(1, 10, [-1]) == 0
    assert lib.vct_stats_noalloc_bytes(0, 10, None) == 0


def test_new_calls_validate_before_touching_the_device(lib):
    from paper_2202_13927_gb300 import vct
    n = C.c_size_t(7)
    assert lib.vct_simulate_workspace_bytes(None, None, 0, None, C.byref(n)) == -1 and n.value == 0
    assert lib.vct_checkpoint(None, None, 0, None, 10, None, None, None) == -1
    assert lib.vct_resume(None, None, 0, None, 0, None, None, None) == -1
    assert lib.vct_bg_cdf(None, 0, None, None) == 0           # nothing to do
    assert lib.vct_bg_cdf(None, 1, None, None) == -1
    q = (C.c_double * 2)(0.5, 1.5)
    assert lib.vct_dose_quantiles(None, 1, q, 2, None, None) == -1
    assert b"[0, 1]" in lib.vct_last_error()
    assert lib.vct_dose_quantiles(None, 1, q, 0, None, None) == -1
    assert lib.vct_dose_quantiles(None, 1, q, vct.MAX_QUANTILES + 1, None, None) == -1
    assert lib.vct_stats_with_workspace(None, 1, 5, None, 0, None, 0, None, None) == -1
    assert lib.vct_surrogate_set_lr(None, 1e-3) == -1
