"""ctypes front of the FP64 CPU oracle (``vct_oracle.c``).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It imports nothing from the CUDA package; inputs arrive as the plain
dictionaries the seeded workload generators produce.

Every function here marshals arguments only; the arithmetic is in the C file,
whose header lists the paper sections (Eq. 1-3, Sec. III-C, IV-A, IV-B) and
the project readings it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vct_oracle.c")
_HDR = os.path.join(_HERE, "vct_oracle.h")
_LIB = os.path.join(_HERE, "libvct_oracle.so")
_lock = threading.Lock()
_lib = None

NPAR, NROW, NX, MAXMEALS = 16, 17, 11, 8
PARAM_NAMES = ["EGP0", "F01", "k12", "ka1", "ka2", "ka3", "SIT", "SID", "SIE", "ke",
               "VI", "VG", "tauS", "tauD", "AG", "tauCGM"]
STATE_NAMES = ["D1", "D2", "S1", "S2", "I", "x1", "x2", "x3", "Q1", "Q2", "Gsc"]


class PopDesc(C.Structure):
    _fields_ = [("bw_mean", C.c_double), ("bw_sd", C.c_double),
                ("p_mean", C.c_double * NPAR), ("p_sd", C.c_double * NPAR),
                ("g_sp", C.c_double), ("min_basal_u_per_h", C.c_double),
                ("sigma_q1", C.c_double), ("cgm_sd", C.c_double),
                ("seed", C.c_uint64), ("max_attempts", C.c_int32), ("pad", C.c_int32),
                ("tau_gg_min", C.c_double), ("s_gg", C.c_double)]


class DayPlan(C.Structure):
    _fields_ = [("n_meals", C.c_int32), ("pad", C.c_int32), ("minute", C.c_float * MAXMEALS),
                ("g_per_kg", C.c_float * MAXMEALS)]


class Scenario(C.Structure):
    _fields_ = [("kp_mult", C.c_double), ("ki_mult", C.c_double), ("kd_mult", C.c_double),
                ("kp_per_ub", C.c_double), ("ti_min", C.c_double), ("td_min", C.c_double),
                ("i_max", C.c_double), ("basal_scale", C.c_double),
                ("meal_mean_g", C.c_double), ("meal_sd_g", C.c_double),
                ("meal_minute", C.c_double * MAXMEALS), ("n_meals", C.c_int32),
                ("bolus", C.c_int32), ("horizon", C.c_int64), ("stream_id", C.c_uint32),
                ("pad", C.c_uint32), ("day_plans", C.c_void_p), ("n_day_plans", C.c_int32),
                ("meal_cv", C.c_float), ("glucagon", C.c_int32), ("pad2", C.c_int32),
                ("gg_threshold", C.c_double), ("gg_gain", C.c_double), ("gg_max_ug", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("ts_min", C.c_double), ("substeps", C.c_int32), ("integrator", C.c_int32),
                ("noise_refine", C.c_int32), ("pad", C.c_int32), ("edge_band", C.c_double * 8)]


class Stats(C.Structure):
    _fields_ = [("tir", C.c_uint32 * 5), ("hypo_episodes", C.c_uint32),
                ("q1_clamps", C.c_uint32), ("status", C.c_uint32),
                ("g_mean", C.c_double), ("g_var", C.c_double), ("g_min", C.c_double),
                ("g_max", C.c_double), ("basal_u", C.c_double), ("bolus_u", C.c_double),
                ("n_samples", C.c_uint32), ("pad", C.c_uint32), ("glucagon_ug", C.c_double),
                ("near_edge", C.c_uint32 * 8)]


STATS_DTYPE = np.dtype([("tir", "<u4", (5,)), ("hypo_episodes", "<u4"), ("q1_clamps", "<u4"),
                        ("status", "<u4"), ("g_mean", "<f8"), ("g_var", "<f8"),
                        ("g_min", "<f8"), ("g_max", "<f8"), ("basal_u", "<f8"),
                        ("bolus_u", "<f8"), ("n_samples", "<u4"), ("pad", "<u4"),
                        ("glucagon_ug", "<f8"), ("near_edge", "<u4", (2, 4))])
assert STATS_DTYPE.itemsize == C.sizeof(Stats)


def compile_source(src: str, out: str) -> str:
    """gcc a source file of the oracle (no FMA contraction, so x86 and Arm agree)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", "-I", _HERE, "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle if its library is missing or older than its sources."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str):
    """Open a build of ``vct_oracle.c`` at ``path`` and declare its entry points."""
    l = C.CDLL(path)
    p = C.c_void_p
    l.vcto_philox4x32_10.argtypes = [p, p, p]
    l.vcto_normals4.argtypes = [p, p, p]
    l.vcto_box_muller.argtypes = [C.c_uint32, C.c_uint32, p]
    l.vcto_basal.argtypes = [p, C.c_double, p, p]
    l.vcto_basal.restype = C.c_int
    l.vcto_create_population.argtypes = [p, C.c_int64, C.c_int64, p, p, p, p, p, C.c_int]
    l.vcto_create_population.restype = C.c_int
    l.vcto_simulate.argtypes = [p, C.c_int64, C.c_int64, p, p, p, p, p, p, p, p, p, p,
                                p, p, C.c_int]
    l.vcto_simulate.restype = C.c_int
    l.vcto_drift.argtypes = [p, p, C.c_double, C.c_double, p]
    return l


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def pop_desc(pop: dict) -> PopDesc:
    d = PopDesc()
    d.bw_mean, d.bw_sd = pop["bw_mean"], pop["bw_sd"]
    for j in range(NPAR):
        d.p_mean[j] = pop["p_mean"][j]
        d.p_sd[j] = pop["p_sd"][j]
    d.g_sp = pop["g_sp"]
    d.min_basal_u_per_h = pop["min_basal_u_per_h"]
    d.sigma_q1 = pop["sigma_q1"]
    d.cgm_sd = pop["cgm_sd"]
    d.seed = pop["seed"]
    d.max_attempts = pop["max_attempts"]
    d.tau_gg_min = float(pop.get("tau_gg_min", 0.0))
    d.s_gg = float(pop.get("s_gg", 0.0))
    return d


def scenario(sc: dict) -> Scenario:
    s = Scenario()
    for f in ("kp_mult", "ki_mult", "kd_mult", "kp_per_ub", "ti_min", "td_min", "i_max",
              "basal_scale", "meal_mean_g", "meal_sd_g"):
        setattr(s, f, float(sc[f]))
    mm = list(sc["meal_minute"])
    for j, v in enumerate(mm):
        s.meal_minute[j] = float(v)
    s.n_meals = len(mm)
    s.bolus = int(sc["bolus"])
    s.horizon = int(sc["horizon_periods"])
    s.stream_id = int(sc.get("stream_id", 0))
    plans = sc.get("day_plans")
    if plans:
        arr = (DayPlan * len(plans))()
        for d, dp in enumerate(plans):
            arr[d].n_meals = len(dp["minute"])
            for j, (m, g) in enumerate(zip(dp["minute"], dp["g_per_kg"])):
                arr[d].minute[j] = m
                arr[d].g_per_kg[j] = g
        s.day_plans = C.cast(arr, C.c_void_p)
        s.n_day_plans = len(plans)
        s.meal_cv = float(sc.get("meal_cv", 0.0))
        s._keep = arr
    s.glucagon = int(bool(sc.get("glucagon", False)))
    s.gg_threshold = float(sc.get("gg_threshold", 0.0))
    s.gg_gain = float(sc.get("gg_gain", 0.0))
    s.gg_max_ug = float(sc.get("gg_max_ug", 0.0))
    return s


# Range edges of Sec. IV-A in mmol/L (54, 70, 180, 250 mg/dL over 18).
EDGES_MMOL = (54.0 / 18.0, 70.0 / 18.0, 180.0 / 18.0, 250.0 / 18.0)
# Default windows of the near-edge counts: 1e-4 x edge (the FP32 form's relative
# tolerance on trajectories) and 1e-3 mg/dL (the stated window of exact range counts).
EDGE_BANDS = (tuple(1e-4 * e for e in EDGES_MMOL), (1e-3 / 18.0,) * 4)


def opts(o: dict) -> Opts:
    r = Opts()
    r.ts_min = float(o.get("ts_min", 5.0))
    r.substeps = int(o.get("substeps", 10))
    r.integrator = int(o.get("integrator", 0))
    r.noise_refine = int(o.get("noise_refine", 1))
    bands = o.get("edge_band", EDGE_BANDS)
    for w in range(2):
        for e in range(4):
            r.edge_band[4 * w + e] = float(bands[w][e])
    return r


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().vcto_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def normals4(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.float64)
    lib().vcto_normals4(_ptr(c), _ptr(k), _ptr(out))
    return out


def box_muller(w0: int, w1: int) -> np.ndarray:
    """The two normals of one Philox word pair."""
    out = np.zeros(2, np.float64)
    lib().vcto_box_muller(int(w0), int(w1), _ptr(out))
    return out


def basal(row, g_sp):
    r = np.ascontiguousarray(row, dtype=np.float64)
    ub = np.zeros(1)
    x0 = np.zeros(NX)
    rc = lib().vcto_basal(_ptr(r), float(g_sp), _ptr(ub), _ptr(x0))
    return rc, float(ub[0]), x0


def drift(row, x, u, d) -> np.ndarray:
    r = np.ascontiguousarray(row, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    f = np.zeros(NX)
    lib().vcto_drift(_ptr(r), _ptr(xx), float(u), float(d), _ptr(f))
    return f


def create_population(pop: dict, n: int | None = None, first: int | None = None,
                      nthreads: int = 0) -> dict:
    n = pop["n_patients"] if n is None else n
    first = pop.get("first_patient", 0) if first is None else first
    nthreads = nthreads or os.cpu_count() or 1
    d = pop_desc(pop)
    rows = np.zeros((n, NROW))
    ub = np.zeros(n)
    x0 = np.zeros((n, NX))
    status = np.zeros(n, np.int32)
    attempts = np.zeros(n, np.int32)
    rc = lib().vcto_create_population(C.byref(d), first, n, _ptr(rows), _ptr(ub), _ptr(x0),
                                      _ptr(status), _ptr(attempts), nthreads)
    if rc != 0:
        raise RuntimeError(f"vcto_create_population failed: {rc}")
    return {"rows": rows, "u_b": ub, "x0": x0, "status": status, "attempts": attempts,
            "first": first}


def simulate(pop: dict, people: dict, sc: dict, o: dict | None = None, *, trace_g=False,
             trace_y=False, trace_u=False, trace_x=False, trace_z=False,
             day_doses=False, nthreads: int = 0) -> dict:
    """Run the closed loop for every patient of ``people`` (from create_population)."""
    o = o or {}
    n = people["rows"].shape[0]
    horizon = int(sc["horizon_periods"])
    nthreads = nthreads or os.cpu_count() or 1
    d, s, op = pop_desc(pop), scenario(sc), opts(o)
    out = np.zeros(n, STATS_DTYPE)
    tg = np.zeros((n, horizon)) if trace_g else None
    ty = np.zeros((n, horizon)) if trace_y else None
    tu = np.zeros((n, horizon)) if trace_u else None
    tx = np.zeros((n, horizon, NX)) if trace_x else None
    tz = np.zeros((n, horizon, 2)) if trace_z else None
    per_day = int(round(1440.0 / float(o.get("ts_min", 5.0))))
    dd = np.zeros((n, horizon // per_day, 3)) if day_doses else None
    rows = np.ascontiguousarray(people["rows"], dtype=np.float64)
    ub = np.ascontiguousarray(people["u_b"], dtype=np.float64)
    x0 = np.ascontiguousarray(people["x0"], dtype=np.float64)
    rc = lib().vcto_simulate(C.byref(d), int(people.get("first", 0)), n, _ptr(rows), _ptr(ub),
                             _ptr(x0), C.byref(s), C.byref(op), _ptr(out), _ptr(tg), _ptr(ty),
                             _ptr(tu), _ptr(tx), _ptr(tz), _ptr(dd), nthreads)
    if rc != 0:
        raise RuntimeError(f"vcto_simulate failed: {rc}")
    res = {"stats": out}
    if trace_g:
        res["g"] = tg
    if trace_y:
        res["y"] = ty
    if trace_u:
        res["u"] = tu
    if trace_x:
        res["x"] = tx
    if trace_z:
        res["z"] = tz
    if day_doses:
        res["day_doses"] = dd
    return res
