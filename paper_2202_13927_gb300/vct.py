"""Thin ctypes binding of ``libvct.so`` (the C-ABI in ``include/vct.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  PyTorch supplies device memory and streams.  If the library is
missing or fails to load, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

NPARAM, NROW, NSTATE, MAX_MEALS, NBINS = 16, 17, 11, 8, 5
FP64, FP32 = 0, 1
TRACE_NONE, TRACE_F16, TRACE_F32, TRACE_F64 = 0, 1, 2, 3
TRACE_CGM, TRACE_BG = 0, 1
PATIENT_NONFINITE, PATIENT_REJECTED = 1, 2
STATUS_NAMES = {0: "VCT_OK", -1: "VCT_ERR_ARG", -2: "VCT_ERR_CUDA", -3: "VCT_ERR_OOM",
                -4: "VCT_ERR_REJECT", -5: "VCT_ERR_TIMEOUT", -6: "VCT_ERR_NONFINITE",
                -7: "VCT_ERR_STATE"}


class VctError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class PopulationDesc(C.Structure):
    _fields_ = [("n_patients", C.c_int64), ("first_patient", C.c_int64), ("seed", C.c_uint64),
                ("bw_mean", C.c_double), ("bw_sd", C.c_double),
                ("p_mean", C.c_double * NPARAM), ("p_sd", C.c_double * NPARAM),
                ("g_sp", C.c_double), ("min_basal_u_per_h", C.c_double),
                ("sigma_q1", C.c_double), ("cgm_sd", C.c_double),
                ("max_attempts", C.c_int32), ("reserved", C.c_int32),
                ("tau_gg_min", C.c_double), ("s_gg", C.c_double)]


class DayPlan(C.Structure):
    _fields_ = [("n_meals", C.c_int32), ("reserved", C.c_int32),
                ("minute", C.c_float * MAX_MEALS), ("g_per_kg", C.c_float * MAX_MEALS)]


class Scenario(C.Structure):
    _fields_ = [("kp_mult", C.c_double), ("ki_mult", C.c_double), ("kd_mult", C.c_double),
                ("kp_per_ub", C.c_double), ("ti_min", C.c_double), ("td_min", C.c_double),
                ("i_max", C.c_double), ("basal_scale", C.c_double),
                ("meal_mean_g", C.c_double), ("meal_sd_g", C.c_double),
                ("meal_minute", C.c_double * MAX_MEALS), ("n_meals", C.c_int32),
                ("bolus", C.c_int32), ("horizon_periods", C.c_int64),
                ("stream_id", C.c_uint32), ("reserved", C.c_uint32),
                ("day_plans", C.c_void_p), ("n_day_plans", C.c_int32), ("meal_cv", C.c_float),
                ("glucagon", C.c_int32), ("reserved2", C.c_int32), ("gg_threshold", C.c_double),
                ("gg_gain", C.c_double), ("gg_max_ug", C.c_double)]


class SimOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("substeps", C.c_int32), ("ts_min", C.c_double),
                ("trace", C.c_void_p), ("trace_patients", C.c_int64),
                ("trace_dtype", C.c_int32), ("trace_kind", C.c_int32),
                ("block_size", C.c_int32), ("patients_per_thread", C.c_int32),
                ("steps_per_chunk", C.c_int32), ("persistent", C.c_int32),
                ("reg_cap", C.c_int32), ("reserved", C.c_int32),
                ("period_begin", C.c_int64), ("period_end", C.c_int64),
                ("state_in", C.c_void_p), ("state_out", C.c_void_p), ("bg_hist", C.c_void_p),
                ("dose_hist", C.c_void_p), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t)]


BG_BINS = 301   # 0.1 mmol/L bins of G(t_k), the last one >= 30 mmol/L
MAX_QUANTILES = 16  # quantiles per vct_dose_quantiles call
DOSE_BINS = 400  # per-day dose bins (Fig. 5), the last one open
DOSE_BIN_WIDTHS = {"basal_u": 0.25, "bolus_u": 0.25, "glucagon_ug": 5.0}


class PatientStats(C.Structure):
    _fields_ = [("tir", C.c_uint32 * NBINS), ("hypo_episodes", C.c_uint32),
                ("q1_clamps", C.c_uint32), ("status", C.c_uint32), ("n_samples", C.c_uint32),
                ("reserved", C.c_uint32), ("g_mean", C.c_double), ("g_var", C.c_double),
                ("g_min", C.c_double), ("g_max", C.c_double), ("basal_u", C.c_double),
                ("bolus_u", C.c_double), ("glucagon_ug", C.c_double)]


class PopulationStats(C.Structure):
    _fields_ = [("n_patients", C.c_int64), ("n_flagged", C.c_int64),
                ("tir_total", C.c_uint64 * NBINS), ("tir_mean", C.c_double * NBINS),
                ("tir_quantile", (C.c_double * 5) * NBINS), ("worst_patient", C.c_int64),
                ("worst_g_min", C.c_double), ("g_mean_mean", C.c_double),
                ("g_mean_var", C.c_double), ("basal_u_mean", C.c_double),
                ("bolus_u_mean", C.c_double), ("horizon_periods", C.c_int64),
                ("below_min", C.c_uint32 * 4), ("below_max", C.c_uint32 * 4),
                ("glucagon_ug_mean", C.c_double)]


class PopulationInfo(C.Structure):
    _fields_ = [("n_patients", C.c_int64), ("first_patient", C.c_int64),
                ("n_rejected", C.c_int64), ("dev_rows", C.c_void_p), ("dev_u_b", C.c_void_p),
                ("dev_x0", C.c_void_p), ("dev_status", C.c_void_p),
                ("dev_attempts", C.c_void_p), ("n_pad", C.c_int64)]


PATIENT_STATS_DTYPE = np.dtype([("tir", "<u4", (5,)), ("hypo_episodes", "<u4"),
                                ("q1_clamps", "<u4"), ("status", "<u4"), ("n_samples", "<u4"),
                                ("reserved", "<u4"), ("g_mean", "<f8"), ("g_var", "<f8"),
                                ("g_min", "<f8"), ("g_max", "<f8"), ("basal_u", "<f8"),
                                ("bolus_u", "<f8"), ("glucagon_ug", "<f8")])
assert PATIENT_STATS_DTYPE.itemsize == C.sizeof(PatientStats)

# name -> (argtypes, restype)
_P = C.c_void_p
SIGNATURES = {
    "vct_last_error": ([], C.c_char_p),
    "vct_version": ([], C.c_char_p),
    "vct_create_population": ([_P, _P, _P], C.c_int),
    "vct_population_from_host": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "vct_destroy_population": ([_P], C.c_int),
    "vct_population_redraw": ([_P, C.c_uint64, _P], C.c_int),
    "vct_population_info_get": ([_P, _P], C.c_int),
    "vct_population_export": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "vct_simulate": ([_P, _P, C.c_int32, _P, _P, _P], C.c_int),
    "vct_state_bytes": ([C.c_int32, C.c_int64], C.c_size_t),
    "vct_stats": ([_P, C.c_int32, C.c_int64, _P, C.c_int64, _P, _P], C.c_int),
    "vct_stats_noalloc": ([_P, C.c_int32, C.c_int64, _P, C.c_int64, _P, _P], C.c_int),
    "vct_stats_noalloc_bytes": ([C.c_int32, C.c_int64, _P], C.c_size_t),
    "vct_stats_with_workspace": ([_P, C.c_int32, C.c_int64, _P, C.c_int64, _P, C.c_size_t, _P, _P],
                                 C.c_int),
    "vct_stats_workspace_bytes": ([C.c_int32, C.c_int64, _P], C.c_size_t),
    "vct_simulate_workspace_bytes": ([_P, _P, C.c_int32, _P, _P], C.c_int),
    "vct_checkpoint": ([_P, _P, C.c_int32, _P, C.c_int64, _P, _P, _P], C.c_int),
    "vct_resume": ([_P, _P, C.c_int32, _P, C.c_int64, _P, _P, _P], C.c_int),
    "vct_bg_cdf": ([_P, C.c_int32, _P, _P], C.c_int),
    "vct_dose_quantiles": ([_P, C.c_int32, _P, C.c_int32, _P, _P], C.c_int),
    "vct_sync": ([_P], C.c_int),
    "vct_philox_fill": ([_P, C.c_int64, C.c_uint64, _P, _P, C.c_int32, _P], C.c_int),
    "vct_box_muller_words": ([_P, C.c_int64, C.c_int32, _P, _P], C.c_int),
    "vct_struct_size": ([C.c_char_p], C.c_size_t),
    "vct_autotune": ([_P, _P, C.c_int32, _P, _P, _P, _P, _P], C.c_int),
    "vct_plan_create": ([_P, _P, C.c_int32, _P, _P, _P, _P], C.c_int),
    "vct_plan_launch": ([_P, _P], C.c_int),
    "vct_plan_opts": ([_P, _P], C.c_int),
    "vct_plan_destroy": ([_P], C.c_int),
    "vct_surrogate_create": ([_P, _P, _P, _P], C.c_int),
    "vct_surrogate_destroy": ([_P], C.c_int),
    "vct_surrogate_n_params": ([], C.c_size_t),
    "vct_surrogate_get": ([_P, _P, _P], C.c_int),
    "vct_surrogate_set": ([_P, _P, _P], C.c_int),
    "vct_surrogate_features": ([_P, _P, _P, C.c_int32, _P, _P], C.c_int),
    "vct_surrogate_step": ([_P, _P, _P, C.c_int64, C.c_int32, _P, _P], C.c_int),
    "vct_surrogate_train": ([_P, _P, _P, C.c_int32, _P, C.c_int32, C.c_uint64, _P, _P], C.c_int),
    "vct_surrogate_predict": ([_P, _P, C.c_int64, _P, _P], C.c_int),
    "vct_surrogate_screen": ([_P, _P, _P, C.c_int64, C.c_int32, _P, _P], C.c_int),
    "vct_surrogate_screen_device": ([_P, _P, _P, C.c_int64, C.c_int32, _P, _P], C.c_int),
    "vct_probe": ([C.c_int32, C.c_int32, _P, _P, _P], C.c_int),
    "vct_surrogate_status": ([_P, _P], C.c_int),
    "vct_surrogate_inject_stall": ([_P, C.c_int32], C.c_int),
    "vct_surrogate_set_lr": ([_P, C.c_double], C.c_int),
}

PROBE_KINDS = {"ffma": 0, "dfma": 1, "imad": 2, "mufu": 3, "imad_hi": 4, "ffma2": 5, "i2f": 6,
               "imad_wide": 7}


def probe(kind: str, iters: int = 4096, stream=None) -> float:
    """Measured rate of one operation kind, in tera lane-operations per second."""
    ms = C.c_float()
    ops = C.c_double()
    _check(load().vct_probe(PROBE_KINDS[kind], iters, C.byref(ms), C.byref(ops),
                            _stream_ptr(stream)))
    return ops.value / (ms.value * 1e-3) / 1e12

SURR_FEATURES, SURR_KF, SURR_HIDDEN = 18, 32, 256


class SurrogateDesc(C.Structure):
    _fields_ = [("batch", C.c_int32), ("reserved", C.c_int32), ("seed", C.c_uint64),
                ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double), ("weight_decay", C.c_double)]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libvct.so (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libvct.so not found at {path}; run paper_2202_13927_gb300.build")
            lib = C.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _check_struct_sizes(lib)
            _lib = lib
    return _lib


def _check_struct_sizes(lib):
    for name, cls in (("vct_population_desc", PopulationDesc), ("vct_scenario", Scenario),
                      ("vct_sim_opts", SimOpts), ("vct_patient_stats", PatientStats),
                      ("vct_population_stats", PopulationStats),
                      ("vct_population_info", PopulationInfo),
                      ("vct_surrogate_desc", SurrogateDesc)):
        got = lib.vct_struct_size(name.encode())
        if got != C.sizeof(cls):
            raise RuntimeError(f"struct {name}: library {got} B, binding {C.sizeof(cls)} B")


def _check(rc: int):
    if rc != 0:
        raise VctError(rc, load().vct_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ------------------------------------------------------------------ marshalling
def population_desc(pop: dict) -> PopulationDesc:
    d = PopulationDesc()
    d.n_patients = int(pop["n_patients"])
    d.first_patient = int(pop.get("first_patient", 0))
    d.seed = int(pop["seed"])
    d.bw_mean, d.bw_sd = float(pop["bw_mean"]), float(pop["bw_sd"])
    for j in range(NPARAM):
        d.p_mean[j] = float(pop["p_mean"][j])
        d.p_sd[j] = float(pop["p_sd"][j])
    d.g_sp = float(pop["g_sp"])
    d.min_basal_u_per_h = float(pop["min_basal_u_per_h"])
    d.sigma_q1 = float(pop["sigma_q1"])
    d.cgm_sd = float(pop["cgm_sd"])
    d.max_attempts = int(pop["max_attempts"])
    d.tau_gg_min = float(pop.get("tau_gg_min", 0.0))
    d.s_gg = float(pop.get("s_gg", 0.0))
    return d


def scenario_struct(sc: dict) -> Scenario:
    s = Scenario()
    for f in ("kp_mult", "ki_mult", "kd_mult", "kp_per_ub", "ti_min", "td_min", "i_max",
              "basal_scale", "meal_mean_g", "meal_sd_g"):
        setattr(s, f, float(sc[f]))
    mm = list(sc["meal_minute"])
    if len(mm) > MAX_MEALS:
        raise ValueError(f"at most {MAX_MEALS} meals per day")
    for j, v in enumerate(mm):
        s.meal_minute[j] = float(v)
    s.n_meals = len(mm)
    s.bolus = int(bool(sc["bolus"]))
    s.horizon_periods = int(sc["horizon_periods"])
    s.stream_id = int(sc.get("stream_id", 0))
    plans = sc.get("day_plans")
    if plans:
        arr = (DayPlan * len(plans))()
        for d, dp in enumerate(plans):
            if len(dp["minute"]) > MAX_MEALS:
                raise ValueError(f"at most {MAX_MEALS} meals per protocol day")
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


def scenario_array(scs) -> C.Array:
    if isinstance(scs, dict):
        scs = [scs]
    arr = (Scenario * len(scs))()
    keep = []
    for i, sc in enumerate(scs):
        st = scenario_struct(sc)
        keep.append(getattr(st, "_keep", None))   # protocol days referenced by pointer
        arr[i] = st
    arr._keep = keep
    return arr


FP64_LIBRARY = 2   # diagnostic normals through the CUDA library's log, sqrt, sincospi
_PRECISION = {"fp64": FP64, "fp32": FP32, FP64: FP64, FP32: FP32, "fp64_library": FP64_LIBRARY}
_TRACE_DTYPES = {None: TRACE_NONE, "f16": TRACE_F16, "f32": TRACE_F32, "f64": TRACE_F64}


def sim_opts(o: dict | None = None, **kw) -> SimOpts:
    o = dict(o or {})
    o.update(kw)
    r = SimOpts()
    r.precision = _PRECISION[o.get("precision", "fp32")]
    r.substeps = int(o.get("substeps", 10))
    r.ts_min = float(o.get("ts_min", 5.0))
    r.trace = o.get("trace_ptr") or None
    r.trace_patients = int(o.get("trace_patients", 0))
    r.trace_dtype = _TRACE_DTYPES[o.get("trace_dtype")]
    r.trace_kind = TRACE_BG if o.get("trace_kind", "cgm") == "bg" else TRACE_CGM
    r.block_size = int(o.get("block_size", 0))
    r.patients_per_thread = int(o.get("patients_per_thread", 0))
    r.steps_per_chunk = int(o.get("steps_per_chunk", 0))
    r.persistent = int(bool(o.get("persistent", False)))
    r.reg_cap = int(o.get("reg_cap", 0))
    r.bg_hist = o.get("bg_hist") or None
    r.dose_hist = o.get("dose_hist") or None
    r.period_begin = int(o.get("period_begin", 0))
    r.period_end = int(o.get("period_end", 0))
    r.state_in = o.get("state_in") or None
    r.state_out = o.get("state_out") or None
    r.workspace = o.get("workspace") or None
    r.workspace_bytes = int(o.get("workspace_bytes", 0))
    return r


# ------------------------------------------------------------------ objects
class Population:
    """A population drawn on the GPU (or uploaded from host arrays)."""

    def __init__(self, handle: int, desc: PopulationDesc):
        self._h = C.c_void_p(handle)
        self.desc = desc

    @classmethod
    def create(cls, pop: dict, stream=None) -> "Population":
        lib = load()
        d = population_desc(pop)
        h = C.c_void_p()
        _check(lib.vct_create_population(C.byref(d), _stream_ptr(stream), C.byref(h)))
        return cls(h.value, d)

    @classmethod
    def from_host(cls, pop: dict, rows, u_b, x0, stream=None) -> "Population":
        lib = load()
        d = population_desc(pop)
        rows = np.ascontiguousarray(rows, np.float64)
        u_b = np.ascontiguousarray(u_b, np.float64)
        x0 = np.ascontiguousarray(x0, np.float64)
        n = d.n_patients
        if rows.shape != (n, NROW) or u_b.shape != (n,) or x0.shape != (n, NSTATE):
            raise ValueError("rows [n,17], u_b [n], x0 [n,11] expected")
        h = C.c_void_p()
        _check(lib.vct_population_from_host(C.byref(d), rows.ctypes.data, u_b.ctypes.data,
                                            x0.ctypes.data, _stream_ptr(stream), C.byref(h)))
        return cls(h.value, d)

    @property
    def handle(self):
        return self._h

    @property
    def n(self) -> int:
        return int(self.desc.n_patients)

    def redraw(self, seed: int, stream=None):
        """A new cohort with another seed, same buffers (asynchronous)."""
        _check(load().vct_population_redraw(self._h, int(seed), _stream_ptr(stream)))
        self.desc.seed = int(seed)

    def info(self) -> PopulationInfo:
        inf = PopulationInfo()
        _check(load().vct_population_info_get(self._h, C.byref(inf)))
        return inf

    def export(self) -> dict:
        n = self.n
        rows = np.zeros((n, NROW))
        ub = np.zeros(n)
        x0 = np.zeros((n, NSTATE))
        status = np.zeros(n, np.uint32)
        attempts = np.zeros(n, np.int32)
        _check(load().vct_population_export(self._h, rows.ctypes.data, ub.ctypes.data,
                                            x0.ctypes.data, status.ctypes.data,
                                            attempts.ctypes.data))
        return {"rows": rows, "u_b": ub, "x0": x0, "status": status, "attempts": attempts,
                "first": int(self.desc.first_patient)}

    def close(self):
        if self._h and self._h.value:
            lib = _lib
            if lib is not None:
                lib.vct_destroy_population(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats_buffer(n_scen: int, n_patients: int, device="cuda"):
    import torch
    return torch.empty(n_scen * n_patients * PATIENT_STATS_DTYPE.itemsize, dtype=torch.uint8,
                       device=device)


def stats_to_numpy(buf) -> np.ndarray:
    return buf.cpu().numpy().view(PATIENT_STATS_DTYPE)


def state_bytes(n_scen: int, n_patients: int) -> int:
    return int(load().vct_state_bytes(n_scen, n_patients))


def simulate(pop: Population, scenarios, opts: dict | None = None, out=None, stream=None,
             **kw):
    """Enqueue the closed-loop simulation; returns the device stats buffer (uint8)."""
    lib = load()
    arr = scenario_array(scenarios)
    o = sim_opts(opts, **kw)
    if out is None:
        out = stats_buffer(len(arr), pop.n)
    if out.numel() < len(arr) * pop.n * PATIENT_STATS_DTYPE.itemsize:
        raise ValueError("stats buffer too small")
    _check(lib.vct_simulate(pop.handle, C.cast(arr, C.c_void_p), len(arr), C.byref(o),
                            out.data_ptr(), _stream_ptr(stream)))
    return out


def simulate_workspace_bytes(pop: Population, scenarios, opts: dict | None = None, **kw) -> int:
    """Device scratch one simulate() call with these arguments needs; passing a
    buffer of that size as opts['workspace'] makes the call allocate nothing."""
    arr = scenario_array(scenarios)
    o = sim_opts(opts, **kw)
    n = C.c_size_t()
    _check(load().vct_simulate_workspace_bytes(pop.handle, C.cast(arr, C.c_void_p), len(arr),
                                               C.byref(o), C.byref(n)))
    return int(n.value)


def checkpoint(pop: Population, scenarios, period_end: int, state_out, opts: dict | None = None,
               out=None, stream=None, **kw):
    """Run up to period_end and write the resumable state into state_out (a
    device buffer of state_bytes()); returns the stats buffer (written only for
    scenarios that end by period_end)."""
    arr = scenario_array(scenarios)
    o = sim_opts(opts, **kw)
    _check(load().vct_checkpoint(pop.handle, C.cast(arr, C.c_void_p), len(arr), C.byref(o),
                                 int(period_end), state_out.data_ptr(),
                                 out.data_ptr() if out is not None else None, _stream_ptr(stream)))
    return out


def resume(pop: Population, scenarios, period_begin: int, state_in, opts: dict | None = None,
           out=None, stream=None, **kw):
    """Continue from a checkpoint's state at period_begin; returns the stats buffer."""
    arr = scenario_array(scenarios)
    o = sim_opts(opts, **kw)
    if out is None:
        out = stats_buffer(len(arr), pop.n)
    _check(load().vct_resume(pop.handle, C.cast(arr, C.c_void_p), len(arr), C.byref(o),
                             int(period_begin), state_in.data_ptr(), out.data_ptr(),
                             _stream_ptr(stream)))
    return out


def sync(stream=None):
    _check(load().vct_sync(_stream_ptr(stream)))


def opts_dict(o: SimOpts) -> dict:
    return {"precision": "fp64" if o.precision == FP64 else "fp32", "substeps": o.substeps,
            "ts_min": o.ts_min, "block_size": o.block_size,
            "patients_per_thread": o.patients_per_thread, "reg_cap": o.reg_cap,
            "steps_per_chunk": o.steps_per_chunk, "persistent": bool(o.persistent)}


def autotune(pop: Population, scenarios, opts: dict | None = None, out=None, stream=None, **kw):
    """Time the launch shapes on a one-day run; returns (chosen options, ms)."""
    lib = load()
    arr = scenario_array(scenarios)
    base = sim_opts(opts, **kw)
    if out is None:
        out = stats_buffer(len(arr), pop.n)
    best = SimOpts()
    ms = C.c_float()
    _check(lib.vct_autotune(pop.handle, C.cast(arr, C.c_void_p), len(arr), C.byref(base),
                            out.data_ptr(), _stream_ptr(stream), C.byref(best), C.byref(ms)))
    return opts_dict(best), ms.value


class Plan:
    """A simulation captured once in a CUDA graph and replayed by launch()."""

    def __init__(self, pop: Population, scenarios, opts: dict | None = None, out=None, stream=None,
                 **kw):
        lib = load()
        self._arr = scenario_array(scenarios)
        self.pop = pop
        self.n_scen = len(self._arr)
        self.out = out if out is not None else stats_buffer(self.n_scen, pop.n)
        o = sim_opts(opts, **kw)
        h = C.c_void_p()
        _check(lib.vct_plan_create(pop.handle, C.cast(self._arr, C.c_void_p), self.n_scen,
                                   C.byref(o), self.out.data_ptr(), _stream_ptr(stream),
                                   C.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(load().vct_plan_launch(self._h, _stream_ptr(stream)))
        return self.out

    def opts(self) -> dict:
        o = SimOpts()
        _check(load().vct_plan_opts(self._h, C.byref(o)))
        return opts_dict(o)

    def close(self):
        if self._h and self._h.value and _lib is not None:
            _lib.vct_plan_destroy(self._h)
        self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def population_stats(dev_stats, n_scen: int, n_patients: int, horizons, first_patient: int = 0,
                     stream=None) -> list[dict]:
    """Population reductions on the GPU; returns one dict per scenario."""
    lib = load()
    hz = np.ascontiguousarray(np.asarray(horizons, np.int64).reshape(-1))
    if hz.size != n_scen:
        raise ValueError("one horizon per scenario")
    res = (PopulationStats * n_scen)()
    ptr = dev_stats.data_ptr() if hasattr(dev_stats, "data_ptr") else int(dev_stats or 0)
    _check(lib.vct_stats(ptr, n_scen, n_patients, hz.ctypes.data, first_patient,
                         C.cast(res, C.c_void_p), _stream_ptr(stream)))
    return [population_stats_dict(r) for r in res]


def population_stats_noalloc(dev_stats, n_scen: int, n_patients: int, horizons,
                             first_patient: int = 0, stream=None) -> list[dict]:
    """population_stats through vct_stats_noalloc: no device allocation; its
    scratch is the library's fixed 8 MiB device array, shared by all calls
    (serialise calls that could overlap on the GPU)."""
    lib = load()
    hz = np.ascontiguousarray(np.asarray(horizons, np.int64).reshape(-1))
    if hz.size != n_scen:
        raise ValueError("one horizon per scenario")
    res = (PopulationStats * n_scen)()
    ptr = dev_stats.data_ptr() if hasattr(dev_stats, "data_ptr") else int(dev_stats or 0)
    _check(lib.vct_stats_noalloc(ptr, n_scen, n_patients, hz.ctypes.data, first_patient,
                                 C.cast(res, C.c_void_p), _stream_ptr(stream)))
    return [population_stats_dict(r) for r in res]


def population_stats_dict(r: PopulationStats) -> dict:
    return {
        "n_patients": r.n_patients, "n_flagged": r.n_flagged,
        "tir_total": np.array(list(r.tir_total), np.uint64),
        "tir_mean": np.array(list(r.tir_mean)),
        "tir_quantile": np.array([[r.tir_quantile[b][q] for q in range(5)] for b in range(NBINS)]),
        "worst_patient": r.worst_patient, "worst_g_min": r.worst_g_min,
        "g_mean_mean": r.g_mean_mean, "g_mean_var": r.g_mean_var,
        "basal_u_mean": r.basal_u_mean, "bolus_u_mean": r.bolus_u_mean,
        "glucagon_ug_mean": r.glucagon_ug_mean,
        "horizon_periods": r.horizon_periods,
        "below_min": np.array(list(r.below_min), np.uint32),
        "below_max": np.array(list(r.below_max), np.uint32),
    }


def bg_cdf(dev_hist, n_scen: int = 1, stream=None) -> np.ndarray:
    """Mean BG curve of Fig. 3 from the device BG histograms a simulation filled
    ([n_scen][BG_BINS]): the fraction of binned samples below each bin's upper
    edge (0.1, 0.2, ... mmol/L), computed by vct_bg_cdf.  Returns
    [n_scen][BG_BINS] (one row squeezed when n_scen == 1)."""
    import torch
    if not (isinstance(dev_hist, torch.Tensor) and dev_hist.is_cuda):
        raise ValueError("bg_cdf takes the device histogram")
    if dev_hist.numel() < n_scen * BG_BINS or dev_hist.element_size() != 4 or not dev_hist.is_contiguous():
        raise ValueError("histogram: contiguous 32-bit [n_scen][BG_BINS]")
    out = torch.empty((n_scen, BG_BINS), dtype=torch.float64, device=dev_hist.device)
    _check(load().vct_bg_cdf(dev_hist.data_ptr(), n_scen, out.data_ptr(), _stream_ptr(stream)))
    res = out.cpu().numpy()
    return res[0] if n_scen == 1 else res


def dose_quantiles(dev_hist, n_scen: int = 1, qs=(0.05, 0.5, 0.95), stream=None) -> np.ndarray:
    """Quantiles of the daily doses of Fig. 5 from the device daily-dose
    histograms a simulation filled ([n_scen][3][DOSE_BINS]), computed by
    vct_dose_quantiles: [n_scen][3][len(qs)] (basal U, bolus U, glucagon ug)."""
    import torch
    if not (isinstance(dev_hist, torch.Tensor) and dev_hist.is_cuda):
        raise ValueError("dose_quantiles takes the device histogram")
    if dev_hist.numel() < n_scen * 3 * DOSE_BINS or dev_hist.element_size() != 4 or not dev_hist.is_contiguous():
        raise ValueError("histogram: contiguous 32-bit [n_scen][3][DOSE_BINS]")
    q = np.ascontiguousarray(np.asarray(qs, np.float64).reshape(-1))
    out = torch.empty((n_scen, 3, q.size), dtype=torch.float64, device=dev_hist.device)
    _check(load().vct_dose_quantiles(dev_hist.data_ptr(), n_scen, q.ctypes.data, q.size,
                                     out.data_ptr(), _stream_ptr(stream)))
    return out.cpu().numpy()


def population_stats_with_workspace(dev_stats, n_scen: int, n_patients: int, horizons, workspace,
                                    first_patient: int = 0, stream=None) -> list[dict]:
    """population_stats with caller-owned device scratch (no allocation in the call)."""
    lib = load()
    hz = np.ascontiguousarray(np.asarray(horizons, np.int64).reshape(-1))
    if hz.size != n_scen:
        raise ValueError("one horizon per scenario")
    res = (PopulationStats * n_scen)()
    ptr = dev_stats.data_ptr() if hasattr(dev_stats, "data_ptr") else int(dev_stats or 0)
    _check(lib.vct_stats_with_workspace(ptr, n_scen, n_patients, hz.ctypes.data, first_patient,
                                        workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                        C.cast(res, C.c_void_p), _stream_ptr(stream)))
    return [population_stats_dict(r) for r in res]


def stats_workspace_bytes(n_scen: int, n_patients: int, horizons) -> int:
    hz = np.ascontiguousarray(np.asarray(horizons, np.int64).reshape(-1))
    return int(load().vct_stats_workspace_bytes(n_scen, n_patients, hz.ctypes.data))


def stats_noalloc_bytes(n_scen: int, n_patients: int, horizons) -> int:
    hz = np.ascontiguousarray(np.asarray(horizons, np.int64).reshape(-1))
    return int(load().vct_stats_noalloc_bytes(n_scen, n_patients, hz.ctypes.data))


def replay(pop: dict, scenario: dict, patient: int, opts: dict | None = None,
           trace_kind: str = "bg", trace_dtype: str = "f64", bg_hist: bool = False):
    """Re-simulate one patient (global id) with a trace, e.g. the worst-case
    patient that vct_stats reports.  Every draw is keyed by the global id, so
    this equals that patient's run inside the whole population.  With bg_hist
    the kernel also bins the patient's samples into a device BG histogram
    (returned third), the input of that patient's curve of Fig. 3."""
    import copy

    import torch
    one = copy.deepcopy(pop)
    one["n_patients"] = 1
    one["first_patient"] = int(patient)
    gp = Population.create(one)
    H = int(scenario["horizon_periods"])
    dt = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16}[trace_dtype]
    tr = torch.zeros((H, 1), dtype=dt, device="cuda")
    o = dict(opts or {})
    o.update(trace_ptr=tr.data_ptr(), trace_patients=1, trace_dtype=trace_dtype,
             trace_kind=trace_kind)
    hist = None
    if bg_hist:
        hist = torch.zeros(BG_BINS, dtype=torch.int32, device="cuda")
        o["bg_hist"] = hist.data_ptr()
    out = simulate(gp, scenario, o)
    sync()
    res = stats_to_numpy(out)[0], tr[:, 0].cpu().numpy().astype(np.float64)
    gp.close()
    return res + (hist,) if bg_hist else res


def philox_fill(ctr, seed: int, precision: str = "fp64", stream=None):
    """Device Philox words and normals for counters ctr (torch uint32-as-int32 [n, 4])."""
    import torch
    lib = load()
    n = ctr.shape[0]
    words = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    dt = torch.float32 if _PRECISION[precision] == FP32 else torch.float64
    normals = torch.empty((n, 4), dtype=dt, device=ctr.device)
    _check(lib.vct_philox_fill(ctr.data_ptr(), n, seed, words.data_ptr(), normals.data_ptr(),
                               _PRECISION[precision], _stream_ptr(stream)))
    return words, normals


def box_muller_words(words, mode: str = "own", stream=None):
    """FP64 Box-Muller normals of device word pairs (uint32-as-int32 [n, 2]):
    mode 'own' = the simulation's transform, 'library' = the CUDA library's."""
    import torch
    n = words.shape[0]
    z = torch.empty((n, 2), dtype=torch.float64, device=words.device)
    _check(load().vct_box_muller_words(words.data_ptr(), n, {"own": 0, "library": 1}[mode],
                                       z.data_ptr(), _stream_ptr(stream)))
    return z


# ------------------------------------------------------------------ surrogate
def unpack_weights(flat: np.ndarray) -> dict:
    """Packed FP32 vector -> W1 [256][18], b1, W2 [256][256], b2, W3 [5][256], b3."""
    h, f = SURR_HIDDEN, SURR_FEATURES
    sizes = [("W1", (h, f)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)), ("W3", (NBINS, h)),
             ("b3", (NBINS,))]
    out, o = {}, 0
    for k, shp in sizes:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n]).reshape(shp)
        o += n
    return out


def pack_weights(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float32).ravel()
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


class Surrogate:
    """The learned surrogate of the closed loop (see include/vct.h)."""

    def __init__(self, scale_pop: dict, batch: int = 4096, seed: int = 0, lr: float = 1e-3,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 weight_decay: float = 0.01, stream=None):
        lib = load()
        d = SurrogateDesc()
        d.batch, d.seed, d.lr, d.beta1, d.beta2, d.eps, d.weight_decay = (
            int(batch), int(seed), lr, beta1, beta2, eps, weight_decay)
        sc = population_desc(scale_pop)
        h = C.c_void_p()
        _check(lib.vct_surrogate_create(C.byref(d), C.byref(sc), _stream_ptr(stream), C.byref(h)))
        self._h = h
        self.batch = int(batch)
        self.n_params = int(lib.vct_surrogate_n_params())

    def weights(self) -> np.ndarray:
        w = np.zeros(self.n_params, np.float32)
        _check(load().vct_surrogate_get(self._h, w.ctypes.data, None))
        return w

    def grads(self) -> np.ndarray:
        g = np.zeros(self.n_params, np.float32)
        _check(load().vct_surrogate_get(self._h, None, g.ctypes.data))
        return g

    def set_weights(self, w, stream=None):
        w = np.ascontiguousarray(w, np.float32)
        assert w.size == self.n_params
        _check(load().vct_surrogate_set(self._h, w.ctypes.data, _stream_ptr(stream)))

    def features(self, pop: Population, scenarios, stream=None):
        import torch
        arr = scenario_array(scenarios)
        x = torch.empty((len(arr) * pop.n, SURR_KF), dtype=torch.float32, device="cuda")
        _check(load().vct_surrogate_features(self._h, pop.handle, C.cast(arr, C.c_void_p), len(arr),
                                             x.data_ptr(), _stream_ptr(stream)))
        return x

    def step(self, x, t, update: bool = False, stream=None) -> float:
        loss = C.c_double()
        _check(load().vct_surrogate_step(self._h, x.data_ptr(), t.data_ptr(), x.shape[0],
                                         int(update), C.byref(loss), _stream_ptr(stream)))
        return loss.value

    def train(self, pop: Population, scenarios, dev_stats, epochs: int, shuffle_seed: int = 0,
              stream=None) -> np.ndarray:
        arr = scenario_array(scenarios)
        losses = np.zeros(max(epochs, 1))
        _check(load().vct_surrogate_train(self._h, pop.handle, C.cast(arr, C.c_void_p), len(arr),
                                          dev_stats.data_ptr(), epochs, shuffle_seed,
                                          losses.ctypes.data, _stream_ptr(stream)))
        return losses[:epochs]

    def set_lr(self, lr: float):
        """Learning rate of the following AdamW steps (moments and step count carry on)."""
        _check(load().vct_surrogate_set_lr(self._h, float(lr)))

    def inject_stall(self, on: bool = True):
        """Test hook: make the next forward passes' bounded waits run out."""
        _check(load().vct_surrogate_inject_stall(self._h, int(bool(on))))

    def status(self, stream=None) -> int:
        """0, or raises VctError(VCT_ERR_TIMEOUT) if a forward pass gave up a
        bounded wait on the tensor cores (synchronises the stream)."""
        _check(load().vct_surrogate_status(self._h, _stream_ptr(stream)))
        return 0

    def predict(self, x, stream=None):
        import torch
        p = torch.empty((x.shape[0], NBINS), dtype=torch.float32, device=x.device)
        _check(load().vct_surrogate_predict(self._h, x.data_ptr(), x.shape[0], p.data_ptr(),
                                            _stream_ptr(stream)))
        return p

    def screen(self, panel: Population, gains, bin: int = 2, stream=None):
        """Scores of candidate gains [n][3]: host values (numpy) or a CUDA FP64
        tensor already on the device (then nothing runs on the host)."""
        import torch
        if isinstance(gains, torch.Tensor) and gains.is_cuda:
            g = gains.reshape(-1, 3)
            if g.dtype != torch.float64 or not g.is_contiguous():
                raise ValueError("device gains must be a contiguous float64 tensor")
            scores = torch.empty(g.shape[0], dtype=torch.float32, device=g.device)
            _check(load().vct_surrogate_screen_device(self._h, panel.handle, g.data_ptr(), g.shape[0],
                                                      bin, scores.data_ptr(), _stream_ptr(stream)))
            return scores
        g = np.ascontiguousarray(np.asarray(gains, np.float64).reshape(-1, 3))
        scores = torch.empty(g.shape[0], dtype=torch.float32, device="cuda")
        _check(load().vct_surrogate_screen(self._h, panel.handle, g.ctypes.data, g.shape[0], bin,
                                           scores.data_ptr(), _stream_ptr(stream)))
        return scores

    def close(self):
        if self._h and self._h.value and _lib is not None:
            _lib.vct_surrogate_destroy(self._h)
        self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
