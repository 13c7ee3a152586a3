"""Benchmark: simulated patient-years per second of the closed-loop trial.

One step = one whole virtual trial on the GPU through the C-ABI: draw the
population (parameters + FP64 basal steady state), simulate every patient in
closed loop for the horizon (FP32 fast form, persistent launch), reduce the
population indicators.  Default workload: the paper's trial shape, 1,000,000
patients x 52 weeks (104,832 control periods of 5 min, 10 Euler-Maruyama
steps of 30 s each).  One patient-year := 52 weeks.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch one process per GPU with torch.distributed.run; each rank
simulates its own block of global patient ids (weak scaling) and rank 0
gathers the per-patient records for the final population reduction.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PATIENT_YEAR = 104_832          # control periods in 52 weeks
# Algorithmic operations per control period of the FP32 form with m = 10,
# counted from the method: 10 Euler steps x 25 (chain variables held scaled,
# F01c and F_R as one min or max and one fma each), 3 Philox4x32-10 calls x 55
# + 2, Box-Muller for 11 normals (81), controller, indicators and bookkeeping (56).
OPS_PER_PERIOD_FP32 = 10 * 25 + 3 * 55 + 2 + 81 + 56
# FP64 form: the same step, 25 FP64 operations per Euler step.
FP64_OPS_PER_PERIOD = 10 * 25
# FP64 operations the FP64 form executes per patient-period, its own Box-Muller
# transform (table-driven log, Newton reciprocal square root, reduced angle)
# included: (DFMA + DADD + DMUL) thread instructions of one Nsight Compute
# capture of 100,000 patients x 2016 periods, (55.346e9 + 9.098e9 + 14.351e9) / 2.016e8.
FP64_OPS_PER_PERIOD_EXECUTED = (55.346e9 + 9.098e9 + 14.351e9) / 2.016e8
SMS, LANES_PER_SM = 152, 128     # GB300: 152 SMs x 4 schedulers x 32 lanes
# DRAM bytes (read + write) per patient of the FP32 m = 10 kernel with one patient
# per thread and the 128-register cap (the lean variant: no trace, BG histogram or
# protocol), from one Nsight Compute capture of 160,000 patients x 2016 periods in
# 128-thread blocks (37,840,896 B read + 28,416 B written); the kernel reads each
# patient's parameters and initial state once, so a launch moves this x its
# patients whatever its block size.
TRAFFIC_PER_PATIENT = (37_840_896 + 28_416) / 160_000
TRAFFIC_SHAPE = (1, 128)          # patients per thread, register cap of that capture
# Executed thread-instructions per patient-period of that kernel on each
# pipe, from the same capture (sm__inst_executed_pipe_*.sum and
# smsp__inst_executed.sum, x 32 lanes, over the 3.2256e8 patient-periods).
# Of the fmaheavy count, IMAD_HI_PER_PERIOD are Philox's high-half products
# (the M1 product of 3 calls x 9 rounds, and the next period's counter) and
# IMAD_WIDE_PER_PERIOD its widening products (the M0 product of the same
# rounds), which that pipe runs at their own, lower rates.
PIPE_INST_PER_PERIOD = {"issue": 595.01, "fmaheavy": 186.06, "fmalite": 194.57, "alu": 175.78,
                        "xu": 23.05, "fp64": 1.26}
IMAD_HI_PER_PERIOD = 28
IMAD_WIDE_PER_PERIOD = 27


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _per_pipe_bound(probes, issue_tops, measured_s_per_period):
    """Lower bound of the FP32 kernel's time per patient-period from each pipe:
    its executed instructions divided by that pipe's measured rate (T lane-ops/s:
    issue = SMs x 128 lanes x clock; fmaheavy and fmalite, 64 lanes each, at the
    INT32 multiply-add probe's rate, the high-half and widening products at
    theirs; ALU, 64
    lanes, at half the issue rate; XU at the MUFU probe; FP64 at the DFMA
    probe).  The largest bound is the one that binds; frac = bound / measured."""
    c = PIPE_INST_PER_PERIOD
    ps = {"issue": c["issue"] / issue_tops,
          "fmaheavy": ((c["fmaheavy"] - IMAD_HI_PER_PERIOD - IMAD_WIDE_PER_PERIOD) / probes["imad"]
                       + IMAD_HI_PER_PERIOD / probes["imad_hi"] + IMAD_WIDE_PER_PERIOD / probes["imad_wide"]),
          "fmalite": c["fmalite"] / probes["imad"],
          "alu": c["alu"] / (issue_tops / 2.0),
          "xu": c["xu"] / probes["mufu"],
          "fp64": c["fp64"] / probes["dfma"]}
    binding = max(ps, key=ps.get)
    meas = measured_s_per_period * 1e12
    return {"ps_per_patient_period": {k: round(v, 3) for k, v in ps.items()}, "binding": binding,
            "bound_ps": round(ps[binding], 3), "measured_ps": round(meas, 3), "frac": ps[binding] / meas,
            "basis": "executed instructions per pipe (ncu, 160,000 x 2016 capture) / measured pipe rates"}


def _cpu_oracle_rate(pop, sc, n_sample, days, nthreads):
    """Patient-years/s of the FP64 oracle on the host cores, bounded sample."""
    from oracle import oracle as O
    from paper_2202_13927_gb300 import workloads as W
    sub_sc = W.with_changes(sc, horizon_periods=int(days * W.PERIODS_PER_DAY))
    people = O.create_population(pop, n=n_sample, first=pop.get("first_patient", 0), nthreads=nthreads)
    t0 = time.perf_counter()
    res = O.simulate(pop, people, sub_sc, {}, nthreads=nthreads)
    dt = time.perf_counter() - t0
    py = n_sample * sub_sc["horizon_periods"] / PATIENT_YEAR
    return py / dt, dt, f"{n_sample} patients x {days} days of the same trial", res["stats"]


def _error_per_statistic(vct, W, pop, sc, oracle_stats, days, shape, stream):
    """The GPU's FP32 and FP64 forms against the oracle's records of the same
    patients (the CPU-baseline sample): error per statistic, and the
    deviation of the range fractions in percentage points."""
    import numpy as np
    n = len(oracle_stats)
    sub_pop = W.with_changes(pop, n_patients=n)
    sub_sc = W.with_changes(sc, horizon_periods=int(days * W.PERIODS_PER_DAY))
    gp = vct.Population.create(sub_pop, stream=stream)
    o = oracle_stats
    ok = o["status"] == 0
    out = {"patients": int(ok.sum()), "days": days}
    for prec, kw in (("fp32", dict(persistent=True, **shape)), ("fp64", {})):
        st = vct.stats_to_numpy(vct.simulate(gp, sub_sc, dict(precision=prec, **kw), stream=stream))
        g = st[ok]
        r = o[ok]
        rep_ = {"status_equal": bool(np.array_equal(st["status"], o["status"]))}
        for f in ("g_mean", "g_var", "g_min", "g_max", "basal_u", "bolus_u"):
            rel = np.abs(g[f] - r[f]) / np.maximum(np.abs(r[f]), 1e-12)
            rep_[f] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean())}
        fg = g["tir"] / g["n_samples"][:, None]
        fr = r["tir"] / r["n_samples"][:, None]
        rep_["tir_fraction_pp"] = {"max_abs_per_patient": float(100 * np.abs(fg - fr).max()),
                                   "population_mean_per_range": [round(float(x), 6) for x in
                                                                 100 * (fg.mean(0) - fr.mean(0))]}
        rep_["tir_counts_equal_fraction"] = float(np.mean(np.all(g["tir"] == r["tir"], axis=1)))
        dh = np.abs(g["hypo_episodes"].astype(np.int64) - r["hypo_episodes"].astype(np.int64))
        rep_["hypo_episodes_mean_abs_diff"] = float(dh.mean())
        rep_["hypo_episodes_max_abs_diff"] = int(dh.max())
        # every count difference explained by the oracle's samples near that edge?
        # per edge e: |samples >= e (GPU) - (oracle)| <= oracle samples within the
        # window of e; hypo episodes: |difference| <= samples near 70 mg/dL
        cg = np.cumsum(g["tir"].astype(np.int64)[:, ::-1], axis=1)[:, ::-1][:, 1:]
        cr = np.cumsum(r["tir"].astype(np.int64)[:, ::-1], axis=1)[:, ::-1][:, 1:]
        expl = {}
        for w, name in enumerate(("window_1e-4_x_edge", "window_1e-3_mg_dl")):
            near = r["near_edge"][:, w, :].astype(np.int64)
            ok_r = np.all(np.abs(cg - cr) <= near, axis=1)
            ok_h = dh <= near[:, 1]
            expl[name] = {"ranges_explained_fraction": float(ok_r.mean()),
                          "hypo_explained_fraction": float(ok_h.mean()),
                          "unexplained_range_moves_per_patient": float(
                              np.maximum(np.abs(cg - cr) - near, 0).sum(axis=1).mean())}
        rep_["near_edge_explanation"] = expl
        out[prec] = rep_
    gp.close()
    return out


def _batched_uneven(vct, W, stream):
    """256 scenarios x 4,096 patients, horizons 1-52 weeks: one persistent,
    graph-captured, autotuned launch."""
    import torch
    pop, scs = W.batched_uneven()
    gp = vct.Population.create(pop, stream=stream)
    plan = vct.Plan(gp, scs, {"precision": "fp32", "persistent": True}, stream=stream)
    plan.launch(stream=stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.launch(stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    s = a.elapsed_time(b) / 1000.0
    periods = sum(sc["horizon_periods"] for sc in scs) * pop["n_patients"]
    out = {"value": periods / PATIENT_YEAR / s, "unit": "patient-years/s", "launch_ms": 1000 * s,
           "scenarios": len(scs), "patients_per_scenario": pop["n_patients"],
           "patient_years": periods / PATIENT_YEAR, "launch": plan.opts()}
    plan.close()
    gp.close()
    return out


def _cgm_trace(vct, W, stream, shape):
    """The paper-scale trial with the CGM traces of its first 10,000 patients
    kept in FP16 (time-major, 2.1 GB): the trace's cost and write rate."""
    import torch
    pop, sc, opts = W.workload("paper_scale")
    H, n_tr = sc["horizon_periods"], 10_000
    gp = vct.Population.create(pop, stream=stream)
    tr = torch.empty((H, n_tr), dtype=torch.float16, device="cuda")
    kw = dict(opts, persistent=True, **shape)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    times = {}
    for name, extra in (("plain", {}), ("traced", {"trace_ptr": tr.data_ptr(), "trace_patients": n_tr,
                                                   "trace_dtype": "f16", "trace_kind": "cgm"})):
        out = vct.simulate(gp, sc, dict(kw, **extra), stream=stream)   # warm-up
        torch.cuda.synchronize()
        a.record(stream)
        vct.simulate(gp, sc, dict(kw, **extra), out=out, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        times[name] = a.elapsed_time(b) / 1000.0
    ok = bool(torch.isfinite(tr[-1]).all().item())
    gp.close()
    nbytes = H * n_tr * 2
    return {"traced_patients": n_tr, "trace_bytes": nbytes, "launch_s": times["traced"],
            "plain_launch_s": times["plain"], "overhead_pct": 100.0 * (times["traced"] / times["plain"] - 1.0),
            "trace_write_gbs": nbytes / times["traced"] / 1e9, "last_row_finite": ok}


def _trial_a_vs_b(vct, W, stream):
    """The paper's experiment (Sec. IV): 1,000,000 patients x 52 weeks on the
    year protocol, trial A (correct basal) and trial B (basal 50 % low), both
    arms in one plan with common random numbers, the controller with its
    glucagon mode (the paper's AP is dual-hormone)."""
    import numpy as np
    import torch
    pop, _, _ = W.workload("paper_scale")
    arms = [W.protocol_scenario(364, meal_cv=0.1, glucagon=True),
            W.protocol_scenario(364, meal_cv=0.1, basal_scale=0.5, glucagon=True)]
    gp = vct.Population.create(pop, stream=stream)
    dose = torch.zeros(2 * 3 * vct.DOSE_BINS, dtype=torch.int32, device="cuda")   # Fig. 5
    plan = vct.Plan(gp, arms, {"precision": "fp32", "persistent": True,
                               "dose_hist": dose.data_ptr()}, stream=stream)
    dose.zero_()                              # the autotuner's trial runs added to it
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.launch(stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    s = a.elapsed_time(b) / 1000.0
    summ = vct.population_stats(plan.out, 2, pop["n_patients"], [a_["horizon_periods"] for a_ in arms],
                                stream=stream)
    out = {"value": 2 * pop["n_patients"] * 364 / 364 / s, "unit": "patient-years/s",
           "launch_s": s, "arms": {}}
    dq = vct.dose_quantiles(dose, 2, (0.05, 0.5, 0.95), stream=stream)   # Fig. 5, in the library
    recs = vct.stats_to_numpy(plan.out).reshape(2, pop["n_patients"])
    for name, sm, q, r in zip(("A", "B"), summ, dq, recs):
        out["arms"][name] = {"tir_mean_pct": [round(100 * x, 2) for x in sm["tir_mean"]],
                             "tir_70_180_median_pct": round(100 * sm["tir_quantile"][2][2], 2),
                             "worst_patient": sm["worst_patient"],
                             "worst_g_min": round(sm["worst_g_min"], 3),
                             "basal_u_per_day": round(sm["basal_u_mean"] / 364, 3),
                             "bolus_u_per_day": round(sm["bolus_u_mean"] / 364, 3),
                             "glucagon_ug_per_day": round(sm["glucagon_ug_mean"] / 364, 3),
                             "daily_dose_p5_p50_p95": {
                                 k: [round(float(v), 2) for v in q[j]]
                                 for j, k in enumerate(vct.DOSE_BIN_WIDTHS)},
                             # patients the Q1 clamp (G = 0) ever caught, and below 54 mg/dL
                             "patients_q1_clamped": int((r["q1_clamps"] > 0).sum()),
                             "patients_below_54_mg_dl": int((r["tir"][:, 0] > 0).sum()),
                             "patients_below_54_over_1pct": int((r["tir"][:, 0] > 0.01 * r["n_samples"]).sum())}
    out["launch"] = plan.opts()
    plan.close()
    gp.close()
    return out


def _surrogate(vct, W, stream, peaks):
    """Screening 1e6 controller tunings on a 128-patient panel, and training steps."""
    import numpy as np
    import torch
    panel_pop = W.population(128, 5)
    gp = vct.Population.create(panel_pop, stream=stream)
    s = vct.Surrogate(panel_pop, batch=4096, seed=1)
    g = np.exp(np.random.default_rng(0).uniform(np.log(0.3), np.log(3.0), size=(1_000_000, 3)))
    gd = torch.from_numpy(g).cuda()          # candidates resident in HBM
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        s.screen(gp, gd, stream=stream)
    torch.cuda.synchronize()
    a.record(stream)
    s.screen(gp, gd, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    s.status()
    # end to end: host gains, copied in by the call
    a.record(stream)
    s.screen(gp, g, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms_host = a.elapsed_time(b)
    rows = g.shape[0] * 128
    flop = rows * 2 * (18 * 256 + 256 * 256 + 256 * 5)   # the model's 18 -> 256 -> 256 -> 5
    tf = flop / ms / 1e9
    x = torch.randn(4096, 32, device="cuda")
    x[:, 18:] = 0
    t = torch.softmax(torch.randn(4096, 5, device="cuda"), 1)
    for _ in range(3):
        s.step(x, t, update=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(20):
        s.step(x, t, update=True)
    b.record(stream)
    torch.cuda.synchronize()
    step_ms = a.elapsed_time(b) / 20
    s.close()
    gp.close()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    return {"screen_candidates": g.shape[0], "panel": 128, "screen_ms": ms,
            "screen_ms_host_gains": ms_host,
            "screen_rows_per_s": rows / ms * 1e3,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": bf16, "unit": "TFLOP/s",
                         "frac": tf / bf16, "kernel": "forward_kernel<screen>"},
            "train_step_ms": step_ms, "train_samples_per_s": 4096 / step_ms * 1e3}


def _surrogate_workflow(vct, W, stream, shape):
    """The learned surrogate's workflow: train on 2,097,152 four-week
    closed-loop runs (2,048 PID tunings x 1,024 patients), screen 10^6
    tunings on a 128-patient panel, and judge it by full simulation on one
    verification cohort (10,000 patients x 52 weeks):
      * equal simulation budget: for k = 10, 100, 1000 the best verified TIR of
        the surrogate's top k against the best of k random tunings (the search
        without the network), with the cohort's standard error;
      * the surrogate's error on its top 1,000 split into (i) the network
        against its own target (the panel's simulated 28-day TIR), (ii) the
        panel against the verification cohort (both 28 days), (iii) 28 days
        against 52 weeks on the cohort;
      * the training loss per epoch minus the entropy of the targets (the
        Kullback-Leibler divergence the training can still remove)."""
    import numpy as np
    import torch
    rng = np.random.default_rng(50)
    lg = lambda n: np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=(n, 3)))
    tune = lambda g, days: W.scenario(days, kp_mult=g[0], ki_mult=g[1], kd_mult=g[2])
    sim_kw = dict(precision="fp32", persistent=True, **shape)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ev[0].record(stream)
        r = fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return r, ev[0].elapsed_time(ev[1]) / 1000.0

    def tir_of(stats, n_scen, n_pat):
        st = vct.stats_to_numpy(stats)
        f = (st["tir"][:, 2] / np.maximum(st["n_samples"], 1)).reshape(n_scen, n_pat)
        return f.mean(axis=1), f.std(axis=1) / np.sqrt(n_pat)

    train_pop = W.population(1024, 51)
    gp = vct.Population.create(train_pop, stream=stream)
    g_train = lg(2048)
    scs = [tune(g, 28) for g in g_train]
    stats, t_sim = timed(lambda: vct.simulate(gp, scs, sim_kw, stream=stream))
    tr = vct.stats_to_numpy(stats)
    t = tr["tir"] / np.maximum(tr["n_samples"], 1)[:, None]
    entropy = float(np.mean(-np.sum(np.where(t > 0, t * np.log(np.where(t > 0, t, 1.0)), 0.0), axis=1)))
    s = vct.Surrogate(train_pop, batch=4096, seed=52, lr=2e-3)
    schedule = ((12, 2e-3), (12, 6e-4), (8, 2e-4))    # epochs at each learning rate

    def train_all():
        out = []
        for j, (ep, lr) in enumerate(schedule):
            s.set_lr(lr)
            out.append(s.train(gp, scs, stats, epochs=ep, shuffle_seed=53 + j, stream=stream))
        return np.concatenate(out)
    losses, t_train = timed(train_all)
    epochs = int(sum(ep for ep, _ in schedule))
    panel_pop = W.population(128, 54)
    panel = vct.Population.create(panel_pop, stream=stream)
    cand = torch.from_numpy(lg(1_000_000)).cuda()
    scores, t_screen = timed(lambda: s.screen(panel, cand, bin=2, stream=stream))
    s.status()
    pred = scores.cpu().numpy().astype(np.float64)
    order = np.argsort(-pred)
    top = order[:1000]
    g_cand = cand.cpu().numpy()
    rand = rng.choice(len(g_cand), 1000, replace=False)
    verify_g = np.concatenate([g_cand[top], g_cand[rand], np.ones((1, 3))])
    vpop = W.population(10_000, 55)
    vgp = vct.Population.create(vpop, stream=stream)
    nv = vpop["n_patients"]
    vscs = [tune(g, 364) for g in verify_g]
    vstats, t_verify = timed(lambda: vct.simulate(vgp, vscs, sim_kw, stream=stream))
    tir, se = tir_of(vstats, len(vscs), nv)
    t_top, t_rand, t_nom = tir[:1000], tir[1000:2000], float(tir[-1])
    se_top = se[:1000]
    # the error split on the top 1,000: panel at 28 days, cohort at 28 days
    pscs = [tune(g, 28) for g in g_cand[top]]
    p28, _ = tir_of(vct.simulate(panel, pscs, sim_kw, stream=stream), 1000, panel_pop["n_patients"])
    c28, _ = tir_of(vct.simulate(vgp, pscs, sim_kw, stream=stream), 1000, nv)
    # the network against its target on random tunings (no selection on its own errors)
    r28, _ = tir_of(vct.simulate(panel, [tune(g, 28) for g in g_cand[rand]], sim_kw, stream=stream), 1000,
                    panel_pop["n_patients"])
    torch.cuda.synchronize()
    pct = lambda x: round(100 * float(x), 3)
    equal = {}
    for k in (10, 100, 1000):
        bt, br = float(t_top[:k].max()), float(t_rand[:k].max())
        se_k = float(np.sqrt(se_top[int(np.argmax(t_top[:k]))] ** 2 + se[1000 + int(np.argmax(t_rand[:k]))] ** 2))
        equal[str(k)] = {"best_of_surrogate_top_k": pct(bt), "best_of_k_random": pct(br),
                         "gain_pp": pct(bt - br), "gain_over_se": round((bt - br) / se_k, 2)}
    rank = lambda v: np.argsort(np.argsort(v))
    out = {
        "training_runs": len(scs) * train_pop["n_patients"], "train_sim_s": t_sim,
        "train_epochs": epochs, "train_s": t_train,
        "train_step_ms": 1000 * t_train / (epochs * (len(scs) * train_pop["n_patients"] // 4096)),
        "loss_per_epoch": [round(float(x), 5) for x in losses],
        "target_entropy": round(entropy, 5),
        "kl_per_epoch": [round(float(x) - entropy, 5) for x in losses],
        "screen_candidates": len(g_cand), "screen_s": t_screen,
        "verify": {"patients": nv, "days": 364, "tunings": len(vscs),
                   "patient_years": len(vscs) * nv, "s": t_verify,
                   "cohort_se_pp_median": pct(np.median(se))},
        "equal_budget": equal,
        "error_split_top1000_mean_abs_pp": {
            "i_network_vs_panel_28d": pct(np.abs(pred[top] - p28).mean()),
            "ii_panel_vs_cohort_28d": pct(np.abs(p28 - c28).mean()),
            "iii_28d_vs_52w_cohort": pct(np.abs(c28 - t_top).mean()),
            "total_network_vs_cohort_52w": pct(np.abs(pred[top] - t_top).mean())},
        "error_split_top1000_mean_signed_pp": {
            "i": pct((pred[top] - p28).mean()), "ii": pct((p28 - c28).mean()),
            "iii": pct((c28 - t_top).mean())},
        "network_vs_panel_28d_on_1000_random": {"mean_abs_pp": pct(np.abs(pred[rand] - r28).mean()),
                                                 "mean_signed_pp": pct((pred[rand] - r28).mean()),
                                                 "rank_correlation": round(float(np.corrcoef(
                                                     rank(pred[rand]), rank(r28))[0, 1]), 3)},
        "train_schedule": [{"epochs": ep, "lr": lr} for ep, lr in schedule],
        "rank_correlation_top1000": round(float(np.corrcoef(rank(pred[top]), rank(t_top))[0, 1]), 3),
        "rank_correlation_network_vs_panel_28d": round(float(np.corrcoef(rank(pred[top]), rank(p28))[0, 1]), 3),
        "tir_70_180_pct": {"median_of_top1000": pct(np.median(t_top)),
                           "median_of_1000_random": pct(np.median(t_rand)), "nominal": pct(t_nom)},
    }
    s.close()
    for g_ in (gp, panel, vgp):
        g_.close()
    return out


def _workload_name(name, n, H):
    """The workload both arms name in their config."""
    return f"{name}: {n} patients x {H} periods (5 min, m=10 EM steps of 30 s) per GPU"


def run_reference(args):
    """--impl reference: the FP64 oracle, as it stands, on the host cores."""
    from paper_2202_13927_gb300 import workloads as W
    rank, world, _ = (int(os.environ.get(k, d)) for k, d in (("RANK", 0), ("WORLD_SIZE", 1), ("LOCAL_RANK", 0)))
    if rank != 0:
        return 0
    pop, sc, _ = W.workload(args.workload)
    cores = os.cpu_count() or 1
    n_sample = args.ref_patients
    rates = []
    for i in range(args.warmup + args.steps):
        r, dt, desc, _ = _cpu_oracle_rate(pop, sc, n_sample, args.ref_days, cores)
        if i >= args.warmup:
            rates.append((r, dt))
    total_py = sum(r * dt for r, dt in rates)
    total_t = sum(dt for _, dt in rates)
    value = total_py / total_t
    line = {
        "impl": "reference", "metric": "simulated patient-years/s", "value": value,
        "unit": "patient-years/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_name(args.workload, pop["n_patients"], sc["horizon_periods"]),
                   "sample": desc + " per step (bounded), FP64 oracle on the host cores"},
        "cpu_baseline": {"value": value, "unit": "patient-years/s", "cores": cores,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "patient-years/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="paper_scale", choices=["paper_scale", "fp32_4w", "small", "profile", "profile_year"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ppt", type=int, default=0)
    ap.add_argument("--reg-cap", type=int, default=0,
                    help="with --block: fixed register cap (0, 128, 112, 96, 80; 192, 168, 128 with --ppt 2); no autotuning")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the probes, the batched-scenario, trial A/B, trace and surrogate measurements")
    ap.add_argument("--extras", default="probes,batched,trial,trace,surrogate,workflow",
                    help="comma list of the extra measurements to run")
    ap.add_argument("--trace-patients", type=int, default=0,
                    help="also write the FP16 CGM traces of the first N patients (time-major) in the timed step")
    ap.add_argument("--ref-patients", type=int, default=1024)
    ap.add_argument("--ref-days", type=int, default=364)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2202_13927_gb300 import dist as D
    from paper_2202_13927_gb300 import vct, workloads as W

    rank, world, local = D.env_rank_world()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vct.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    pop, sc, opts = W.workload(args.workload)
    n = pop["n_patients"]
    first, _ = D.shard_range(rank, world, n)
    pop = W.with_changes(pop, first_patient=first)
    H = sc["horizon_periods"]
    sim_kw = dict(opts, persistent=True, block_size=args.block, patients_per_thread=args.ppt,
                  reg_cap=args.reg_cap)
    trace_buf = None
    if args.trace_patients > 0:   # Fig. 2's traces: y_k of the first N patients, FP16, time-major
        trace_buf = torch.empty((H, args.trace_patients), dtype=torch.float16, device=dev)
        sim_kw.update(trace_ptr=trace_buf.data_ptr(), trace_patients=args.trace_patients,
                      trace_dtype="f16", trace_kind="cgm")
    out = vct.stats_buffer(1, n, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    ev = []
    # the population handle and the graph-captured, autotuned simulation plan
    # are built once; every step draws a new cohort (new seed) into them
    gp_main = vct.Population.create(pop, stream=stream)
    plan = vct.Plan(gp_main, sc, sim_kw, out=out, stream=stream)
    tuned = plan.opts()
    seed0 = pop["seed"]
    step_no = [0]

    def step(record):
        step_no[0] += 1
        gp_main.redraw(seed0 + 1000 * step_no[0], stream=stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.launch(stream=stream)
        b.record(stream)
        recs = D.gather_records(out, rank, world)
        if rank == 0:
            summ = vct.population_stats(recs, 1, n * world, [H], first_patient=0, stream=stream)[0]
        else:
            summ = None
        flush.zero_()
        if record:
            ev.append((a, b))
        return summ

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            summ = step(True)
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    elapsed = t0.elapsed_time(t1) / 1000.0
    sim_ms = [a.elapsed_time(b) for a, b in ev]
    if world > 1:
        t = torch.tensor([elapsed], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
    py_per_step = n * world * H / PATIENT_YEAR
    value = py_per_step * args.steps / elapsed

    # e2e through the public API with host buffers: descriptor and scenario in,
    # per-patient records and the population summary out (pinned host memory)
    host_out = torch.empty(out.numel(), dtype=torch.uint8, pin_memory=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        gp = vct.Population.create(pop, stream=stream)
        vct.simulate(gp, sc, dict(sim_kw, **tuned), out=out, stream=stream)
        host_out.copy_(out, non_blocking=True)
        vct.population_stats(out, 1, n, [H], first_patient=first, stream=stream)
        gp.close()
    torch.cuda.synchronize()
    e_el = time.perf_counter() - e0
    if world > 1:  # the whole job's time: the slowest rank
        t = torch.tensor([e_el], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e_el = float(t.item())
    h2d = vct.C.sizeof(vct.PopulationDesc) + vct.C.sizeof(vct.Scenario) + vct.C.sizeof(vct.SimOpts) + 8
    d2h = out.numel() + vct.C.sizeof(vct.PopulationStats)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    peaks, peak_src = _peaks()
    clocks = clk.summary()
    sim_s = statistics.mean(sim_ms) / 1000.0
    ops_launch = n * H * OPS_PER_PERIOD_FP32
    achieved = ops_launch / sim_s / 1e12
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = SMS * LANES_PER_SM * f_max / 1e12
    lean = args.trace_patients == 0      # the workload asks for no trace, histogram or protocol
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": f"sim_kernel_r<float,10,{tuned['patients_per_thread']},{tuned['reg_cap']}>"
                          f"{' lean' if lean else ''} block {tuned['block_size']}",
                "peak_basis": f"152 SMs x 128 lanes x {f_max/1e6:.0f} MHz (max SM clock, {peak_src})",
                "ops_per_period": OPS_PER_PERIOD_FP32, "launch_ms": 1000 * sim_s}
    if lean and (tuned["patients_per_thread"], tuned["reg_cap"]) == TRAFFIC_SHAPE:
        roofline["traffic"] = TRAFFIC_PER_PATIENT * n
        roofline["traffic_basis"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum, 160000-patient capture, scaled by patients"
    if clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / (SMS * LANES_PER_SM * clocks["sm_mhz"] * 1e6 / 1e12)

    line = {
        "metric": "simulated patient-years/s", "value": value, "unit": "patient-years/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": _workload_name(args.workload, n, H), "form": "FP32 persistent",
                   "patients_per_gpu": n, "horizon_periods": H, "l2": "256 MB buffer written between steps; inputs > L2",
                   "step": "population draw + closed-loop simulation + population reduction",
                   "launch": tuned},
        "e2e": {"value": py_per_step * args.steps / e_el, "unit": "patient-years/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 6 * args.steps,
        "roofline": roofline,
        "clocks": clocks,
        "paper_context": {"value": 203.3, "unit": "patient-years/s",
                          "note": "1e6 patients x 52 weeks in 1 h 22 min, 2x EPYC 7542, larger model; context only"},
        "summary": {"tir_mean": [round(x, 5) for x in summ["tir_mean"]],
                    "worst_patient": summ["worst_patient"]},
    }

    if not args.no_fp64:
        # the plain FP64 form on a bounded sample of the same trial
        n64, days64 = 100_000, 7
        pop64 = W.with_changes(pop, n_patients=n64)
        sc64 = W.with_changes(sc, horizon_periods=days64 * W.PERIODS_PER_DAY)
        gp = vct.Population.create(pop64, stream=stream)
        o64 = vct.stats_buffer(1, n64, dev)
        vct.simulate(gp, sc64, dict(opts, precision="fp64"), out=o64, stream=stream)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        vct.simulate(gp, sc64, dict(opts, precision="fp64"), out=o64, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        s64 = a.elapsed_time(b) / 1000.0
        line["fp64_plain"] = {"value": n64 * sc64["horizon_periods"] / PATIENT_YEAR / s64,
                              "unit": "patient-years/s", "sample": f"{n64} patients x {days64} days",
                              "launch_ms": 1000 * s64,
                              "fp64_ops_per_s": n64 * sc64["horizon_periods"] * FP64_OPS_PER_PERIOD / s64,
                              "executed_fp64_ops_per_s":
                                  n64 * sc64["horizon_periods"] * FP64_OPS_PER_PERIOD_EXECUTED / s64}
        gp.close()

    extras = set() if args.no_extras else set(filter(None, args.extras.split(",")))
    if "probes" in extras:
        # measured issue rates of this GPU (roofline denominators)
        probes = {k: vct.probe(k) for k in ("ffma", "dfma", "imad", "imad_hi", "imad_wide", "mufu", "ffma2", "i2f")}
        line["probe_tops"] = {k: round(v, 3) for k, v in probes.items()}
        roofline["frac_of_ffma_probe"] = achieved / probes["ffma"]
        if lean and (tuned["patients_per_thread"], tuned["reg_cap"]) == TRAFFIC_SHAPE:
            roofline["per_pipe"] = _per_pipe_bound(probes, peak, sim_s / (n * H))
        if "fp64_plain" in line:
            line["fp64_plain"]["frac_of_dfma_probe"] = line["fp64_plain"]["fp64_ops_per_s"] / 1e12 / probes["dfma"]
            line["fp64_plain"]["executed_frac_of_dfma_probe"] = (
                line["fp64_plain"]["executed_fp64_ops_per_s"] / 1e12 / probes["dfma"])
    if "batched" in extras:
        line["batched_uneven"] = _batched_uneven(vct, W, stream)
    if "trial" in extras:
        line["trial_a_vs_b"] = _trial_a_vs_b(vct, W, stream)
    if "trace" in extras:
        line["cgm_trace"] = _cgm_trace(vct, W, stream, {k: tuned[k] for k in
                                                        ("block_size", "patients_per_thread", "reg_cap")})
    if "surrogate" in extras:
        line["surrogate"] = _surrogate(vct, W, stream, peaks)
    if "workflow" in extras:
        line["surrogate_workflow"] = _surrogate_workflow(vct, W, stream, {k: tuned[k] for k in
                                                                   ("block_size", "patients_per_thread", "reg_cap")})

    if not args.no_cpu_baseline:
        r, dt, desc, ostats = _cpu_oracle_rate(pop, sc, 2048, 52 * 7, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": r, "unit": "patient-years/s", "cores": os.cpu_count() or 1,
                                "kind": "oracle", "sample": desc, "seconds": dt}
        # the per-core rate: the oracle on one thread, a sample 1/32 the size
        r1, dt1, desc1, _ = _cpu_oracle_rate(pop, sc, 64, 52 * 7, 1)
        line["cpu_baseline"]["single_thread"] = {"value": r1, "unit": "patient-years/s", "threads": 1,
                                                 "sample": desc1, "seconds": dt1}
        # the same sample's records against the GPU forms (error per statistic)
        line["error_vs_oracle"] = _error_per_statistic(
            vct, W, pop, sc, ostats, 52 * 7, {k: tuned[k] for k in ("block_size", "patients_per_thread", "reg_cap")},
            stream)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
