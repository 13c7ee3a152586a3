"""A virtual clinical trial end to end (Sec. IV of arXiv 2202.13927).

Draws the cohort on the GPU, runs every trial arm in one graph-captured
persistent launch, reduces the per-patient indicators, and returns the data
behind the paper's result figures:

  * Fig. 3 -- time spent below each BG level: the population's mean curve (from
    the exact histogram of every binned sample, 0.1 mmol/L bins), the
    worst-case patient's curve (that patient re-simulated alone with a BG
    trace, exact because every draw is keyed by patient and period) and the
    span over all patients at the four range edges;
  * Fig. 4 -- the mean range fractions and the box plot (min, quartiles, max)
    of the per-patient fractions, and the worst-case patient's fractions;
  * Fig. 5 -- the distributions of the total daily basal and bolus insulin and
    bolus glucagon (per patient-day histograms).

The default trial is the paper's comparison: one million patients over 52
weeks of the year protocol, arm A with the correct basal rate and arm B with
the basal rate 50 % low, the controller with its glucagon mode, both arms on
common random numbers.  Everything runs in the CUDA library; this module only
arranges the calls.

    python -m paper_2202_13927_gb300.trial --patients 100000 --weeks 4 --out trial.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import vct
from . import workloads as W

RANGES = ("<54", "54-70", "70-180", "180-250", ">=250")      # mg/dL
EDGES_MMOL = (54.0 / 18.0, 70.0 / 18.0, 180.0 / 18.0, 250.0 / 18.0)
PAPER_ARMS = ({"name": "A", "basal_scale": 1.0, "glucagon": True},
              {"name": "B", "basal_scale": 0.5, "glucagon": True})


def _arm_scenario(arm: dict, days: int, protocol: str) -> dict:
    kw = {k: v for k, v in arm.items() if k != "name"}
    if protocol == "year":
        return W.protocol_scenario(days, **kw)
    return W.scenario(days, **kw)


def run_trial(n_patients: int = 1_000_000, weeks: int = 52, seed: int = 3, protocol: str = "year",
              arms=PAPER_ARMS, precision: str = "fp32", replay_worst: bool = True, stream=None) -> dict:
    """Run the trial; returns a dict of plain lists and numbers (JSON-ready)."""
    import torch

    days = 7 * int(weeks)
    pop = W.population(int(n_patients), int(seed))
    scs = [_arm_scenario(a, days, protocol) for a in arms]
    S, H = len(scs), days * W.PERIODS_PER_DAY
    gp = vct.Population.create(pop, stream=stream)
    bg = torch.zeros(S * vct.BG_BINS, dtype=torch.int32, device="cuda")
    dose = torch.zeros(S * 3 * vct.DOSE_BINS, dtype=torch.int32, device="cuda")
    plan = vct.Plan(gp, scs, {"precision": precision, "persistent": True,
                              "bg_hist": bg.data_ptr(), "dose_hist": dose.data_ptr()}, stream=stream)
    bg.zero_()                      # the autotuner's short runs added to them
    dose.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    plan.launch(stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    launch_s = a.elapsed_time(b) / 1000.0
    summ = vct.population_stats(plan.out, S, gp.n, [H] * S, stream=stream)
    recs = vct.stats_to_numpy(plan.out).reshape(S, gp.n)
    dose_h = dose.cpu().numpy().astype(np.int64).reshape(S, 3, vct.DOSE_BINS)
    # Fig. 3's mean curves and Fig. 5's quantiles, computed by the library from
    # the device histograms
    cdfs = vct.bg_cdf(bg, S, stream=stream).reshape(S, vct.BG_BINS)
    dq = vct.dose_quantiles(dose, S, (0.05, 0.25, 0.5, 0.75, 0.95), stream=stream)
    result = {
        "patients": gp.n, "weeks": int(weeks), "protocol": protocol, "precision": precision,
        "launch_s": launch_s, "patient_years_per_s": S * gp.n * days / 364.0 / launch_s,
        "launch": plan.opts(), "ranges_mg_dl": list(RANGES), "bg_bin_mmol_l": 0.1, "arms": {},
    }
    for arm, sc, sm, cdf, hd, q, rec in zip(arms, scs, summ, cdfs, dose_h, dq, recs):
        r = {
            "n_counted": int(sm["n_patients"]), "n_flagged": int(sm["n_flagged"]),
            # patients whose glucose the Q1 clamp ever held at zero (P8)
            "n_q1_clamped": int((rec["q1_clamps"] > 0).sum()),
            # Fig. 4
            "tir_mean_pct": [100.0 * float(x) for x in sm["tir_mean"]],
            "tir_box_pct": {rng: [100.0 * float(x) for x in sm["tir_quantile"][j]]
                            for j, rng in enumerate(RANGES)},
            "worst_patient": int(sm["worst_patient"]), "worst_g_min": float(sm["worst_g_min"]),
            # Fig. 3
            "mean_cdf": [float(x) for x in cdf],
            "span_below_edges_pct": {f"{18 * e:.0f}": [100.0 * int(lo) / H, 100.0 * int(hi) / H]
                                     for e, lo, hi in zip(EDGES_MMOL, sm["below_min"], sm["below_max"])},
            # Fig. 5
            "daily_dose_hist": {k: [int(x) for x in hd[j]] for j, k in enumerate(vct.DOSE_BIN_WIDTHS)},
            "daily_dose_quantiles": {k: [float(x) for x in q[j]] for j, k in enumerate(vct.DOSE_BIN_WIDTHS)},
            "mean_daily": {"basal_u": sm["basal_u_mean"] / days, "bolus_u": sm["bolus_u_mean"] / days,
                           "glucagon_ug": sm["glucagon_ug_mean"] / days},
        }
        if replay_worst and sm["n_patients"] > 0:
            tdt = "f32" if precision == "fp32" else "f64"
            rec, g, wh = vct.replay(pop, sc, int(sm["worst_patient"]), {"precision": precision},
                                    trace_dtype=tdt, bg_hist=True)
            r["worst_cdf"] = [float(x) for x in vct.bg_cdf(wh, 1)]
            r["worst_tir_pct"] = [100.0 * int(x) / max(int(rec["n_samples"]), 1) for x in rec["tir"]]
            r["worst_replay_g_min"] = float(rec["g_min"])
        result["arms"][arm.get("name", str(len(result["arms"])))] = r
    plan.close()
    gp.close()
    return result


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description="Run a virtual clinical trial (paper Sec. IV) on the GPU.")
    ap.add_argument("--patients", type=int, default=1_000_000)
    ap.add_argument("--weeks", type=int, default=52)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--protocol", choices=["year", "fixed"], default="year")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-glucagon", action="store_true", help="insulin-only controller in both arms")
    ap.add_argument("--out", default="-", help="JSON output file ('-' = stdout)")
    args = ap.parse_args(argv)
    arms = [dict(a, glucagon=not args.no_glucagon) for a in PAPER_ARMS]
    t0 = time.perf_counter()
    res = run_trial(args.patients, args.weeks, args.seed, args.protocol, arms, args.precision)
    res["wall_s"] = time.perf_counter() - t0
    text = json.dumps(res)
    if args.out == "-":
        print(text)
    else:
        with open(args.out, "w") as f:
            f.write(text)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
