"""Seeded synthetic inputs: populations, scenarios and simulation options.

This module holds inputs only -- numbers and their seeded generators -- and
none of the method's arithmetic.  Both the CUDA library (through ``vct.py``)
and the FP64 oracle consume the plain dictionaries built here, so that both
sides see identical inputs.

The paper (arXiv 2202.13927) prints neither the parameter values nor their
distributions: Sec. IV-B only says that the parameters are drawn from the
distributions of Hovorka et al. (2002) and that sets are kept when all values
are nonnegative, the normal ones lie within one standard deviation and the
basal rate is at least 0.4 U/h.  The nominal values below are those of the
Hovorka 2004 core model; the coefficients of variation are a stated reading
(20 % for rates, volumes and time constants, 50 % for the insulin
sensitivities; A_G and the CGM lag fixed, as Sec. IV-B fixes the
CGM-related parameters for all patients).  Body weight (Sec. II-A: normal)
is N(75, 12) kg.

Workloads (the paper's trial shape, Sec. IV: one million patients over 52
weeks; three meals a day):
  * ``small``         1,000 patients x 7 days, FP64 parity case
  * ``fp32_4w``       100,000 patients x 28 days
  * ``paper_scale``   1,000,000 patients x 364 days (52 weeks)
  * ``batched``       256 scenarios x 4,096 patients, horizons 1-52 weeks
"""
from __future__ import annotations

import copy

import numpy as np

PARAM_NAMES = ["EGP0", "F01", "k12", "ka1", "ka2", "ka3", "SIT", "SID", "SIE", "ke",
               "VI", "VG", "tauS", "tauD", "AG", "tauCGM"]
STATE_NAMES = ["D1", "D2", "S1", "S2", "I", "x1", "x2", "x3", "Q1", "Q2", "Gsc"]

# Hovorka et al. 2004 nominal values (units: mmol, L, kg, min, mU).
NOMINAL = {
    "EGP0": 0.0161,     # mmol/kg/min
    "F01": 0.0097,      # mmol/kg/min
    "k12": 0.066,       # 1/min
    "ka1": 0.006,       # 1/min
    "ka2": 0.06,        # 1/min
    "ka3": 0.03,        # 1/min
    "SIT": 51.2e-4,     # 1/min per mU/L
    "SID": 8.2e-4,      # 1/min per mU/L
    "SIE": 520e-4,      # per mU/L
    "ke": 0.138,        # 1/min
    "VI": 0.12,         # L/kg
    "VG": 0.16,         # L/kg
    "tauS": 55.0,       # min
    "tauD": 40.0,       # min
    "AG": 0.8,          # -
    "tauCGM": 10.0,     # min
}
CV = {name: 0.2 for name in PARAM_NAMES}
CV.update({"SIT": 0.5, "SID": 0.5, "SIE": 0.5, "AG": 0.0, "tauCGM": 0.0})

MINUTES_PER_DAY = 1440.0
PERIODS_PER_DAY = 288          # Ts = 5 min
PERIODS_PER_WEEK = 7 * PERIODS_PER_DAY
PATIENT_YEAR_PERIODS = 52 * PERIODS_PER_WEEK   # 104,832 control periods


def population(n_patients: int, seed: int, *, first_patient: int = 0,
               sigma_q1: float = 0.5, cgm_sd: float = 0.2, g_sp: float = 6.0,
               min_basal_u_per_h: float = 0.4, max_attempts: int = 64) -> dict:
    """Population descriptor: distribution table, seed and noise levels."""
    return {
        "n_patients": int(n_patients),
        "first_patient": int(first_patient),
        "seed": int(seed),
        "bw_mean": 75.0,
        "bw_sd": 12.0,
        "p_mean": [NOMINAL[k] for k in PARAM_NAMES],
        "p_sd": [NOMINAL[k] * CV[k] for k in PARAM_NAMES],
        "g_sp": float(g_sp),
        "min_basal_u_per_h": float(min_basal_u_per_h),
        "sigma_q1": float(sigma_q1),
        "cgm_sd": float(cgm_sd),
        "max_attempts": int(max_attempts),
        # two-state s.c. glucagon model, shared by all patients (Sec. IV-B):
        # absorption time constant and sensitivity of EGP to the second compartment
        "tau_gg_min": 20.0,    # min
        "s_gg": 1.0,           # kg/ug
    }


def scenario(horizon_days: float, *, kp_mult: float = 1.0, ki_mult: float = 1.0,
             kd_mult: float = 1.0, meal_mean_g: float = 50.0, meal_sd_g: float = 10.0,
             meal_minute=(420.0, 720.0, 1080.0), bolus: bool = True,
             basal_scale: float = 1.0, stream_id: int = 0,
             horizon_periods: int | None = None, glucagon: bool = False) -> dict:
    """One trial arm: PID plus meal bolus, three meals a day at 07, 12, 18 h;
    with ``glucagon`` the controller switches to glucagon mode (no insulin,
    glucagon microboli) while the CGM value is below 70 mg/dL."""
    h = int(round(horizon_days * PERIODS_PER_DAY)) if horizon_periods is None else int(horizon_periods)
    return {
        "kp_mult": float(kp_mult), "ki_mult": float(ki_mult), "kd_mult": float(kd_mult),
        "kp_per_ub": 0.1,        # nominal Kp = 0.1 ub_hat per mmol/L
        "ti_min": 300.0, "td_min": 30.0,
        "i_max": 1440.0,         # mmol min / L
        "basal_scale": float(basal_scale),
        "meal_mean_g": float(meal_mean_g), "meal_sd_g": float(meal_sd_g),
        "meal_minute": [float(m) for m in meal_minute],
        "bolus": bool(bolus),
        "horizon_periods": h,
        "stream_id": int(stream_id),
        "glucagon": bool(glucagon),
        "gg_threshold": 70.0 / 18.0,   # mmol/L
        "gg_gain": 10.0,               # ug per mmol/L below the threshold
        "gg_max_ug": 20.0,             # ug per period
    }


def sim_opts(precision: str = "fp32", *, substeps: int = 10, ts_min: float = 5.0) -> dict:
    """Integration settings: Ts = 5 min control period, m = 10 steps of 30 s."""
    return {"precision": precision, "substeps": int(substeps), "ts_min": float(ts_min)}


def batched_uneven(n_scen: int = 256, n_patients: int = 4096, seed: int = 4,
                   max_weeks: int = 52) -> tuple[dict, list[dict]]:
    """Scenario sweep: PID gains log-uniform in [0.3, 3] x nominal (each gain
    independently), meal means uniform in [30, 90] g, horizons uniform in
    1..max_weeks weeks; one population shared by all scenarios."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(0.3), np.log(3.0)
    scs = []
    for s in range(n_scen):
        g = np.exp(rng.uniform(lo, hi, size=3))
        meal = rng.uniform(30.0, 90.0)
        weeks = int(rng.integers(1, max_weeks + 1))
        scs.append(scenario(0, kp_mult=g[0], ki_mult=g[1], kd_mult=g[2], meal_mean_g=meal,
                            horizon_periods=weeks * PERIODS_PER_WEEK, stream_id=0))
    return population(n_patients, seed), scs


# --------------------------------------------------------------- the year protocol
# Sec. II-B, Table I: week types per season (13 weeks each) and day types per
# week type (7 days each).  Six vacation weeks plus ten public holidays count as
# eight vacation weeks over the year.
SEASON_WEEKS = {
    "winter": {"standard": 6, "active": 4, "vacation": 3},
    "spring": {"standard": 6, "active": 6, "vacation": 1},
    "summer": {"standard": 7, "active": 3, "vacation": 3},
    "autumn": {"standard": 9, "active": 3, "vacation": 1},
}
WEEK_DAYS = {
    "standard": {"standard": 4, "active": 1, "movie": 1, "late": 1},
    "active": {"standard": 3, "active": 3, "movie": 1, "late": 0},
    "vacation": {"standard": 5, "active": 0, "movie": 0, "late": 2},
}
# Table II: meal sizes in g of carbohydrate per kg body weight.
MEAL_G_PER_KG = {"large": 1.29, "medium": 0.86, "small": 0.57, "snack": 0.29}

# Readings (the meal clock times are drawn only in Fig. 1):
#  * seasons in the order winter, spring, summer, autumn (the year starts in January);
#    within a season standard and active weeks alternate, vacation weeks close it;
#  * day order Monday..Sunday: standard week S S S S A M L, active week A S A S M A S,
#    vacation week S S S S S L L (S standard, A active, M movie night, L late night);
#  * winter and autumn day: breakfast 07:00 small, lunch 12:00 medium, snack 15:00,
#    dinner 18:00 large; spring and summer: the snack moves before lunch (10:00) and
#    dinner is medium (both stated in Fig. 1's caption);
#  * movie night adds a snack at 21:00, late night snacks at 21:00 and 23:00;
#  * vacation weeks "eat more": breakfast is a medium meal;
#  * the active day's exercise is not modelled (its model is not in the paper), so its
#    meals are those of a standard day.
_WEEK_ORDER = {
    "standard": ["standard"] * 4 + ["active", "movie", "late"],
    "active": ["active", "standard", "active", "standard", "movie", "active", "standard"],
    "vacation": ["standard"] * 5 + ["late", "late"],
}


def _season_week_order(comp: dict) -> list:
    s, a, v = comp["standard"], comp["active"], comp["vacation"]
    order = []
    while s or a:
        if s:
            order.append("standard")
            s -= 1
        if a:
            order.append("active")
            a -= 1
    return order + ["vacation"] * v


def _day_plan(season: str, week_type: str, day_type: str) -> dict:
    cold = season in ("winter", "autumn")
    breakfast = "medium" if week_type == "vacation" else "small"
    meals = [(420.0, breakfast)]
    if cold:
        meals += [(720.0, "medium"), (900.0, "snack"), (1080.0, "large")]
    else:
        meals += [(600.0, "snack"), (720.0, "medium"), (1080.0, "medium")]
    if day_type == "movie":
        meals.append((1260.0, "snack"))
    elif day_type == "late":
        meals += [(1260.0, "snack"), (1380.0, "snack")]
    meals.sort()
    return {"minute": [m for m, _ in meals], "g_per_kg": [MEAL_G_PER_KG[k] for _, k in meals],
            "season": season, "week": week_type, "day": day_type}


def paper_protocol() -> list:
    """The Northern-European year of Sec. II-B: 52 weeks = 364 day plans."""
    days = []
    for season in ("winter", "spring", "summer", "autumn"):
        for week_type in _season_week_order(SEASON_WEEKS[season]):
            for day_type in _WEEK_ORDER[week_type]:
                days.append(_day_plan(season, week_type, day_type))
    return days


def protocol_scenario(horizon_days: float, meal_cv: float = 0.1, **kw) -> dict:
    """A trial arm that follows the year protocol instead of three fixed meals."""
    sc = scenario(horizon_days, **kw)
    sc["day_plans"] = paper_protocol()
    sc["meal_cv"] = float(meal_cv)
    return sc


WORKLOADS = {
    "small": dict(n=1000, days=7, seed=1, precision="fp64"),
    "fp32_4w": dict(n=100_000, days=28, seed=2, precision="fp32"),
    "paper_scale": dict(n=1_000_000, days=364, seed=3, precision="fp32"),
    # profiling case: the paper-scale kernel on 160,000 patients x 7 days
    "profile": dict(n=160_000, days=7, seed=3, precision="fp32"),
    # the same over 52 weeks: a trace of 10,000 patients (2.1 GB) outgrows the L2
    "profile_year": dict(n=160_000, days=364, seed=3, precision="fp32"),
}


def workload(name: str) -> tuple[dict, dict, dict]:
    w = WORKLOADS[name]
    return (population(w["n"], w["seed"]), scenario(w["days"]), sim_opts(w["precision"]))


def with_changes(d: dict, **kw) -> dict:
    out = copy.deepcopy(d)
    out.update(kw)
    return out
