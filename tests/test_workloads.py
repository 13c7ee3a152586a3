"""The seeded input recipe (no GPU): the workloads have the sizes, horizons,
precisions and distributions that the benchmark and the parity tests claim.

* the named workloads: 10^3 x 7 days FP64, 10^5 x 28 days FP32, 10^6 x 52
  weeks FP32 (the paper's trial shape, Sec. IV), the 160,000 x 7-day
  profiling case; Ts = 5 min, so 52 weeks = 104,832 periods;
* the default trial arm: three meals at 07, 12 and 18 h of N(50, 10) g,
  PID with bolus, correct basal;
* the population table: Hovorka nominal values, a 20 % / 50 % CV reading,
  A_G and the CGM lag fixed, BW ~ N(75, 12) kg, G_sp = 6 mmol/L, and the
  acceptance rule's 0.4 U/h (Sec. IV-B);
* the scenario sweep: gains log-uniform in [0.3, 3] x nominal, meal means
  uniform in [30, 90] g, whole-week horizons uniform in 1..52 weeks, a pure
  function of its seed.
"""
import numpy as np
from scipy import stats

from paper_2202_13927_gb300 import workloads as W


def test_named_workloads():
    expect = {"small": (1000, 7, 1, "fp64"), "fp32_4w": (100_000, 28, 2, "fp32"),
              "paper_scale": (1_000_000, 364, 3, "fp32"), "profile": (160_000, 7, 3, "fp32"),
              "profile_year": (160_000, 364, 3, "fp32")}
    assert set(W.WORKLOADS) == set(expect)
    for name, (n, days, seed, prec) in expect.items():
        pop, sc, opts = W.workload(name)
        assert (pop["n_patients"], pop["seed"], opts["precision"]) == (n, seed, prec)
        assert sc["horizon_periods"] == days * 288
        assert opts["substeps"] == 10 and opts["ts_min"] == 5.0       # h = 30 s
    assert W.PATIENT_YEAR_PERIODS == 104_832 == W.workload("paper_scale")[1]["horizon_periods"]


def test_default_arm_and_population_table():
    sc = W.scenario(1)
    assert sc["meal_minute"] == [420.0, 720.0, 1080.0]
    assert (sc["meal_mean_g"], sc["meal_sd_g"], sc["bolus"], sc["basal_scale"]) == (50.0, 10.0, True, 1.0)
    assert (sc["kp_mult"], sc["ki_mult"], sc["kd_mult"], sc["glucagon"]) == (1.0, 1.0, 1.0, False)
    pop = W.population(10, 1)
    assert (pop["bw_mean"], pop["bw_sd"], pop["g_sp"], pop["min_basal_u_per_h"]) == (75.0, 12.0, 6.0, 0.4)
    assert (pop["sigma_q1"], pop["cgm_sd"]) == (0.5, 0.2)
    for j, k in enumerate(W.PARAM_NAMES):
        assert pop["p_mean"][j] == W.NOMINAL[k]
        cv = 0.0 if k in ("AG", "tauCGM") else (0.5 if k in ("SIT", "SID", "SIE") else 0.2)
        assert pop["p_sd"][j] == W.NOMINAL[k] * cv, k


def test_scenario_sweep_distributions():
    pop, scs = W.batched_uneven()
    assert len(scs) == 256 and pop["n_patients"] == 4096 and pop["seed"] == 4
    gains = np.array([[s["kp_mult"], s["ki_mult"], s["kd_mult"]] for s in scs])
    assert gains.min() >= 0.3 and gains.max() <= 3.0
    lo, hi = np.log(0.3), np.log(3.0)
    for j in range(3):      # log-uniform, each gain on its own
        assert stats.kstest(np.log(gains[:, j]), stats.uniform(lo, hi - lo).cdf).pvalue > 1e-4
    assert abs(np.corrcoef(gains[:, 0], gains[:, 1])[0, 1]) < 5 / np.sqrt(256)
    meals = np.array([s["meal_mean_g"] for s in scs])
    assert meals.min() >= 30.0 and meals.max() <= 90.0
    assert stats.kstest(meals, stats.uniform(30.0, 60.0).cdf).pvalue > 1e-4
    weeks = np.array([s["horizon_periods"] for s in scs]) / W.PERIODS_PER_WEEK
    assert np.all(weeks == np.round(weeks)) and weeks.min() >= 1 and weeks.max() <= 52
    assert len(set(weeks.astype(int))) > 40          # the horizons really are uneven
    # a pure function of the seed
    _, again = W.batched_uneven()
    assert again == scs
    _, other = W.batched_uneven(seed=5)
    assert other != scs
