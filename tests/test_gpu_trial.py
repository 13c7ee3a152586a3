"""The trial runner end to end (Sec. IV: trial A with the correct basal rate,
trial B with the basal rate 50 % low, Figs. 3-5), on a small cohort.

Every number the runner returns comes from the library's kernels; the checks
here are the relations that must hold between them: the curves are CDFs, the
worst-case patient re-simulated alone reaches the same minimum the population
pass reported, its time below each edge lies inside the population's span,
and the daily-dose histograms count one entry per counted patient-day.
"""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def trial():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2202_13927_gb300 import trial as T
    from paper_2202_13927_gb300 import vct
    vct.load()
    return T


def _check_arm(T, r, days, H):
    tir = np.array(r["tir_mean_pct"])
    assert abs(tir.sum() - 100.0) < 1e-9
    for rng in T.RANGES:
        q = np.array(r["tir_box_pct"][rng])
        assert np.all(np.diff(q) >= 0) and q[0] >= 0 and q[-1] <= 100
    for key in ("mean_cdf", "worst_cdf"):
        c = np.array(r[key])
        assert np.all(np.diff(c) >= 0) and abs(c[-1] - 1.0) < 1e-12
    # the mean curve against the range fractions (every counted patient has
    # the same number of samples, so the pooled and the per-patient means
    # agree): 54 and 180 mg/dL are the bin edges 3.0 and 10.0 mmol/L, equal up
    # to samples whose 10 G rounds across the edge; 70 mg/dL (3.89 mmol/L)
    # lies inside the bin [3.8, 3.9)
    c = 100.0 * np.array(r["mean_cdf"])
    assert abs(c[29] - tir[0]) < 0.01
    assert abs(c[99] - tir[:3].sum()) < 0.01
    assert c[37] - 0.01 <= tir[:2].sum() <= c[38] + 0.01
    # the worst-case patient re-simulated alone
    assert r["worst_replay_g_min"] == r["worst_g_min"]
    below = np.cumsum(r["worst_tir_pct"])[:4]
    for j, e in enumerate(("54", "70", "180", "250")):
        lo, hi = r["span_below_edges_pct"][e]
        assert lo - 1e-9 <= below[j] <= hi + 1e-9
    # Fig. 5: one count per counted patient-day in each of the three histograms
    for k, h in r["daily_dose_hist"].items():
        assert sum(h) == r["n_counted"] * days, k
    assert 0 <= r["n_q1_clamped"] <= r["n_counted"] + r["n_flagged"]
    q = r["daily_dose_quantiles"]["basal_u"]
    assert np.all(np.diff(q) >= 0) and q[0] > 0


def test_trial_a_vs_b_small_cohort(trial, tmp_path):
    T = trial
    res = T.run_trial(n_patients=3000, weeks=1, seed=11)
    days, H = 7, 7 * 288
    assert set(res["arms"]) == {"A", "B"}
    for r in res["arms"].values():
        assert r["n_counted"] + r["n_flagged"] <= res["patients"]
        _check_arm(T, r, days, H)
    A, B = res["arms"]["A"], res["arms"]["B"]
    # trial B's controller believes the basal rate is half the true one: it
    # gives less basal insulin and the cohort runs higher
    assert B["mean_daily"]["basal_u"] < A["mean_daily"]["basal_u"]
    assert B["tir_mean_pct"][3] + B["tir_mean_pct"][4] > A["tir_mean_pct"][3] + A["tir_mean_pct"][4]
    # the command line writes the same structure as JSON
    out = tmp_path / "trial.json"
    assert T.main(["--patients", "500", "--weeks", "1", "--out", str(out)]) == 0
    got = json.loads(out.read_text())
    assert got["patients"] == 500 and set(got["arms"]) == {"A", "B"}
    _check_arm(T, got["arms"]["A"], days, H)
