"""The year protocol of Sec. II-B (Tables I and II) and its use by the oracle.

No GPU needed.  Pins: the transcription of Table I (13 weeks per season, 7 days
per week type, eight vacation weeks = six weeks plus ten public holidays),
Table II's own 70 kg column (1.29/0.86/0.57/0.29 g/kg give 90/60/40/20 g),
and, with meal noise off, the bolus total in closed form: TDD/500 times the
body weight times the sum of g/kg over the days simulated.
"""
import collections

import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_13927_gb300 import workloads as W


def test_table_one_compositions():
    for season, comp in W.SEASON_WEEKS.items():
        assert sum(comp.values()) == 13, season
    for week, comp in W.WEEK_DAYS.items():
        assert sum(comp.values()) == 7, week
    assert sum(c["vacation"] for c in W.SEASON_WEEKS.values()) == 6 + 2


def test_generated_year_follows_table_one():
    days = W.paper_protocol()
    assert len(days) == 364
    for si, season in enumerate(("winter", "spring", "summer", "autumn")):
        weeks = [days[(13 * si + w) * 7] for w in range(13)]
        assert all(d["season"] == season for d in days[91 * si:91 * (si + 1)])
        got = collections.Counter(d["week"] for d in weeks)
        assert dict(got) == {k: v for k, v in W.SEASON_WEEKS[season].items() if v}
    for w in range(52):
        week = days[7 * w:7 * (w + 1)]
        kind = week[0]["week"]
        assert all(d["week"] == kind for d in week)
        got = collections.Counter(d["day"] for d in week)
        assert dict(got) == {k: v for k, v in W.WEEK_DAYS[kind].items() if v}


def test_table_two_seventy_kg_column():
    grams = {k: 70.0 * v for k, v in W.MEAL_G_PER_KG.items()}
    for k, g in zip(("large", "medium", "small", "snack"), (90, 60, 40, 20)):
        assert grams[k] == pytest.approx(g, abs=0.5)


def test_day_plans_are_valid_and_seasonal():
    for d in W.paper_protocol():
        assert d["minute"] == sorted(set(d["minute"])) and len(d["minute"]) <= 8
        assert all(m % 5 == 0 for m in d["minute"])
        dinner = d["g_per_kg"][d["minute"].index(1080.0)]
        cold = d["season"] in ("winter", "autumn")
        assert dinner == (W.MEAL_G_PER_KG["large"] if cold else W.MEAL_G_PER_KG["medium"])
        extra = {"standard": 0, "active": 0, "movie": 1, "late": 2}[d["day"]]
        assert len(d["minute"]) == 4 + extra


def test_protocol_bolus_closed_form():
    pop = W.population(20, 91)
    people = O.create_population(pop)
    days = 10
    sc = W.protocol_scenario(days, meal_cv=0.0)
    st = O.simulate(pop, people, sc, {})["stats"]
    plans = W.paper_protocol()
    # the sizes travel as float32 and are summed in float64
    gkg = sum(float(np.float32(g)) for d in range(days) for g in plans[d]["g_per_kg"])
    for i in range(20):
        ub_hat = people["u_b"][i] * sc["basal_scale"]
        tdd = 48.0 * ub_hat * 60.0 / 1000.0
        expect = tdd / 500.0 * people["rows"][i, 16] * float(gkg)
        assert st["bolus_u"][i] == pytest.approx(expect, rel=1e-12)
    # the protocol cycles: day 364 repeats day 0 (same plan, same per-kg sizes)
    long = W.protocol_scenario(366, meal_cv=0.0)
    long["horizon_periods"] = 366 * 288
    assert len(long["day_plans"]) == 364
