"""Values the paper prints, kept as text fixtures under ``tests/golden/`` (each
file cites its table or section), against the transcriptions and the oracle.

* Table I: the week and day compositions the year protocol is generated from;
* Table II: the meal sizes per kg, and the printed 70 kg column they imply;
* Sec. II-B: 52 weeks, eight of them vacation (six plus ten public holidays);
* Sec. IV-A: the oracle's range edges (54, 70, 180, 250 mg/dL over 18) are the
  printed mmol/L edges 3, 3.9, 10, 13.9 to the printed precision, and a BG
  sample changes range exactly there.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_13927_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    """Non-comment lines of a fixture, split on whitespace."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


def test_table_one_transcription():
    rows = _rows("table1_compositions.txt")
    seasons, weeks = rows[:4], rows[4:]
    for name, std, act, vac in seasons:
        assert W.SEASON_WEEKS[name] == {"standard": int(std), "active": int(act), "vacation": int(vac)}
    for name, std, act, movie, late in weeks:
        assert W.WEEK_DAYS[name] == {"standard": int(std), "active": int(act), "movie": int(movie),
                                     "late": int(late)}
    assert len(seasons) == len(W.SEASON_WEEKS) == 4 and len(weeks) == len(W.WEEK_DAYS) == 3
    # Sec. II-B: 13 weeks a season; 6 vacation weeks + 10 public holidays as 2 more
    assert all(sum(int(v) for v in r[1:]) == 13 for r in seasons)
    assert sum(int(r[3]) for r in seasons) == 6 + 2
    assert all(sum(int(v) for v in r[1:]) == 7 for r in weeks)


def test_table_two_transcription_and_seventy_kg_column():
    rows = _rows("table2_meal_sizes.txt")
    assert len(rows) == len(W.MEAL_G_PER_KG) == 4
    for name, per_kg, g70 in rows:
        assert W.MEAL_G_PER_KG[name] == float(per_kg)
        # the printed 70 kg column is the per-kg size times 70, rounded to whole grams
        assert round(70.0 * W.MEAL_G_PER_KG[name]) == int(g70)


def _bin_of(g):
    """Range index the oracle gives one BG sample g (mmol/L), taken at t_0."""
    row = np.array([W.NOMINAL[k] for k in O.PARAM_NAMES] + [80.0])
    row[O.PARAM_NAMES.index("VG")] = 0.125            # V_G BW = 10 L
    x0 = np.zeros(O.NX)
    x0[O.STATE_NAMES.index("Q1")] = 10.0 * g
    x0[O.STATE_NAMES.index("Gsc")] = g
    people = {"rows": row[None, :], "u_b": np.array([0.0]), "x0": x0[None, :], "first": 0}
    pop = W.population(1, 1, sigma_q1=0.0, cgm_sd=0.0)
    sc = W.scenario(0, horizon_periods=1, meal_minute=())
    tir = O.simulate(pop, people, sc, {})["stats"]["tir"][0]
    assert tir.sum() == 1
    return int(np.argmax(tir))


@pytest.mark.parametrize("j", range(4))
def test_range_edges_are_the_printed_ones(j):
    printed = float(_rows("bg_ranges.txt")[j][0])
    edge = (54.0, 70.0, 180.0, 250.0)[j] / 18.0        # mg/dL edges over 18 (mmol/L)
    assert round(edge, 1) == printed
    # the oracle's sample moves from range j to j + 1 exactly at the edge
    assert _bin_of(edge * (1 - 1e-9)) == j
    assert _bin_of(edge * (1 + 1e-9)) == j + 1
    assert _bin_of(edge - 0.05) == j and _bin_of(edge + 0.05) == j + 1
