"""Pins of the oracle's daily doses (Fig. 5: distributions of the total daily
basal and bolus insulin and bolus glucagon).

Each whole day of a patient contributes the basal insulin (U), bolus insulin
(U) and glucagon (ug) delivered in its periods; the pins use a controller
whose insulin rate is known in closed form.
"""
import numpy as np

from oracle import oracle as O
from paper_2202_13927_gb300 import workloads as W


def test_constant_controller_gives_exact_daily_basal_and_bolus_per_meal():
    # zero PID gains: u_pid = ub_hat in every period, so a day's basal is
    # ub_hat 1440 / 1000 U; meals in the first and the last period of the day
    # must be booked on that day
    pop = W.population(30, 61)
    people = O.create_population(pop)
    sc = W.scenario(3, kp_mult=0.0, ki_mult=0.0, kd_mult=0.0, basal_scale=0.8,
                    meal_minute=(0.0, 1435.0))
    res = O.simulate(pop, people, sc, {}, trace_u=True, day_doses=True)
    ok = people["status"] == 0
    ub_hat = 0.8 * people["u_b"][ok]
    dd = res["day_doses"][ok]
    assert dd.shape[1] == 3
    np.testing.assert_allclose(dd[:, :, 0], np.repeat(ub_hat[:, None] * 1.44, 3, axis=1), rtol=1e-13)
    bolus_rate = (res["u"][ok] - ub_hat[:, None]) * 5.0 / 1000.0          # U per period
    per_day = bolus_rate.reshape(-1, 3, W.PERIODS_PER_DAY).sum(axis=2)
    np.testing.assert_allclose(dd[:, :, 1], per_day, rtol=1e-9, atol=1e-12)
    assert np.all(bolus_rate[:, 0] > 0) and np.all(bolus_rate[:, 287] > 0)
    assert np.all(dd[:, :, 2] == 0.0)


def test_daily_doses_add_up_to_the_trial_totals():
    pop = W.population(100, 62)
    people = O.create_population(pop)
    sc = W.scenario(4, basal_scale=1.5, glucagon=True)
    res = O.simulate(pop, people, sc, {}, day_doses=True)
    st, dd = res["stats"], res["day_doses"]
    ok = (people["status"] == 0) & (st["status"] == 0)
    np.testing.assert_allclose(dd[ok, :, 0].sum(axis=1), st["basal_u"][ok], rtol=1e-12)
    np.testing.assert_allclose(dd[ok, :, 1].sum(axis=1), st["bolus_u"][ok], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dd[ok, :, 2].sum(axis=1), st["glucagon_ug"][ok], rtol=1e-12, atol=1e-12)
    assert dd[ok, :, 2].sum() > 0


def test_always_glucagon_mode_gives_the_cap_every_period_and_partial_days_are_left_out():
    pop = W.population(10, 63)
    people = O.create_population(pop)
    sc = dict(W.scenario(1, horizon_periods=2 * W.PERIODS_PER_DAY + 100), glucagon=True,
              gg_threshold=1e6, gg_gain=1e9, gg_max_ug=7.0)
    dd = O.simulate(pop, people, sc, {}, day_doses=True)["day_doses"]
    ok = people["status"] == 0
    assert dd.shape[1] == 2          # the third day is not complete
    np.testing.assert_array_equal(dd[ok, :, 2], 7.0 * W.PERIODS_PER_DAY)
    np.testing.assert_array_equal(dd[ok, :, :2], 0.0)
