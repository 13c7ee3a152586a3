"""Pins of the oracle's glucagon compartments and glucagon mode (Sec. IV-B:
two-state s.c. glucagon model; Sec. IV-C: the AP's glucagon mode gives no
insulin and only glucagon microboli).

Each pin comes from mathematics the oracle does not use: the exact solution of
the Euler recursion of a linear two-compartment chain under constant
infusion, the one-step effect of Z2 on Q1, and special cases in which the mode
never or always applies.
"""
import numpy as np

from oracle import oracle as O
from paper_2202_13927_gb300 import workloads as W


def _always(sc, gmax=20.0):
    """Glucagon mode in every period with the largest microbolus."""
    return dict(sc, glucagon=True, gg_threshold=1e6, gg_gain=1e9, gg_max_ug=gmax)


def test_two_compartment_chain_matches_the_exact_euler_solution():
    # constant infusion r = gmax/Ts from Z1 = Z2 = 0; with a = 1 - h/tau the
    # recursion z1' = a z1 + h r, z2' = a z2 + (h/tau) z1 has the closed form
    #   z1_n = r tau (1 - a^n),  z2_n = r tau (1 - a^n - n (h/tau) a^(n-1))
    pop = W.population(3, 41, sigma_q1=0.0)
    people = O.create_population(pop)
    sc = _always(W.scenario(1, horizon_periods=60), gmax=15.0)
    res = O.simulate(pop, people, sc, {}, trace_z=True)
    tau, ts, m = pop["tau_gg_min"], 5.0, 10
    h = ts / m
    r = 15.0 / ts
    a = 1.0 - h / tau
    n = np.arange(60) * m
    z1 = r * tau * (1.0 - a ** n)
    z2 = r * tau * (1.0 - a ** n - n * (h / tau) * np.where(n > 0, a ** (n - 1.0), 0.0))
    for i in range(3):
        np.testing.assert_allclose(res["z"][i, :, 0], z1, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(res["z"][i, :, 1], z2, rtol=1e-12, atol=1e-12)
    # everything infused is in the compartments or has left Z2 (mass balance)
    assert np.all(res["z"][:, -1, 0] + res["z"][:, -1, 1] < r * h * n[-1])


def test_glucagon_raises_q1_by_egp0_s_gg_z2_in_the_first_step_it_acts():
    # m = 3 steps of h = 0.5 min: Z2 is 0 in steps 0 and 1 and (h/tau) h r in
    # step 2, so after one period Q1 differs from the run with s_gg = 0 by
    # exactly h EGP0 s_gg (h/tau) h r and nothing else has moved yet
    base = W.population(4, 42, sigma_q1=0.0)
    people = O.create_population(base)
    sc = _always(W.scenario(1, horizon_periods=2), gmax=12.0)
    o = {"ts_min": 1.5, "substeps": 3}
    s_gg = 0.8
    on = O.simulate(dict(base, s_gg=s_gg), people, sc, o, trace_x=True)["x"]
    off = O.simulate(dict(base, s_gg=0.0), people, sc, o, trace_x=True)["x"]
    h, tau, r = 0.5, base["tau_gg_min"], 12.0 / 1.5
    egp0 = people["rows"][:, 0]
    dq1 = on[:, 1, 8] - off[:, 1, 8]
    np.testing.assert_allclose(dq1, h * egp0 * s_gg * (h / tau) * h * r, rtol=1e-9)
    other = [j for j in range(11) if j != 8]
    np.testing.assert_array_equal(on[:, 1, other], off[:, 1, other])
    np.testing.assert_array_equal(on[:, 0], off[:, 0])


def test_a_threshold_never_reached_leaves_the_insulin_loop_unchanged():
    pop = W.population(40, 43)
    people = O.create_population(pop)
    sc = W.scenario(2)
    off = O.simulate(pop, people, sc, {})["stats"]
    never = O.simulate(pop, people, dict(sc, glucagon=True, gg_threshold=-1.0), {})["stats"]
    assert off.tobytes() == never.tobytes()
    assert np.all(never["glucagon_ug"] == 0.0)


def test_glucagon_mode_withholds_insulin_and_counts_every_microbolus():
    pop = W.population(20, 44)
    people = O.create_population(pop)
    sc = _always(W.scenario(1), gmax=20.0)
    st = O.simulate(pop, people, sc, {})["stats"]
    ok = people["status"] == 0
    assert np.all(st["basal_u"][ok] == 0.0) and np.all(st["bolus_u"][ok] == 0.0)
    np.testing.assert_array_equal(st["glucagon_ug"][ok], 20.0 * W.PERIODS_PER_DAY)
    # a microbolus below the cap is proportional to the distance below the threshold
    sc2 = dict(W.scenario(1), glucagon=True, gg_threshold=50.0, gg_gain=0.5, gg_max_ug=1e9)
    res = O.simulate(pop, people, sc2, {}, trace_y=True)
    y = res["y"][ok]
    np.testing.assert_allclose(res["stats"]["glucagon_ug"][ok],
                               np.where(y < 50.0, 0.5 * (50.0 - y), 0.0).sum(axis=1), rtol=1e-12)


def test_glucagon_mode_shortens_hypoglycaemia():
    # a controller that believes the basal 50 % too high drives patients low;
    # the glucagon mode must cut the time below 70 mg/dL, and larger
    # microboli must cut it further
    pop = W.population(200, 45)
    people = O.create_population(pop)
    sc = W.scenario(3, basal_scale=1.5)
    ok = people["status"] == 0
    low = []
    for extra in ({}, {"glucagon": True}, {"glucagon": True, "gg_gain": 40.0, "gg_max_ug": 40.0}):
        st = O.simulate(pop, people, dict(sc, **extra), {})["stats"][ok]
        low.append(int(st["tir"][:, :2].sum()))
        if extra:
            assert st["glucagon_ug"].sum() > 0.0
    assert low[0] > 0 and low[1] < 0.8 * low[0] and low[2] < low[1]
