"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of ``oracle/vct_oracle.c`` (a dropped
term, a wrong sign, scale, index or constant, a boundary moved by one), builds
the copy, swaps it in for the oracle's library and runs the pin that should
catch it: the pin must fail.  The numpy oracles (``popstats.py``, ``mlp.py``)
get the same treatment, their copies executed as fresh modules.  The
committed oracle is never touched; the C copies live in pytest's temporary
directory.
"""
import pytest

from oracle import oracle as O
from tests import test_day_doses_oracle as DD
from tests import test_glucagon_oracle as GG
from tests import test_golden_paper as GP
from tests import test_oracle_pins as P
from tests import test_protocol as PR

# (name, original text, mistake, pin); the original must occur in the source
MUTANTS = [
    # Eq. 1 drift, Hovorka's glucose subsystem
    ("drop_k12_q2_in_q1", "- x[XO_X1] * x[XO_Q1] + p[VO_K12] * x[XO_Q2] + u_g +",
     "- x[XO_X1] * x[XO_Q1] + u_g +", P.test_basal_state_is_a_fixed_point_of_the_closed_loop),
    ("q2_loss_sign", "- (p[VO_K12] + x[XO_X2]) * x[XO_Q2];", "+ (p[VO_K12] + x[XO_X2]) * x[XO_Q2];",
     P.test_basal_state_is_a_fixed_point_of_the_closed_loop),
    ("egp_sign", "bw * (1.0 - x[XO_X3]);", "bw * (1.0 + x[XO_X3]);",
     P.test_basal_state_is_a_fixed_point_of_the_closed_loop),
    ("x2_uses_s_it", "p[VO_KA2] * p[VO_SID] * x[XO_I]", "p[VO_KA2] * p[VO_SIT] * x[XO_I]",
     P.test_insulin_step_reaches_closed_form_steady_state),
    ("plasma_insulin_scale", "x[XO_S2] / (p[VO_TAUS] * p[VO_VI] * bw)", "x[XO_S2] / (p[VO_VI] * bw)",
     P.test_insulin_step_reaches_closed_form_steady_state),
    ("renal_slope", "0.003 * (g - 9.0)", "0.03 * (g - 9.0)",
     lambda: P.test_ornstein_uhlenbeck_branches_exact_em_moments("renal")),
    ("f01c_kink", "p[VO_F01] * bw * g / 4.5", "p[VO_F01] * bw * g / 4.0",
     lambda: P.test_ornstein_uhlenbeck_branches_exact_em_moments("low_glucose")),
    ("cgm_lag_doubled", "(g - x[XO_GSC]) / p[VO_TAUCGM]", "(g - x[XO_GSC]) / (2.0 * p[VO_TAUCGM])",
     P.test_cgm_lag_closed_form),
    # meals (grams to mmol, A_G)
    ("carb_mmol_factor", "(1000.0 / 180.16)", "(1000.0 / 18.016)", P.test_meal_mass_balance_and_timing),
    ("drop_ag", "f[XO_D1] = p[VO_AG] * d -", "f[XO_D1] = d -", P.test_meal_mass_balance_and_timing),
    # Euler-Maruyama noise
    ("noise_scale_h", "d->sigma_q1 * sqrt(h)", "d->sigma_q1 * h", P.test_brownian_special_case_exact_law),
    # Philox4x32-10 and Box-Muller
    ("philox_weyl_constant", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;", P.test_philox_matches_curand_host_generator),
    ("philox_swapped_words", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;",
     P.test_philox_matches_curand_host_generator),
    ("box_muller_second_normal", "z[1] = r * sin(two_pi * u1);",
     "z[1] = r * cos(two_pi * u1);", P.test_box_muller_normals_moments_and_ks),
    ("uniform_without_half_offset", "return ((double)w + 0.5) * (1.0 / 4294967296.0);",
     "return ((double)w + 1.0) * (1.0 / 4294967296.0);", P.test_box_muller_at_the_extreme_words_in_closed_form),
    # measures (Sec. IV-A) and the controller (Eq. 3)
    ("upper_closed_bins", "if (g >= edges[e]) b++;", "if (g > edges[e]) b++;",
     P.test_bins_are_lower_closed_at_an_exact_edge),
    ("near_edge_window_open", "if (fabs(g - edges[e]) <= o->edge_band[w][e])",
     "if (fabs(g - edges[e]) < o->edge_band[w][e])", P.test_near_edge_counts_special_cases),
    ("near_edge_wrong_window", "<= o->edge_band[w][e]) st->near_edge[w][e]++;",
     "<= o->edge_band[0][e]) st->near_edge[w][e]++;", P.test_near_edge_counts_equal_trace_recount),
    ("hypo_edge_moved", "70.0 / 18.0", "72.0 / 18.0", lambda: GP.test_range_edges_are_the_printed_ones(1)),
    ("derivative_sign", "(y - y_prev) / ts", "(y_prev - y) / ts", P.test_derivative_action_telescopes),
    ("no_integral_clamp", "if (integral > sc->i_max) integral = sc->i_max;", "",
     P.test_pi_action_removes_a_wrong_basal_belief_unless_the_integral_saturates),
    # population draw (Sec. IV-B)
    ("acceptance_two_sd", "fabs(zt) <= 1.0", "fabs(zt) <= 2.0", P.test_population_acceptance_rule),
    ("basal_rule_units", "u * 60.0 / 1000.0 < d->min_basal_u_per_h", "u * 60.0 / 100.0 < d->min_basal_u_per_h",
     P.test_population_acceptance_rule),
    # glucagon (Sec. IV-B, IV-C) and the daily doses (Fig. 5)
    ("glucagon_effect_scale", "f[XO_Q1] += p[VO_EGP0] * d->s_gg * z2;", "f[XO_Q1] += d->s_gg * z2;",
     GG.test_glucagon_raises_q1_by_egp0_s_gg_z2_in_the_first_step_it_acts),
    ("bolus_in_glucagon_mode", "if (glucagon_mode) bolus_u = 0.0;", "",
     GG.test_glucagon_mode_withholds_insulin_and_counts_every_microbolus),
    ("day_boundary_off_by_one", "if ((k + 1) % per_day == 0) {", "if (k % per_day == 0) {",
     DD.test_constant_controller_gives_exact_daily_basal_and_bolus_per_meal),
    # measurement and meal noise (Eq. 1d; the meal reading)
    ("cgm_noise_squared", "d->cgm_sd * cgm_normal(", "d->cgm_sd * d->cgm_sd * cgm_normal(",
     P.test_cgm_measurement_noise_law),
    ("meal_draw_shared_across_days", "(uint32_t)(day * sc->n_meals + j)", "(uint32_t)(day + j)",
     P.test_meal_carbs_are_independent_draws),
    ("meal_noise_scale", "sc->meal_mean_g + sc->meal_sd_g * meal_normal",
     "sc->meal_mean_g + sc->meal_sd_g * sc->meal_sd_g * meal_normal", P.test_meal_carbs_are_independent_draws),
    # controller (Eq. 3), bolus rule and limits
    ("kp_sign", "ub_hat + kp * e_k", "ub_hat - kp * e_k",
     P.test_pi_action_removes_a_wrong_basal_belief_unless_the_integral_saturates),
    ("ki_times_ti", "sc->ki_mult * kp_nom / sc->ti_min", "sc->ki_mult * kp_nom * sc->ti_min",
     P.test_pi_action_removes_a_wrong_basal_belief_unless_the_integral_saturates),
    ("derivative_at_first_period", "k == 0 ? 0.0 : (y - y_prev) / ts", "(y - y_prev) / ts",
     P.test_derivative_action_telescopes),
    ("basal_belief_not_scaled", "sc->basal_scale * job->ub[i]", "job->ub[i]",
     P.test_insulin_step_reaches_closed_form_steady_state),
    ("tdd_of_one_day", "2.0 * 24.0 * (ub_hat", "24.0 * (ub_hat", PR.test_protocol_bolus_closed_form),
    ("protocol_meal_for_70kg", "double grams = (double)dp->g_per_kg[j] * p[VO_BW];",
     "double grams = (double)dp->g_per_kg[j] * 70.0;", PR.test_protocol_bolus_closed_form),
    ("no_insulin_floor", "if (u_pid < 0.0) u_pid = 0.0;", "", P.test_insulin_rate_is_never_negative),
    ("no_glucagon_cap", "if (gg > sc->gg_max_ug) gg = sc->gg_max_ug;", "",
     DD.test_always_glucagon_mode_gives_the_cap_every_period_and_partial_days_are_left_out),
    ("z2_chain_rate", "fz2 = (z1 - z2) / tau_gg;", "fz2 = (z1 - 2.0 * z2) / tau_gg;",
     GG.test_two_compartment_chain_matches_the_exact_euler_solution),
    ("no_q1_clamp", "if (x[XO_Q1] < 0.0) {", "if (x[XO_Q1] < -1e300) {", P.test_q1_is_clamped_at_zero_and_counted),
    ("renal_threshold", "g > 9.0 ? 0.003", "g > 10.0 ? 0.003",
     lambda: P.test_ornstein_uhlenbeck_branches_exact_em_moments("renal")),
    # indicators (Sec. III-C, IV-A)
    ("no_episode_at_first_sample", "(k == 0 || g_prev >= edges[1])", "(g_prev >= edges[1])",
     P.test_a_run_that_starts_low_is_one_hypoglycaemia_episode),
    ("variance_without_mean", "ss += (gbuf[j] - mean) * (gbuf[j] - mean);", "ss += gbuf[j] * gbuf[j];",
     P.test_online_indicators_equal_trace_recomputation),
    # basal steady state (the state every run starts from)
    ("basal_q2", "x0[XO_Q2] = x1 * q1 / (p[VO_K12] + x2);", "x0[XO_Q2] = x1 * q1 / p[VO_K12];",
     P.test_basal_state_is_a_fixed_point_of_the_closed_loop),
    ("basal_s1", "x0[XO_S1] = ub * p[VO_TAUS];", "x0[XO_S1] = ub;",
     P.test_basal_state_is_a_fixed_point_of_the_closed_loop),
]


@pytest.fixture(scope="module")
def source():
    with open(O._SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(name, old, new, pin, source, tmp_path, monkeypatch):
    assert old in source, name
    src = tmp_path / f"{name}.c"
    src.write_text(source.replace(old, new))
    mutant = O.load(O.compile_source(str(src), str(tmp_path / f"lib{name}.so")))
    monkeypatch.setattr(O, "_lib", mutant)
    try:
        pin()
    except AssertionError:
        return
    pytest.fail(f"the pin {getattr(pin, '__name__', pin)} passed with '{name}' planted")


def test_unmutated_copy_passes_the_same_pins(source, tmp_path, monkeypatch):
    """The harness itself: a faithful copy built the same way passes every pin."""
    src = tmp_path / "copy.c"
    src.write_text(source)
    monkeypatch.setattr(O, "_lib", O.load(O.compile_source(str(src), str(tmp_path / "libcopy.so"))))
    for _, _, _, pin in MUTANTS:
        pin()


# The numpy oracles: the mistake is planted in a copy of the module's source,
# executed as a fresh module and put in place of the module the pins call.
from oracle import mlp as _mlp  # noqa: E402
from oracle import popstats as _popstats  # noqa: E402
from tests import test_mlp_oracle as ML  # noqa: E402
from tests import test_popstats_oracle as PS  # noqa: E402

PY_MUTANTS = [
    # population reductions (Sec. IV-D, Fig. 3)
    ("quantile_interpolated", _popstats, PS, "OP", 'method="inverted_cdf"', 'method="linear"',
     PS.test_hand_worked_four_patient_example),
    ("worst_ties_to_highest_id", _popstats, PS, "OP", "j = int(np.argmin(gmin))",
     "j = int(len(gmin) - 1 - np.argmin(gmin[::-1]))",
     PS.test_flagged_patients_are_left_out_and_ties_go_to_the_lowest_id),
    ("worst_id_of_the_filtered_list", _popstats, PS, "OP", "int(ids[j]) + first_patient",
     "int(j) + first_patient", PS.test_flagged_patients_are_left_out_and_ties_go_to_the_lowest_id),
    ("sample_variance", _popstats, PS, "OP", "gm.var()", "gm.var(ddof=1)",
     PS.test_hand_worked_four_patient_example),
    ("span_not_cumulative", _popstats, PS, "OP", "cum.min(axis=0)", "t[:, :4].min(axis=0)",
     PS.test_hand_worked_four_patient_example),
    ("flags_ignored", _popstats, PS, "OP", "ok = np.asarray(status) == 0",
     "ok = np.ones(len(status), bool)", PS.test_flagged_patients_are_left_out_and_ties_go_to_the_lowest_id),
    ("histogram_rounds", _popstats, PS, "OP", "np.floor(g.ravel() * (1.0 / width))",
     "np.round(g.ravel() * (1.0 / width))", PS.test_bg_histogram_bins_by_hand),
    ("cdf_not_cumulative", _popstats, PS, "OP", "c = np.cumsum(h, axis=-1)", "c = h",
     PS.test_cdf_of_a_histogram_by_hand),
    ("dose_rank_floored", _popstats, PS, "OP", "r = max(int(np.ceil(q * d.size)), 1)",
     "r = max(int(q * d.size), 1)", PS.test_dose_quantiles_by_hand),
    ("dose_lower_edge", _popstats, PS, "OP", "(b[r - 1] + 1.0) * width", "b[r - 1] * width",
     PS.test_dose_quantiles_by_hand),
    ("bg_cdf_upper_bin_open", _popstats, PS, "OP", "(b <= j).sum() / n", "(b < j).sum() / n",
     PS.test_bg_cdf_from_samples_by_hand),
    # surrogate network and AdamW
    ("relu_mask_of_wrong_layer", _mlp, ML, "M", 'dz2 = dh2 * (cache["z2"] > 0)', 'dz2 = dh2 * (cache["z1"] > 0)',
     ML.test_gradients_match_finite_differences),
    ("w2_not_transposed", _mlp, ML, "M", 'dh1 = dz2 @ params["W2"]', 'dh1 = dz2 @ params["W2"].T',
     ML.test_gradients_match_finite_differences),
    ("gradient_not_averaged", _mlp, ML, "M", "- t) / b", "- t)", ML.test_gradients_match_finite_differences),
    ("no_bias_correction", _mlp, ML, "M", "mhat = m / (1.0 - beta1 ** step)", "mhat = m",
     ML.test_first_adamw_step_closed_form),
    ("decay_on_biases", _mlp, ML, "M", 'if k.startswith("W"):', "if True:", ML.test_first_adamw_step_closed_form),
    ("momentum_with_beta2", _mlp, ML, "M", "m[...] = beta1 * m", "m[...] = beta2 * m",
     ML.test_constant_gradient_adamw_steps_in_closed_form),
    ("softmax_without_normaliser", _mlp, ML, "M", "p = e / e.sum(axis=1, keepdims=True)", "p = e",
     ML.test_cross_entropy_minimum_is_the_entropy),
]


def _module_from(module, text, name):
    import types
    m = types.ModuleType(f"{module.__name__}_{name}")
    m.__file__ = module.__file__
    exec(compile(text, module.__file__, "exec"), m.__dict__)
    return m


@pytest.mark.parametrize("name,module,tests_mod,attr,old,new,pin", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_numpy_pin_catches_planted_mistake(name, module, tests_mod, attr, old, new, pin, monkeypatch):
    with open(module.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, name
    monkeypatch.setattr(tests_mod, attr, _module_from(module, text.replace(old, new), name))
    try:
        pin()
    except AssertionError:
        return
    pytest.fail(f"the pin {pin.__name__} passed with '{name}' planted")


def test_unmutated_numpy_copies_pass_the_same_pins(monkeypatch):
    for _, module, tests_mod, attr, _, _, pin in PY_MUTANTS:
        with open(module.__file__) as f:
            copy = _module_from(module, f.read(), "copy")
        monkeypatch.setattr(tests_mod, attr, copy)
        pin()
        monkeypatch.undo()
