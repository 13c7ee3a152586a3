"""Pins of the FP64 oracle to facts outside itself (no GPU needed).

Each test checks the oracle against a library routine, a closed form, an
invariant or a statistical law fixed by the mathematics, chosen so that a
plausible slip (a dropped term, a wrong sign, index or scale) fails one of
them:

* Philox4x32-10 against cuRAND's host generator (library output);
* Box-Muller normals: moments and a Kolmogorov-Smirnov test;
* Euler-Maruyama with the model's own noise term: exact Gaussian law of a
  Brownian special case, exact discrete Ornstein-Uhlenbeck mean and
  variance on the low-glucose (F01c) and renal (F_R) branches;
* meal absorption: mass balance of the gut chain (A_G, 1000/180.16, timing);
* insulin chain: new steady state after a step in u (closed form) and the
  transient against the matrix exponential of the linear subsystem;
* the basal steady state is a fixed point of the whole closed loop;
* convergence order of Euler-Maruyama (1) and of RK4, deterministic and with
  common random numbers, pathwise (strong) and of the mean BG curve (weak);
* the population draw: truncated-normal marginals (KS) and the acceptance rule;
* the CGM lag in closed form, the CGM noise law (mean, variance, KS,
  independence) and the meal draws (daily carbs recovered from the boluses:
  mean, variance, independence across days);
* limits: the insulin rate's floor at zero and the counted Q1 clamp;
* the online indicators against the same quantities recomputed from traces,
  and a run that starts low as exactly one hypoglycaemia episode.
"""
import ctypes as C
import ctypes.util
import glob
import math
import os

import numpy as np
import pytest
from scipy import linalg, stats

from oracle import oracle as O
from paper_2202_13927_gb300 import workloads as W

IDX = {n: i for i, n in enumerate(O.PARAM_NAMES)}
SX = {n: i for i, n in enumerate(O.STATE_NAMES)}


# --------------------------------------------------------------------------- helpers
def _custom_people(row, x0, n, u_b=0.0):
    rows = np.tile(np.asarray(row, float), (n, 1))
    return {"rows": rows, "u_b": np.full(n, float(u_b)), "x0": np.tile(np.asarray(x0, float), (n, 1)),
            "first": 0}


def _nominal_row(**over):
    row = [W.NOMINAL[k] for k in O.PARAM_NAMES] + [75.0]
    for k, v in over.items():
        row[IDX[k] if k != "BW" else 16] = v
    return np.asarray(row, float)


def _glucose_only_row(**over):
    """Insulin has no effect (S_I = 0) and Q2 is cut off (k12 = 0)."""
    base = dict(SIT=0.0, SID=0.0, SIE=0.0, k12=0.0)
    base.update(over)
    return _nominal_row(**base)


def _x0_at(row, g0):
    x = np.zeros(O.NX)
    x[SX["Q1"]] = g0 * row[IDX["VG"]] * row[16]
    x[SX["Gsc"]] = g0
    return x


def _quiet_pop(sigma=0.0, cgm=0.0, seed=11):
    return W.population(1, seed, sigma_q1=sigma, cgm_sd=cgm)


def _no_meal_scenario(periods, **kw):
    sc = W.scenario(0, horizon_periods=periods, meal_minute=(), **kw)
    return sc


# --------------------------------------------------------------------------- Philox
def _find_curand():
    cands = []
    lib = ctypes.util.find_library("curand")
    if lib:
        cands.append(lib)
    for pat in ("/usr/local/cuda/lib64/libcurand.so*", "/usr/local/cuda/targets/*/lib/libcurand.so*",
                "/usr/lib/*/libcurand.so*"):
        cands += sorted(glob.glob(pat))
    try:
        import nvidia  # noqa: F401
        base = os.path.dirname(nvidia.__file__)
        cands += sorted(glob.glob(os.path.join(base, "*", "lib", "libcurand.so*")))
        cands += sorted(glob.glob(os.path.join(base, "*", "*", "lib", "libcurand.so*")))
    except Exception:
        pass
    for c in cands:
        try:
            return C.CDLL(c)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator, seed s, emits block b of four words
    as Philox(counter = (b // 65536, 0, b % 65536, 0), key = (s_lo, s_hi)); the
    oracle's independent implementation must reproduce it word for word."""
    cu = _find_curand()
    if cu is None:
        pytest.skip("libcurand not found")
    gen = C.c_void_p()
    assert cu.curandCreateGeneratorHost(C.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        for seed in (0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 7):
            assert cu.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
            assert cu.curandSetGeneratorOffset(gen, C.c_ulonglong(0)) == 0
            n_blocks = 65536 + 64
            out = np.zeros(4 * n_blocks, np.uint32)
            assert cu.curandGenerate(gen, out.ctypes.data_as(C.c_void_p), C.c_size_t(out.size)) == 0
            key = [seed & 0xFFFFFFFF, seed >> 32]
            picks = list(range(0, 40)) + [1000, 4095, 65535] + list(range(65536, 65536 + 64, 7))
            for b in picks:
                ctr = [b // 65536, 0, b % 65536, 0]
                np.testing.assert_array_equal(O.philox(ctr, key), out[4 * b:4 * b + 4])
    finally:
        cu.curandDestroyGenerator(gen)


def test_philox_every_counter_and_key_word_matters():
    base = np.array([3, 5, 7, 11], np.uint32)
    key = [0x12345678, 0x9ABCDEF0]
    ref = O.philox(base, key)
    for w in range(4):
        c = base.copy()
        c[w] ^= 1
        diff = np.unpackbits((O.philox(c, key) ^ ref).view(np.uint8)).sum()
        assert 40 < diff < 88, (w, diff)  # avalanche: about half of 128 bits flip
    for w in range(2):
        k = list(key)
        k[w] ^= 1
        diff = np.unpackbits((O.philox(base, k) ^ ref).view(np.uint8)).sum()
        assert 40 < diff < 88


# --------------------------------------------------------------------------- normals
def test_box_muller_at_the_extreme_words_in_closed_form():
    """The uniforms are (w + 1/2) 2^-32, strictly inside (0, 1): the smallest
    word gives u0 = 2^-33 and the radius sqrt(66 ln 2), the largest gives
    u0 = 1 - 2^-33 and the radius sqrt(-2 ln(1 - 2^-33)) ~ 2^-16 (an offset of 0
    or 1 instead of 1/2 would give an infinite radius, or one sqrt(2) times this
    one, or 0); the angle is 2 pi (w1 + 1/2) 2^-32, so w1 = 2^30 - 1 and 2^30
    put it half a step either side of a quarter turn."""
    import mpmath as mp
    mp.mp.dps = 40
    u_lo, u_hi = mp.mpf(2) ** -33, 1 - mp.mpf(2) ** -33
    r_lo = float(mp.sqrt(-2 * mp.log(u_lo)))
    r_hi = float(mp.sqrt(-2 * mp.log(u_hi)))
    assert r_lo == pytest.approx(math.sqrt(66.0 * math.log(2.0)), rel=1e-15)
    for w1 in (0, 12345, (1 << 30) - 1, 1 << 30, 0xFFFFFFFF):
        ang = 2 * mp.pi * (mp.mpf(w1) + mp.mpf("0.5")) * mp.mpf(2) ** -32
        for w0, r in ((0, r_lo), (0xFFFFFFFF, r_hi)):
            z = O.box_muller(w0, w1)
            np.testing.assert_allclose(z, [r * float(mp.cos(ang)), r * float(mp.sin(ang))],
                                       rtol=1e-12, atol=1e-12 * r)
            assert math.hypot(*z) == pytest.approx(r, rel=1e-12)
    # a quarter turn lies between w1 = 2^30 - 1 and 2^30: the cosines have opposite signs
    assert O.box_muller(0, (1 << 30) - 1)[0] > 0 > O.box_muller(0, 1 << 30)[0]


def test_box_muller_normals_moments_and_ks():
    key = [2024, 7]
    z = np.concatenate([O.normals4([i, 17, 3, 0], key) for i in range(50000)])
    n = z.size
    se = 1.0 / math.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.skew(z)) < 5 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the two normals of one pair are uncorrelated, and so are the pairs
    zz = z.reshape(-1, 4)
    for a, b in ((0, 1), (2, 3), (0, 2), (1, 3)):
        assert abs(np.corrcoef(zz[:, a], zz[:, b])[0, 1]) < 5 * math.sqrt(1.0 / zz.shape[0])
    # each slot alone is standard normal
    for a in range(4):
        assert stats.kstest(zz[:, a], "norm").pvalue > 1e-4


# --------------------------------------------------------------------------- EM + noise, closed forms
def test_brownian_special_case_exact_law():
    """S_I = 0, k12 = 0, EGP0 = F01, no meal, 4.5 < G < 9: Q1' = sigma dW exactly,
    so Q1(t_k) - Q1(0) ~ N(0, sigma^2 k Ts) under Euler-Maruyama for any h."""
    sigma = 0.1
    row = _glucose_only_row(EGP0=W.NOMINAL["F01"])
    n, periods = 4000, 288
    pop = _quiet_pop(sigma=sigma)
    people = _custom_people(row, _x0_at(row, 6.0), n)
    res = O.simulate(pop, people, _no_meal_scenario(periods), {"substeps": 10}, trace_x=True)
    q1 = res["x"][:, :, SX["Q1"]]
    q10 = people["x0"][0, SX["Q1"]]
    for k in (1, 17, 144, periods - 1):
        dq = q1[:, k] - q10
        var = sigma ** 2 * k * 5.0
        assert abs(dq.mean()) < 5 * math.sqrt(var / n)
        assert abs(dq.var(ddof=1) / var - 1.0) < 5 * math.sqrt(2.0 / (n - 1))
    # the increments of different periods are independent
    inc = np.diff(q1[:, :50], axis=1)
    c = np.corrcoef(inc[:, 10], inc[:, 11])[0, 1]
    assert abs(c) < 5 / math.sqrt(n)


def _discrete_ou(q0, qstar, theta, sigma, h, nsteps):
    a = 1.0 - theta * h
    mean = qstar + (q0 - qstar) * a ** nsteps
    var = sigma ** 2 * h * (1.0 - a ** (2 * nsteps)) / (1.0 - a * a)
    return mean, var


@pytest.mark.parametrize("branch", ["low_glucose", "renal"])
def test_ornstein_uhlenbeck_branches_exact_em_moments(branch):
    """Below 4.5 mmol/L, F01c = F01 BW G/4.5 is linear in Q1; above 9 mmol/L,
    F_R = 0.003 (G - 9) V_G BW is too.  With S_I = 0, k12 = 0 the Q1 equation is
    an OU process whose Euler-Maruyama recursion Q_{n+1} = a Q_n + h c + s sqrt(h) z
    has exact mean Q* + (Q_0 - Q*) a^n and variance s^2 h (1 - a^2n)/(1 - a^2)."""
    sigma, bw, vg, f01 = 0.1, 75.0, W.NOMINAL["VG"], W.NOMINAL["F01"]
    if branch == "low_glucose":
        theta = f01 / (4.5 * vg)
        egp0 = f01 * 3.0 / 4.5          # Q* at G = 3
        qstar = egp0 * bw / theta
        g0 = 3.5
    else:
        theta = 0.003
        egp0 = f01 + 0.003 * vg * 3.0   # Q* at G = 12
        qstar = 9.0 * vg * bw + (egp0 - f01) * bw / theta
        g0 = 10.0
    row = _glucose_only_row(EGP0=egp0)
    n, periods, m = 4000, 400, 10
    h = 5.0 / m
    people = _custom_people(row, _x0_at(row, g0), n)
    res = O.simulate(_quiet_pop(sigma=sigma), people, _no_meal_scenario(periods), {"substeps": m},
                     trace_x=True)
    q1 = res["x"][:, :, SX["Q1"]]
    q0 = people["x0"][0, SX["Q1"]]
    for k in (1, 50, 200, periods - 1):
        mean, var = _discrete_ou(q0, qstar, theta, sigma, h, k * m)
        assert abs(q1[:, k].mean() - mean) < 5 * math.sqrt(var / n)
        assert abs(q1[:, k].var(ddof=1) / var - 1.0) < 5 * math.sqrt(2.0 / (n - 1))
    # noise-free: the mean recursion is exact to rounding
    res0 = O.simulate(_quiet_pop(sigma=0.0), _custom_people(row, _x0_at(row, g0), 1),
                      _no_meal_scenario(periods), {"substeps": m}, trace_x=True)
    for k in (1, 77, periods - 1):
        mean, _ = _discrete_ou(q0, qstar, theta, 0.0, h, k * m)
        assert res0["x"][0, k, SX["Q1"]] == pytest.approx(mean, rel=1e-12)


# --------------------------------------------------------------------------- meal mass balance
def test_meal_mass_balance_and_timing():
    """With S_I = 0, k12 = 0 and EGP0 = F01 the gut chain feeds Q1 only:
    D1 + D2 + Q1 rises by exactly A_G * carbs * 1000/180.16 mmol after the meal
    (Euler-Maruyama keeps linear invariants), the meal starting at its period."""
    row = _glucose_only_row(EGP0=W.NOMINAL["F01"])
    carbs = 5.0
    sc = W.scenario(0, horizon_periods=288, meal_minute=(60.0,), meal_mean_g=carbs, meal_sd_g=0.0,
                    bolus=False)
    people = _custom_people(row, _x0_at(row, 6.0), 1)
    res = O.simulate(_quiet_pop(), people, sc, {"substeps": 10}, trace_x=True)
    x = res["x"][0]
    total = x[:, SX["D1"]] + x[:, SX["D2"]] + x[:, SX["Q1"]]
    q0 = people["x0"][0, SX["Q1"]]
    k_meal = 12
    assert np.all(x[: k_meal + 1, SX["D1"]] == 0.0)
    assert x[k_meal + 1, SX["D1"]] > 0.0
    np.testing.assert_allclose(total[: k_meal + 1], q0, rtol=1e-14)
    expect = q0 + W.NOMINAL["AG"] * carbs * 1000.0 / 180.16
    np.testing.assert_allclose(total[k_meal + 1:], expect, rtol=1e-12)
    # and it all reaches plasma glucose by the end of the day
    g_end = x[-1, SX["Q1"]] / (row[IDX["VG"]] * 75.0)
    assert g_end == pytest.approx(expect / (row[IDX["VG"]] * 75.0), rel=1e-6)


# --------------------------------------------------------------------------- CGM lag
def test_cgm_lag_closed_form():
    """The sensor follows plasma glucose through a first-order lag (Eq. 1d's
    CGM state).  With S_I = 0, k12 = 0, EGP0 = F01 and no meal, G stays at g0,
    so under Euler steps of h the sensor's offset decays as (1 - h/tau_CGM)^n."""
    row = _glucose_only_row(EGP0=W.NOMINAL["F01"])
    g0, off, periods, m = 6.0, 2.0, 48, 10
    x0 = _x0_at(row, g0)
    x0[SX["Gsc"]] = g0 + off
    people = _custom_people(row, x0, 1)
    res = O.simulate(_quiet_pop(), people, _no_meal_scenario(periods), {"substeps": m}, trace_x=True)
    x = res["x"][0]
    np.testing.assert_array_equal(x[:, SX["Q1"]], x0[SX["Q1"]])
    a = 1.0 - (5.0 / m) / row[IDX["tauCGM"]]
    k = np.arange(periods)
    np.testing.assert_allclose(x[:, SX["Gsc"]] - g0, off * a ** (m * k), rtol=1e-11, atol=1e-13)


# --------------------------------------------------------------------------- insulin chain
def test_insulin_step_reaches_closed_form_steady_state():
    """Open loop (gains 0) with the basal doubled: u = 2 u_b; after 4 days
    S1 = S2 = u tau_S, I = u / (V_I BW k_e), x_i = S_i I."""
    pop = W.population(8, 5, sigma_q1=0.0, cgm_sd=0.0)
    people = O.create_population(pop)
    sc = W.scenario(4, kp_mult=0.0, ki_mult=0.0, kd_mult=0.0, basal_scale=2.0, meal_minute=())
    res = O.simulate(pop, people, sc, {"substeps": 10}, trace_x=True)
    for i in range(8):
        p = people["rows"][i]
        u = 2.0 * people["u_b"][i]
        x = res["x"][i, -1]
        i_ss = u / (p[IDX["VI"]] * p[16] * p[IDX["ke"]])
        assert x[SX["S1"]] == pytest.approx(u * p[IDX["tauS"]], rel=1e-9)
        assert x[SX["S2"]] == pytest.approx(u * p[IDX["tauS"]], rel=1e-9)
        assert x[SX["I"]] == pytest.approx(i_ss, rel=1e-9)
        assert x[SX["x1"]] == pytest.approx(p[IDX["SIT"]] * i_ss, rel=1e-6)
        assert x[SX["x2"]] == pytest.approx(p[IDX["SID"]] * i_ss, rel=1e-9)
        assert x[SX["x3"]] == pytest.approx(p[IDX["SIE"]] * i_ss, rel=1e-9)


def test_insulin_transient_converges_to_matrix_exponential():
    """The insulin subsystem (S1, S2, I, x1, x2, x3) is linear for a held u; its
    exact solution is expm of the system matrix (Hovorka 2004 insulin
    equations).  Euler-Maruyama at h, h/2, h/4 converges to it at order 1."""
    pop = W.population(1, 5, sigma_q1=0.0, cgm_sd=0.0)
    people = O.create_population(pop)
    p = people["rows"][0]
    ub = people["u_b"][0]
    ts, periods = 5.0, 36
    sc = W.scenario(0, horizon_periods=periods, kp_mult=0, ki_mult=0, kd_mult=0, basal_scale=3.0,
                    meal_minute=())
    ts_, tau, vi, bw, ke = ts, p[IDX["tauS"]], p[IDX["VI"]], p[16], p[IDX["ke"]]
    ka = [p[IDX["ka1"]], p[IDX["ka2"]], p[IDX["ka3"]]]
    si = [p[IDX["SIT"]], p[IDX["SID"]], p[IDX["SIE"]]]
    A = np.zeros((7, 7))   # states S1 S2 I x1 x2 x3, last = constant input
    A[0, 0] = -1 / tau
    A[0, 6] = 3.0 * ub
    A[1, 0], A[1, 1] = 1 / tau, -1 / tau
    A[2, 1], A[2, 2] = 1 / (tau * vi * bw), -ke
    for j in range(3):
        A[3 + j, 3 + j] = -ka[j]
        A[3 + j, 2] = ka[j] * si[j]
    z0 = np.concatenate([people["x0"][0, [SX["S1"], SX["S2"], SX["I"], SX["x1"], SX["x2"],
                                          SX["x3"]]], [1.0]])
    exact = linalg.expm(A * ts_ * periods - A * ts_) @ z0  # state at t_{H-1}
    errs = []
    for m in (10, 20, 40):
        res = O.simulate(pop, people, sc, {"substeps": m}, trace_x=True)
        got = res["x"][0, -1, [SX["S1"], SX["S2"], SX["I"], SX["x1"], SX["x2"], SX["x3"]]]
        errs.append(np.max(np.abs(got - exact[:6]) / np.abs(exact[:6])))
    assert errs[0] < 2e-2
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


# --------------------------------------------------------------------------- steady state
def test_basal_state_is_a_fixed_point_of_the_closed_loop():
    pop = W.population(20, 9, sigma_q1=0.0, cgm_sd=0.0)
    people = O.create_population(pop)
    assert people["status"].sum() == 0
    sc = W.scenario(7, meal_minute=())
    res = O.simulate(pop, people, sc, {"substeps": 10}, trace_x=True, trace_u=True)
    x0 = people["x0"]
    scale = np.maximum(np.abs(x0), 1e-300)
    drift = np.abs(res["x"] - x0[:, None, :])
    assert np.all(drift[:, :, [0, 1]] == 0.0)           # no meal: gut stays empty
    rel = drift[:, :, 2:] / scale[:, None, 2:]
    assert rel.max() < 1e-12
    np.testing.assert_allclose(res["u"], people["u_b"][:, None] * np.ones_like(res["u"]), rtol=1e-12)
    for i in range(20):
        f = O.drift(people["rows"][i], x0[i], people["u_b"][i], 0.0)
        assert np.all(np.abs(f) <= 1e-14 * np.maximum(np.abs(x0[i]), 1.0))
    st = res["stats"]
    assert np.all(st["tir"][:, 2] == sc["horizon_periods"])
    np.testing.assert_allclose(st["g_mean"], pop["g_sp"], rtol=1e-13)


# --------------------------------------------------------------------------- convergence orders
def _g_trace(pop, people, sc, m, integrator=0, refine=1):
    return O.simulate(pop, people, sc, {"substeps": m, "integrator": integrator,
                                        "noise_refine": refine}, trace_g=True)["g"]


def test_deterministic_orders_em_and_rk4():
    pop = W.population(6, 21, sigma_q1=0.0, cgm_sd=0.0)
    people = O.create_population(pop)
    sc = W.scenario(1, meal_sd_g=0.0)
    ref = _g_trace(pop, people, sc, 300, integrator=1)  # RK4, h = 1 s
    em = [np.abs(_g_trace(pop, people, sc, m) - ref).max() for m in (5, 10, 20, 40)]
    for a, b in zip(em, em[1:]):
        assert 1.7 < a / b < 2.3, em
    rk = [np.abs(_g_trace(pop, people, sc, m, integrator=1) - ref).max() for m in (2, 4)]
    assert rk[0] / rk[1] > 6.0, rk        # the min/max kinks of F01c, F_R cap the ratio below 16
    assert rk[1] < em[-1] / 100


def test_stochastic_strong_order_one_with_common_noise():
    """Additive noise: Euler-Maruyama converges pathwise at order 1.  Coarse runs
    reuse the fine grid's normals, z = (sum of R fine normals)/sqrt(R)."""
    pop = W.population(8, 22, cgm_sd=0.0)
    people = O.create_population(pop)
    sc = W.scenario(1)
    fine = 80
    ref = _g_trace(pop, people, sc, fine, refine=1)
    errs = []
    for m in (5, 10, 20):
        errs.append(np.abs(_g_trace(pop, people, sc, m, refine=fine // m) - ref).max())
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a / b < 2.6, errs


def test_weak_order_one_of_the_mean_glucose_curve():
    """Weak order 1 of Euler-Maruyama: the population mean of G(t) (the mean
    BG curve of Fig. 3) has a bias proportional to h.  The patients are
    identical, so each is one independent noise path of the same SDE; the
    coarse runs reuse the fine normals, so the bias shows without Monte Carlo
    noise.  Against a reference at f substeps the bias at m substeps is
    C (1/m - 1/f), so one halving of h divides it by (1/m - 1/f)/(1/(2m) - 1/f)."""
    pop = W.population(200, 23, cgm_sd=0.0)
    pop["p_sd"] = [0.0] * len(pop["p_sd"])
    pop["bw_sd"] = 0.0
    people = O.create_population(pop)
    assert people["status"].sum() == 0 and np.ptp(people["rows"], axis=0).max() == 0.0
    sc = W.scenario(1, meal_sd_g=0.0)
    fine = 80
    ref = _g_trace(pop, people, sc, fine).mean(axis=0)
    bias = {m: np.abs(_g_trace(pop, people, sc, m, refine=fine // m).mean(axis=0) - ref).max()
            for m in (5, 10, 20, 40)}
    for m in (5, 10, 20):
        expect = (1 / m - 1 / fine) / (1 / (2 * m) - 1 / fine)
        assert abs(bias[m] / bias[2 * m] / expect - 1) < 0.1, (m, bias)
    # at the paper's h = 30 s (m = 10) the mean curve is biased by under 1 mg/dL
    assert bias[10] * 18.0 < 1.0, bias


# --------------------------------------------------------------------------- population
def test_population_marginals_are_truncated_normals():
    pop = W.population(4000, 31, min_basal_u_per_h=0.0)
    people = O.create_population(pop)
    assert people["status"].sum() == 0
    rows = people["rows"]
    for j in range(17):
        mean = pop["p_mean"][j] if j < 16 else pop["bw_mean"]
        sd = pop["p_sd"][j] if j < 16 else pop["bw_sd"]
        if sd == 0.0:
            assert np.all(rows[:, j] == mean)
            continue
        pv = stats.kstest(rows[:, j], stats.truncnorm(-1.0, 1.0, loc=mean, scale=sd).cdf).pvalue
        assert pv > 1e-4, (j, pv)
    # parameters are drawn independently
    c = np.corrcoef(rows[:, IDX["SIT"]], rows[:, IDX["ke"]])[0, 1]
    assert abs(c) < 5 / math.sqrt(4000)


def test_population_acceptance_rule():
    pop = W.population(3000, 32)
    people = O.create_population(pop)
    ok = people["status"] == 0
    assert ok.all()
    rows = people["rows"]
    mean = np.array(pop["p_mean"] + [pop["bw_mean"]])
    sd = np.array(pop["p_sd"] + [pop["bw_sd"]])
    assert np.all(rows >= 0)
    assert np.all(np.abs(rows - mean) <= sd * (1 + 1e-12))
    assert np.all(people["u_b"] * 60.0 / 1000.0 >= 0.4)
    assert people["attempts"].max() <= pop["max_attempts"]
    assert people["attempts"].mean() > 1.0          # the basal rule does reject sets
    # an impossible threshold rejects every patient after max_attempts
    bad = O.create_population(W.population(5, 33, min_basal_u_per_h=100.0, max_attempts=7))
    assert np.all(bad["status"] == 1) and np.all(bad["attempts"] == 7)


def test_population_is_a_function_of_the_global_patient_id():
    pop = W.population(100, 34)
    full = O.create_population(pop)
    tail = O.create_population(pop, n=40, first=60)
    np.testing.assert_array_equal(full["rows"][60:], tail["rows"])
    np.testing.assert_array_equal(full["u_b"][60:], tail["u_b"])


# --------------------------------------------------------------------------- indicators
def test_online_indicators_equal_trace_recomputation():
    pop = W.population(64, 41)
    people = O.create_population(pop)
    sc = W.scenario(3)
    res = O.simulate(pop, people, sc, {}, trace_g=True, trace_u=True)
    st, g, u = res["stats"], res["g"], res["u"]
    edges = np.array([54.0, 70.0, 180.0, 250.0]) / 18.0
    bins = (g[:, :, None] >= edges[None, None, :]).sum(axis=2)
    for b in range(5):
        np.testing.assert_array_equal(st["tir"][:, b], (bins == b).sum(axis=1))
    low = g < edges[1]
    starts = low[:, 0].astype(int) + (low[:, 1:] & ~low[:, :-1]).sum(axis=1)
    np.testing.assert_array_equal(st["hypo_episodes"], starts)
    np.testing.assert_allclose(st["g_mean"], g.mean(axis=1), rtol=1e-13)
    np.testing.assert_allclose(st["g_var"], g.var(axis=1), rtol=1e-10)
    np.testing.assert_array_equal(st["g_min"], g.min(axis=1))
    np.testing.assert_array_equal(st["g_max"], g.max(axis=1))
    np.testing.assert_allclose(st["basal_u"] + st["bolus_u"], u.sum(axis=1) * 5.0 / 1000.0,
                               rtol=1e-12)
    assert np.all(st["n_samples"] == sc["horizon_periods"])
    assert st["hypo_episodes"].sum() > 0 and st["tir"][:, 3].sum() > 0


def test_near_edge_counts_equal_trace_recount():
    """The per-patient near-edge counts (the samples that may change range under
    rounding, used to excuse range-count differences) recounted from the trace
    for both default windows and for a wide window of 0.3 mmol/L."""
    pop = W.population(48, 43)
    people = O.create_population(pop)
    sc = W.scenario(3)
    edges = np.array(O.EDGES_MMOL)
    wide = (0.3, 0.3, 0.3, 0.3)
    for bands in (O.EDGE_BANDS, (wide, tuple(0.1 * edges))):
        res = O.simulate(pop, people, sc, {"edge_band": bands}, trace_g=True)
        g = res["g"]
        for w in range(2):
            band = np.asarray(bands[w])
            want = (np.abs(g[:, :, None] - edges[None, None, :]) <= band[None, None, :]).sum(axis=1)
            np.testing.assert_array_equal(res["stats"]["near_edge"][:, w, :], want)
        if bands[0] == wide:
            assert res["stats"]["near_edge"][:, 0, :].sum() > 100   # the case is not empty


def test_near_edge_counts_special_cases():
    """A sample exactly at an edge is near it for every window, zero included;
    an unbounded window counts every sample at every edge."""
    row = _nominal_row(VG=0.125, BW=80.0)
    rc, ub, x0 = O.basal(row, 10.0)          # G = 10 mmol/L = 180 mg/dL exactly
    assert rc == 0
    people = {"rows": row[None, :], "u_b": np.array([ub]), "x0": x0[None, :], "first": 0}
    pop = W.population(1, 1, sigma_q1=0.0, cgm_sd=0.0, g_sp=10.0)
    st = O.simulate(pop, people, _no_meal_scenario(1), {"edge_band": ((0.0,) * 4, (1e300,) * 4)})["stats"]
    assert list(st["near_edge"][0, 0]) == [0, 0, 1, 0]
    assert list(st["near_edge"][0, 1]) == [1, 1, 1, 1]


def test_a_run_that_starts_low_is_one_hypoglycaemia_episode():
    """An episode starts when a sample enters the range below 70 mg/dL; a patient
    held at rest at 3.5 mmol/L (63 mg/dL) is below from its first sample on, so
    the whole run is exactly one episode, all of it in the 54-70 range."""
    row = _nominal_row()
    rc, ub, x0 = O.basal(row, 3.5)
    assert rc == 0
    people = {"rows": row[None, :], "u_b": np.array([ub]), "x0": x0[None, :], "first": 0}
    pop = W.population(1, 1, sigma_q1=0.0, cgm_sd=0.0, g_sp=3.5)
    st = O.simulate(pop, people, _no_meal_scenario(100), {})["stats"]
    assert st["hypo_episodes"][0] == 1
    assert list(st["tir"][0]) == [0, 100, 0, 0, 0]


# --------------------------------------------------------------------------- measurement and meal noise
def test_cgm_measurement_noise_law():
    """Eq. 1d: y_k = Gsc(t_k) + v_k, v_k ~ N(0, R) independent over k and
    patients.  Without process noise the sensor state is known at t_k, so
    y - Gsc is the measurement noise itself (whatever the controller does)."""
    sd = 0.2
    n_pat, periods = 2000, 48
    pop = W.population(n_pat, 42, sigma_q1=0.0, cgm_sd=sd)
    people = O.create_population(pop)
    res = O.simulate(pop, people, _no_meal_scenario(periods), {}, trace_y=True, trace_x=True)
    v = res["y"] - res["x"][:, :, SX["Gsc"]]
    n = v.size
    assert abs(v.mean()) < 5 * sd / math.sqrt(n)
    assert abs(v.var() / sd ** 2 - 1.0) < 5 * math.sqrt(2.0 / n)
    assert stats.kstest(v.ravel() / sd, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(v[:, 10], v[:, 11])[0, 1]) < 5 / math.sqrt(n_pat)
    assert abs(np.corrcoef(v[0::2, 20], v[1::2, 20])[0, 1]) < 5 / math.sqrt(n_pat / 2)


def test_meal_carbs_are_independent_draws():
    """Meal carbs are N(mean, sd) per meal (clipped at 0, which at 5 SD never
    acts), drawn independently for every meal of every day.  The bolus of a
    day is its carbs times TDD/500, so each day's carbs are recovered from
    the daily bolus: three meals give mean 3 x 50 g and variance 3 x 10^2, and
    consecutive days are uncorrelated."""
    n_pat, days = 2000, 4
    pop = W.population(n_pat, 43, sigma_q1=0.0, cgm_sd=0.0)
    people = O.create_population(pop)
    sc = W.scenario(days)
    res = O.simulate(pop, people, sc, {}, day_doses=True)
    tdd = 48.0 * sc["basal_scale"] * people["u_b"] * 60.0 / 1000.0
    carbs = res["day_doses"][:, :, 1] / (tdd / 500.0)[:, None]
    n = carbs.size
    assert abs(carbs.mean() - 150.0) < 5 * math.sqrt(300.0 / n)
    assert abs(carbs.var() / 300.0 - 1.0) < 5 * math.sqrt(2.0 / n)
    for d in range(days - 1):
        assert abs(np.corrcoef(carbs[:, d], carbs[:, d + 1])[0, 1]) < 5 / math.sqrt(n_pat)


# --------------------------------------------------------------------------- limits
def test_insulin_rate_is_never_negative():
    """Eq. 3's rate is floored at zero: a strong proportional gain drives the
    PID term below zero after meals' glucose falls back, and then the rate is
    exactly zero, never negative."""
    pop = W.population(64, 44)
    people = O.create_population(pop)
    res = O.simulate(pop, people, W.scenario(2, kp_mult=30.0), {}, trace_u=True)
    assert res["u"].min() == 0.0
    assert (res["u"] == 0.0).mean() > 0.01


def test_q1_is_clamped_at_zero_and_counted():
    """P8 reading: Q1 is clamped at zero after each step and the clamps are
    counted.  With no drift on Q1, one step per period and Q1 = 0 at the start,
    each step from zero goes below zero with probability 1/2; a sampled Q1 of
    exactly zero is a clamp (a continuous value never hits it), and every
    clamp but the one after the last sample is seen in the trace."""
    row = _glucose_only_row(EGP0=0.0, F01=0.0)
    n = 400
    people = _custom_people(row, _x0_at(row, 0.0), n)
    res = O.simulate(_quiet_pop(sigma=1.0), people, _no_meal_scenario(30), {"substeps": 1}, trace_x=True)
    q1 = res["x"][:, :, SX["Q1"]]
    assert q1.min() == 0.0
    first = (q1[:, 1] == 0.0).sum()
    assert abs(first - n / 2) < 5 * math.sqrt(n / 4)
    seen = (q1[:, 1:] == 0.0).sum(axis=1)
    extra = res["stats"]["q1_clamps"].astype(int) - seen
    assert extra.min() >= 0 and extra.max() <= 1


def test_nonfinite_parameters_are_flagged_not_fatal():
    pop = W.population(4, 42)
    people = O.create_population(pop)
    people["rows"][2, IDX["k12"]] = np.nan
    res = O.simulate(pop, people, W.scenario(1), {})
    st = res["stats"]
    assert st["status"][2] == 1 and st["n_samples"][2] == 0
    assert np.all(st["status"][[0, 1, 3]] == 0)


def test_bins_are_lower_closed_at_an_exact_edge():
    """V_G BW = 10 L and Q1 = 100 mmol give G = 10 mmol/L = 180 mg/dL exactly; a
    lower-closed range puts that sample in 180-250, not in 70-180."""
    row = _nominal_row(VG=0.125, BW=80.0)
    rc, ub, x0 = O.basal(row, 10.0)
    assert rc == 0
    assert x0[SX["Q1"]] / (0.125 * 80.0) == 10.0
    people = {"rows": row[None, :], "u_b": np.array([ub]), "x0": x0[None, :], "first": 0}
    pop = W.population(1, 1, sigma_q1=0.0, cgm_sd=0.0, g_sp=10.0)
    st = O.simulate(pop, people, _no_meal_scenario(1), {})["stats"]
    assert list(st["tir"][0]) == [0, 0, 0, 1, 0]


def test_pi_action_removes_a_wrong_basal_belief_unless_the_integral_saturates():
    # Eq. 3 with integral action: a controller whose basal belief is 20 % low
    # (or high) and no disturbance (no noise, meals or boluses) must bring the
    # plant back to the setpoint with the insulin rate equal to the true basal;
    # a belief 50 % low needs an integral beyond its clamp (i_max), so an offset
    # above the setpoint remains
    pop = W.population(4, 61, sigma_q1=0.0, cgm_sd=0.0)
    people = O.create_population(pop)
    ub_day = people["u_b"] * 60.0 * 24.0 / 1000.0     # U per day at the true basal rate
    for scale in (0.8, 1.2):
        sc = W.scenario(20, meal_minute=(), bolus=False, basal_scale=scale)
        r = O.simulate(pop, people, sc, {}, trace_y=True, day_doses=True)
        np.testing.assert_allclose(r["y"][:, -1], pop["g_sp"], atol=1e-6)
        np.testing.assert_allclose(r["day_doses"][:, -1, 0], ub_day, rtol=1e-6)
    sc = W.scenario(20, meal_minute=(), bolus=False, basal_scale=0.5)
    r = O.simulate(pop, people, sc, {}, trace_y=True)
    y = r["y"]
    assert np.all(y[:, -1] - pop["g_sp"] > 1.0)                        # the clamp shows
    np.testing.assert_allclose(y[:, -1], y[:, -288], rtol=1e-6)        # and the offset is steady


def test_derivative_action_telescopes():
    # Eq. 3 with only the derivative term (kp = ki = 0): the derivative of the
    # CGM signal, (y_k - y_{k-1}) / Ts with none in the first period, summed over
    # the horizon telescopes, so the basal insulin of a day with meals (and no
    # boluses, noise or zero clipping) is ubh H Ts / 1000 + kd (y_last - y_first) / 1000
    pop = W.population(5, 62, sigma_q1=0.0, cgm_sd=0.0)
    people = O.create_population(pop)
    sc = W.scenario(2, kp_mult=0.0, ki_mult=0.0, bolus=False, meal_mean_g=40.0, meal_sd_g=0.0)
    r = O.simulate(pop, people, sc, {}, trace_y=True)
    y, st = r["y"], r["stats"]
    ub, H, ts = people["u_b"], sc["horizon_periods"], 5.0
    kd = sc["kp_per_ub"] * ub * sc["td_min"]
    assert np.all(np.abs(np.diff(y, axis=1)) < 1.0)          # u = ub (1 + 0.6 dy) never clips at 0
    assert np.abs(y[:, -1] - y[:, 0]).max() > 0.01             # the meals moved the signal
    np.testing.assert_allclose(st["basal_u"], ub * H * ts / 1000.0 + kd * (y[:, -1] - y[:, 0]) / 1000.0,
                               rtol=1e-12)
