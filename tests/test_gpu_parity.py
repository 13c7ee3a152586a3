"""GPU path (through the C-ABI) against the FP64 oracle, element by element.

Tolerances:
  * integer, bit and index work is exact: Philox words, acceptance decisions,
    attempts, statuses, sample counts;
  * FP64 path: glucose trajectories within 1e-12 relative; range counts exact
    except samples whose oracle value lies within 1e-3 mg/dL of an edge;
  * FP32 path: trajectories within 1e-4 relative (floor 1 mmol/L), range
    counts exact except samples within 1e-4 x edge of an edge, population mean
    range fractions within 0.1 percentage point.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import popstats as OP
from paper_2202_13927_gb300 import workloads as W

from tests._parity import (compare_bins, edge_count_excess, hypo_excess, near_hypo_edge_samples,
                           rel_err, variance_error_bound)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vct():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2202_13927_gb300 import vct as V
    V.load()
    return V


def _run(vct, pop_obj, sc, opts, trace=None, trace_kind="bg"):
    n = pop_obj.n
    scs = sc if isinstance(sc, list) else [sc]
    kw = dict(opts)
    tr = None
    if trace:
        total_h = sum(int(s["horizon_periods"]) for s in scs)
        dt = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16}[trace]
        tr = torch.full((total_h, n), float("nan"), dtype=dt, device="cuda")
        kw.update(trace_ptr=tr.data_ptr(), trace_patients=n, trace_dtype=trace, trace_kind=trace_kind)
    buf = vct.simulate(pop_obj, scs, kw)
    vct.sync()
    st = vct.stats_to_numpy(buf)
    g = tr.cpu().numpy().astype(np.float64).T if tr is not None else None
    return st, g


# --------------------------------------------------------------------------- RNG
def test_philox_words_bitwise_and_normals(vct):
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, size=(3000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [7, 123456, 0, 3]
    ctr[3] = [104831, 999999, 255, 2 | (2 << 8)]
    seed = 0xDEADBEEF12345678
    dctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    w, z64 = vct.philox_fill(dctr, seed, "fp64")
    _, z32 = vct.philox_fill(dctr, seed, "fp32")
    w = w.cpu().numpy().view(np.uint32)
    z64, z32 = z64.cpu().numpy(), z32.cpu().numpy().astype(np.float64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(ctr.shape[0]):
        np.testing.assert_array_equal(w[i], O.philox(ctr[i], key))
        zo = O.normals4(ctr[i], key)
        np.testing.assert_allclose(z64[i], zo, rtol=1e-13, atol=1e-14)
        # FP32 Box-Muller: uniforms to 2^-24, __logf/__sincosf to ~2^-21
        np.testing.assert_allclose(z32[i], zo, rtol=2e-5, atol=2e-5)


def _edge_words():
    """Word pairs that probe every branch of the FP64 transform: w0 at and next to
    every power of two (each exponent of the uniform, both ends of its range) and
    at both ends of each of the 4096 reduction intervals of the top exponent, with
    varied angles, and w1 at the start, middle and end of each of the 4096 angle
    intervals with varied radii."""
    w0 = sorted({0, 1, 2, 3, 0xFFFFFFFF, 0xFFFFFFFE, 0xFFFFFFFD} |
                {v for k in range(32) for v in ((1 << k) - 1, 1 << k, (1 << k) + 1)
                 if 0 <= v <= 0xFFFFFFFF} |
                # v = 2 w0 + 1 in [2^32, 2^33): interval j holds w0 in [2^31 + j 2^19, + 2^19)
                {(1 << 31) + j * (1 << 19) + d for j in range(4096) for d in (0, (1 << 19) - 1)})
    w1 = [j * (1 << 20) + d for j in range(4096) for d in (0, 1, (1 << 19) - 1, 1 << 19, (1 << 20) - 1)]
    rng = np.random.default_rng(71)
    a = np.array([(x, int(y)) for x in w0 for y in rng.integers(0, 2 ** 32, size=8)], np.uint64)
    b = np.array([(int(x), y) for y in w1 for x in rng.integers(0, 2 ** 32, size=4)], np.uint64)
    c = np.array([(x, y) for x in w0[::8] for y in w1[::149]], np.uint64)
    return np.concatenate([a, b, c]).astype(np.uint32)


def test_fp64_box_muller_against_the_library_over_the_whole_range(vct):
    """The FP64 form's own Box-Muller transform (table-driven logarithm, Newton
    reciprocal square root, exact angle reduction) against the CUDA library's
    log, sqrt and sincospi on the same words: the branch-probing pairs above
    and 2^22 random pairs, within a few units in the last place of the radius
    (the angle's error is absolute, so the bound scales with the radius)."""
    rng = np.random.default_rng(72)
    edge = _edge_words()
    words = np.concatenate([edge, rng.integers(0, 2 ** 32, size=(1 << 22, 2), dtype=np.uint64).astype(np.uint32)])
    dev = torch.from_numpy(words.view(np.int32)).cuda()
    own = vct.box_muller_words(dev, "own").cpu().numpy()
    lib = vct.box_muller_words(dev, "library").cpu().numpy()
    r = np.hypot(lib[:, 0], lib[:, 1])
    err = np.abs(own - lib).max(axis=1)
    ulps = err / (np.spacing(r))
    assert np.all(np.isfinite(own)), np.nonzero(~np.isfinite(own))
    assert ulps.max() <= 8.0, (ulps.max(), words[np.argmax(ulps)])
    assert np.median(ulps) <= 1.0
    # the radius itself keeps its relative accuracy where it is tiny (u0 near 1)
    ro = np.hypot(own[:, 0], own[:, 1])
    assert np.all(np.abs(ro - r) <= 1e-15 * r + 1e-300), np.max(np.abs(ro - r) / r)
    # the oracle's normals of the branch-probing words (libm log, sqrt, cos, sin)
    ora = np.array([O.box_muller(int(a), int(b)) for a, b in edge])
    re_ = np.hypot(ora[:, 0], ora[:, 1])
    assert np.all(np.abs(own[:len(edge)] - ora).max(axis=1) <= 1e-14 * re_ + 1e-300)
    # and the moments of the 2^23 normals of the random pairs are those of N(0, 1)
    z = own[len(edge):].ravel()
    se = 1.0 / np.sqrt(z.size)
    assert abs(z.mean()) < 5 * se and abs(z.var() - 1.0) < 5 * np.sqrt(2.0) * se


# --------------------------------------------------------------------------- population
def test_population_matches_oracle(vct):
    pop = W.population(1000, 1)
    g = vct.Population.create(pop).export()
    o = O.create_population(pop)
    np.testing.assert_array_equal(g["status"], o["status"].astype(np.uint32) * 2)
    np.testing.assert_array_equal(g["attempts"], o["attempts"])
    np.testing.assert_allclose(g["rows"], o["rows"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(g["u_b"], o["u_b"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(g["x0"], o["x0"], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("case", ["fixed", "wide", "tiny"])
def test_population_draw_cases_match_oracle(vct, case):
    """The population kernel's lanes take patients from a counter and draw one
    Box-Muller pair per loop trip: fixed parameters (sd = 0, no draws), a wide
    distribution (more rejections, extreme basal roots for the closed form),
    and sizes below and just over one block."""
    if case == "fixed":
        pops = [W.with_changes(W.population(37, 31), p_sd=[0.0] * len(W.PARAM_NAMES), bw_sd=0.0)]
    elif case == "wide":
        base = W.population(2000, 32)
        pops = [W.with_changes(base, p_sd=[3.0 * v for v in base["p_sd"]], bw_sd=30.0)]
    else:
        pops = [W.population(n, 33) for n in (1, 3, 129)]
    for pop in pops:
        g = vct.Population.create(pop).export()
        o = O.create_population(pop)
        np.testing.assert_array_equal(g["status"], o["status"].astype(np.uint32) * 2)
        np.testing.assert_array_equal(g["attempts"], o["attempts"])
        # a value mean + sd z is exact up to the rounding of z (the two sides'
        # log and sincospi differ by an ulp or so), i.e. relative to mean + sd:
        # a value near zero (sd z close to -mean) keeps only that absolute accuracy
        scale = np.abs(np.array(list(pop["p_mean"]) + [pop["bw_mean"]])) + \
            np.array(list(pop["p_sd"]) + [pop["bw_sd"]])
        np.testing.assert_array_less(np.abs(g["rows"] - o["rows"]), 4e-15 * scale + 1e-13 * np.abs(o["rows"]))
        # the basal state is a well-conditioned function of the row: it agrees to
        # the row's own relative accuracy
        row_err = np.max(np.abs(g["rows"] - o["rows"]) / np.maximum(np.abs(o["rows"]), 1e-300), axis=1)
        tol = 1e-12 + 20.0 * row_err
        np.testing.assert_array_less(np.abs(g["u_b"] - o["u_b"]), tol * np.abs(o["u_b"]) + 1e-300)
        np.testing.assert_array_less(np.abs(g["x0"] - o["x0"]), tol[:, None] * np.abs(o["x0"]) + 1e-300)
        if case == "fixed":
            assert np.all(g["attempts"] == 1) and np.all(g["rows"] == g["rows"][:1])
        if case == "wide":
            assert g["attempts"].max() > 8  # set-level rejection is exercised


def test_population_shard_is_a_slice_and_rejections_are_flagged(vct):
    pop = W.population(1000, 3)
    full = vct.Population.create(pop).export()
    part = vct.Population.create(W.with_changes(pop, n_patients=333, first_patient=600)).export()
    np.testing.assert_array_equal(full["rows"][600:933], part["rows"])
    np.testing.assert_array_equal(full["u_b"][600:933], part["u_b"])
    bad = vct.Population.create(W.population(50, 4, min_basal_u_per_h=1e3, max_attempts=5))
    assert bad.info().n_rejected == 50
    ex = bad.export()
    assert np.all(ex["status"] == vct.PATIENT_REJECTED) and np.all(ex["attempts"] == 5)
    st, _ = _run(vct, bad, W.scenario(1), {"precision": "fp32"})
    assert np.all(st["status"] == vct.PATIENT_REJECTED) and np.all(st["n_samples"] == 0)


# --------------------------------------------------------------------------- FP64 plain form
@pytest.fixture(scope="module")
def small_fp64(vct):
    pop, sc, _ = W.workload("small")
    gpu_pop = vct.Population.create(pop)
    st, g = _run(vct, gpu_pop, sc, {"precision": "fp64"}, trace="f64")
    people = O.create_population(pop)
    ora = O.simulate(pop, people, sc, {}, trace_g=True)
    return st, g, ora


def test_fp64_trajectories_within_1e12(small_fp64):
    st, g, ora = small_fp64
    assert np.isfinite(g).all()
    err = rel_err(g, ora["g"], floor=1e-6)
    assert err.max() <= 1e-12, err.max()


def test_fp64_indicators_match_oracle(small_fp64):
    st, g, ora = small_fp64
    o = ora["stats"]
    np.testing.assert_array_equal(st["status"], o["status"])
    np.testing.assert_array_equal(st["n_samples"], o["n_samples"])
    excused, bad = compare_bins(st["tir"], o["tir"], ora["g"], 1e-3 / 18.0)
    assert bad.size == 0, (bad[:5], st["tir"][bad[:5]], o["tir"][bad[:5]])
    dh = np.abs(st["hypo_episodes"].astype(int) - o["hypo_episodes"].astype(int))
    assert np.all(dh <= near_hypo_edge_samples(ora["g"], 1e-3 / 18.0))
    near = o["near_edge"][:, 1, :]     # 1e-3 mg/dL, counted by the oracle
    assert edge_count_excess(st["tir"], o["tir"], near).size == 0
    assert hypo_excess(st["hypo_episodes"], o["hypo_episodes"], near[:, 1]).size == 0
    np.testing.assert_array_equal(st["q1_clamps"], o["q1_clamps"])
    np.testing.assert_allclose(st["g_mean"], o["g_mean"], rtol=1e-12)
    np.testing.assert_allclose(st["g_var"], o["g_var"], rtol=1e-9)
    np.testing.assert_allclose(st["g_min"], o["g_min"], rtol=1e-12)
    np.testing.assert_allclose(st["g_max"], o["g_max"], rtol=1e-12)
    np.testing.assert_allclose(st["basal_u"], o["basal_u"], rtol=1e-12)
    np.testing.assert_allclose(st["bolus_u"], o["bolus_u"], rtol=1e-12)
    assert o["tir"][:, [0, 1, 3]].sum() > 0  # the case exercises several ranges


# --------------------------------------------------------------------------- FP32 fast form
@pytest.fixture(scope="module")
def small_fp32(vct):
    pop = W.population(1000, 7)
    sc = W.scenario(7)
    gpu_pop = vct.Population.create(pop)
    st, g = _run(vct, gpu_pop, sc, {"precision": "fp32", "persistent": True}, trace="f32")
    people = O.create_population(pop)
    ora = O.simulate(pop, people, sc, {}, trace_g=True)
    return st, g, ora


def test_fp32_trajectories_within_1e4(small_fp32):
    st, g, ora = small_fp32
    err = rel_err(g, ora["g"], floor=1.0)
    assert err.max() <= 1e-4, err.max()


def test_fp32_indicators_match_oracle(small_fp32):
    st, g, ora = small_fp32
    o = ora["stats"]
    np.testing.assert_array_equal(st["status"], o["status"])
    np.testing.assert_array_equal(st["n_samples"], o["n_samples"])
    edges = np.array([54.0, 70.0, 180.0, 250.0]) / 18.0
    excused, bad = compare_bins(st["tir"], o["tir"], ora["g"], 1e-4 * edges)
    assert bad.size == 0, (bad[:5], st["tir"][bad[:5]], o["tir"][bad[:5]])
    # per edge, and the hypoglycaemia episodes per patient: a difference only
    # where the oracle has samples within 1e-4 x edge of that edge
    near = o["near_edge"][:, 0, :]
    bad = edge_count_excess(st["tir"], o["tir"], near)
    assert bad.size == 0, (bad[:5], st["tir"][bad[:5]], o["tir"][bad[:5]], near[bad[:5]])
    bad = hypo_excess(st["hypo_episodes"], o["hypo_episodes"], near[:, 1])
    assert bad.size == 0, (bad[:5], st["hypo_episodes"][bad[:5]], o["hypo_episodes"][bad[:5]])
    assert o["hypo_episodes"].sum() > 100     # the case has episodes to compare
    mean_frac_gpu = st["tir"].sum(0) / st["n_samples"].sum()
    mean_frac_ora = o["tir"].sum(0) / o["n_samples"].sum()
    assert np.abs(mean_frac_gpu - mean_frac_ora).max() <= 1e-3  # 0.1 percentage point
    np.testing.assert_allclose(st["g_mean"], o["g_mean"], rtol=1e-4)
    # the variance within the FP32 budget given each patient's largest sample error
    eps = np.abs(g - ora["g"]).max(axis=1)
    bound = variance_error_bound(o["g_var"], o["g_mean"], 6.0, eps)
    assert np.all(np.abs(st["g_var"] - o["g_var"]) <= bound), np.max(np.abs(st["g_var"] - o["g_var"]) / bound)
    assert np.median(bound / o["g_var"]) <= 1e-3, np.median(bound / o["g_var"])  # and it is tight
    np.testing.assert_allclose(st["g_min"], o["g_min"], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(st["g_max"], o["g_max"], rtol=1e-4)
    np.testing.assert_allclose(st["basal_u"], o["basal_u"], rtol=1e-4)
    np.testing.assert_allclose(st["bolus_u"], o["bolus_u"], rtol=1e-5)
    np.testing.assert_array_equal(st["q1_clamps"], o["q1_clamps"])


def test_fp32_cgm_trace_in_fp16(vct):
    pop = W.population(300, 8)
    sc = W.scenario(2)
    st, y = _run(vct, vct.Population.create(pop), sc, {"precision": "fp32"}, trace="f16",
                 trace_kind="cgm")
    ora = O.simulate(pop, O.create_population(pop), sc, {}, trace_y=True)
    err = np.abs(y - ora["y"]) / np.maximum(np.abs(ora["y"]), 1.0)
    assert err.max() <= 2.0 ** -11 + 1e-4


def test_traced_lean_kernel_equals_the_full_kernel(vct):
    """A traced run with nothing else takes the lean kernel with only its trace
    branch kept; asking for a BG histogram as well takes the full kernel: the
    records and the FP16 and FP32 traces agree bit for bit, and so do the records
    of the untraced lean run (ragged: 300 patients, two scenarios)."""
    pop = W.population(300, 9)
    gp = vct.Population.create(pop)
    scs = [W.scenario(2), W.scenario(1, kp_mult=0.5)]
    base = {"precision": "fp32", "reg_cap": 128, "block_size": 128, "patients_per_thread": 1,
            "persistent": True}
    plain, _ = _run(vct, gp, scs, base)
    hist = torch.zeros((2, vct.BG_BINS), dtype=torch.int32, device="cuda")
    for dt in ("f16", "f32"):
        lean, yl = _run(vct, gp, scs, base, trace=dt, trace_kind="cgm")
        full, yf = _run(vct, gp, scs, dict(base, bg_hist=hist.data_ptr()), trace=dt, trace_kind="cgm")
        assert lean.tobytes() == full.tobytes() == plain.tobytes(), dt
        assert np.array_equal(yl, yf), dt
        assert np.all(np.isfinite(yl))


# --------------------------------------------------------------------------- invariance
def test_tuning_batching_and_persistence_are_bitwise_invariant(vct):
    pop = W.population(777, 9)
    gp = vct.Population.create(pop)
    scs = [W.scenario(2), W.scenario(3, kp_mult=2.0, meal_mean_g=70.0),
           W.scenario(1, basal_scale=0.5, stream_id=3)]
    ref = [_run(vct, gp, s, {"precision": "fp32"})[0].tobytes() for s in scs]
    for block in (64, 128, 256):
        for ppt in (1, 2):
            for persistent in (False, True):
                st, _ = _run(vct, gp, scs, {"precision": "fp32", "block_size": block,
                                            "patients_per_thread": ppt, "persistent": persistent})
                for j in range(3):
                    assert st[j * 777:(j + 1) * 777].tobytes() == ref[j], (block, ppt, persistent, j)
    # FP64 form: block size does not matter either
    a, _ = _run(vct, gp, scs[0], {"precision": "fp64", "block_size": 64})
    b, _ = _run(vct, gp, scs[0], {"precision": "fp64", "block_size": 256, "persistent": True})
    assert a.tobytes() == b.tobytes()


def test_common_random_numbers_follow_stream_id(vct):
    pop = W.population(200, 10)
    gp = vct.Population.create(pop)
    a, _ = _run(vct, gp, W.scenario(1, stream_id=0), {"precision": "fp32"})
    b, _ = _run(vct, gp, W.scenario(1, stream_id=0, kp_mult=1.0), {"precision": "fp32"})
    c, _ = _run(vct, gp, W.scenario(1, stream_id=1), {"precision": "fp32"})
    assert a.tobytes() == b.tobytes()
    assert not np.array_equal(a["g_mean"], c["g_mean"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_checkpoint_resume_is_bitwise(vct, precision):
    pop = W.population(300, 11)
    gp = vct.Population.create(pop)
    sc = W.scenario(3)
    full, _ = _run(vct, gp, sc, {"precision": precision})
    nbytes = vct.state_bytes(1, 300)
    s1 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    s2 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    out = vct.stats_buffer(1, 300)
    vct.simulate(gp, sc, {"precision": precision, "period_end": 400, "state_out": s1.data_ptr()}, out=out)
    vct.simulate(gp, sc, {"precision": precision, "period_begin": 400, "period_end": 501,
                          "state_in": s1.data_ptr(), "state_out": s2.data_ptr()}, out=out)
    vct.simulate(gp, sc, {"precision": precision, "period_begin": 501, "state_in": s2.data_ptr()},
                 out=out)
    vct.sync()
    assert vct.stats_to_numpy(out).tobytes() == full.tobytes()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_checkpoint_and_resume_calls_are_bitwise(vct, precision):
    """vct_checkpoint / vct_resume: stop at period 400, again at 501 (a
    checkpoint resumed from a checkpoint), finish; and two scenarios of which
    one ends before the checkpoint (its records are written then)."""
    pop = W.population(300, 11)
    gp = vct.Population.create(pop)
    sc = W.scenario(3)
    full, _ = _run(vct, gp, sc, {"precision": precision})
    nbytes = vct.state_bytes(1, 300)
    s1 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    s2 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    vct.checkpoint(gp, sc, 400, s1, {"precision": precision})
    vct.checkpoint(gp, sc, 501, s2, {"precision": precision, "period_begin": 400, "state_in": s1.data_ptr()})
    out = vct.resume(gp, sc, 501, s2, {"precision": precision})
    vct.sync()
    assert vct.stats_to_numpy(out).tobytes() == full.tobytes()
    scs = [W.scenario(1), W.scenario(3, kp_mult=2.0)]
    both, _ = _run(vct, gp, scs, {"precision": precision})
    s3 = torch.zeros(vct.state_bytes(2, 300), dtype=torch.uint8, device="cuda")
    out = vct.stats_buffer(2, 300)
    vct.checkpoint(gp, scs, 300, s3, {"precision": precision}, out=out)
    vct.resume(gp, scs, 300, s3, {"precision": precision}, out=out)
    vct.sync()
    assert vct.stats_to_numpy(out).tobytes() == both.tobytes()
    with pytest.raises(vct.VctError):   # a scenario ends by the checkpoint: its records need out
        vct.checkpoint(gp, scs, 300, s3, {"precision": precision})


def test_caller_workspace_makes_the_same_run(vct):
    """vct_simulate and vct_stats on caller-owned scratch: the same records and
    summaries as with the library's stream-ordered scratch; a workspace that
    is too small is rejected before anything runs."""
    pop = W.population(700, 19)
    gp = vct.Population.create(pop)
    scs = [W.scenario(2), W.protocol_scenario(3, meal_cv=0.1)]
    for kw in ({}, {"steps_per_chunk": 97}):
        ref, _ = _run(vct, gp, scs, dict(kw, precision="fp32"))
        need = vct.simulate_workspace_bytes(gp, scs, dict(kw, precision="fp32"))
        assert need > 0
        ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        got = vct.simulate(gp, scs, dict(kw, precision="fp32", workspace=ws.data_ptr(),
                                         workspace_bytes=need))
        vct.sync()
        assert vct.stats_to_numpy(got).tobytes() == ref.tobytes(), kw
        with pytest.raises(vct.VctError, match="workspace"):
            vct.simulate(gp, scs, dict(kw, precision="fp32", workspace=ws.data_ptr(),
                                       workspace_bytes=need - 1))
    h = [s["horizon_periods"] for s in scs]
    wsb = vct.stats_workspace_bytes(2, 700, h)
    assert wsb == vct.stats_noalloc_bytes(2, 700, h)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    a = vct.population_stats(got, 2, 700, h)
    b = vct.population_stats_with_workspace(got, 2, 700, h, ws)
    for x, y in zip(a, b):
        assert x["worst_patient"] == y["worst_patient"]
        np.testing.assert_array_equal(x["tir_quantile"], y["tir_quantile"])
        assert x["g_mean_mean"] == y["g_mean_mean"] and x["g_mean_var"] == y["g_mean_var"]
    with pytest.raises(vct.VctError, match="workspace"):
        vct.population_stats_with_workspace(got, 2, 700, h, ws[:wsb - 8])


def test_shard_results_equal_the_full_run(vct):
    pop = W.population(1000, 12)
    sc = W.scenario(2)
    full, _ = _run(vct, vct.Population.create(pop), sc, {"precision": "fp32"})
    part, _ = _run(vct, vct.Population.create(W.with_changes(pop, n_patients=250, first_patient=500)),
                   sc, {"precision": "fp32"})
    assert full[500:750].tobytes() == part.tobytes()


# --------------------------------------------------------------------------- edge cases
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_edge_cases_against_oracle(vct, precision):
    pop = W.population(33, 13)
    gp = vct.Population.create(pop)
    people = O.create_population(pop)
    cases = [
        W.scenario(0, horizon_periods=1),
        W.scenario(0, horizon_periods=0),
        W.scenario(1, meal_minute=()),
        W.scenario(1, meal_minute=(0.0, 1435.0)),
        W.scenario(1, meal_minute=(420.0, 420.0, 720.0), meal_sd_g=30.0),  # two meals in one period
        W.scenario(1, bolus=False, kp_mult=0.0, ki_mult=0.0, kd_mult=0.0),
        W.scenario(2, basal_scale=0.5),
    ]
    tol = 1e-11 if precision == "fp64" else 2e-4
    for sc in cases:
        st, _ = _run(vct, gp, sc, {"precision": precision})
        o = O.simulate(pop, people, sc, {})["stats"]
        np.testing.assert_array_equal(st["n_samples"], o["n_samples"])
        np.testing.assert_array_equal(st["status"], o["status"])
        if sc["horizon_periods"] == 0:
            assert np.all(st["tir"] == 0)
            continue
        np.testing.assert_allclose(st["g_mean"], o["g_mean"], rtol=tol)
        np.testing.assert_allclose(st["bolus_u"], o["bolus_u"], rtol=tol, atol=1e-12)
        np.testing.assert_allclose(st["basal_u"], o["basal_u"], rtol=tol)


def test_single_patient_and_substep_count(vct):
    pop = W.population(1, 14)
    gp = vct.Population.create(pop)
    people = O.create_population(pop)
    for m in (1, 3, 10, 12):
        sc = W.scenario(1)
        st, g = _run(vct, gp, sc, {"precision": "fp64", "substeps": m}, trace="f64")
        ora = O.simulate(pop, people, sc, {"substeps": m}, trace_g=True)
        assert rel_err(g, ora["g"], floor=1e-6).max() <= 1e-12, m


def test_noise_free_steady_state(vct):
    pop = W.population(100, 15, sigma_q1=0.0, cgm_sd=0.0)
    gp = vct.Population.create(pop)
    sc = W.scenario(7, meal_minute=())
    st64, g64 = _run(vct, gp, sc, {"precision": "fp64"}, trace="f64")
    assert np.abs(g64 - 6.0).max() <= 1e-12 * 6.0
    assert np.all(st64["tir"][:, 2] == sc["horizon_periods"])
    # FP32: the rounded coefficients have their own fixed point, a few 1e-5 away
    st32, g32 = _run(vct, gp, sc, {"precision": "fp32"}, trace="f32")
    assert np.abs(g32 - 6.0).max() <= 1e-4 * 6.0
    assert np.abs(g32[:, -1] - g32[:, -2]).max() <= 1e-6 * 6.0  # and it stays there


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_controller_identities_on_the_gpu(vct, precision, tol):
    """Eq. 3 on the GPU, checked against properties of the controller rather
    than against the oracle alone: with only the derivative term, the basal
    insulin telescopes to ubh H Ts / 1000 + kd (y_last - y_first) / 1000 over
    the kernel's own CGM trace; with a 20 % wrong basal belief, integral action
    returns the patient to the setpoint."""
    pop = W.population(64, 62, sigma_q1=0.0, cgm_sd=0.0)
    gp = vct.Population.create(pop)
    people = O.create_population(pop)
    ub = people["u_b"]
    sc = W.scenario(2, kp_mult=0.0, ki_mult=0.0, bolus=False, meal_mean_g=40.0, meal_sd_g=0.0)
    st, y = _run(vct, gp, sc, {"precision": precision}, trace="f64", trace_kind="cgm")
    kd = sc["kp_per_ub"] * ub * sc["td_min"]
    assert np.all(np.abs(np.diff(y, axis=1)) < 1.0)
    np.testing.assert_allclose(st["basal_u"], ub * sc["horizon_periods"] * 5.0 / 1000.0
                               + kd * (y[:, -1] - y[:, 0]) / 1000.0, rtol=tol)
    o = O.simulate(pop, people, sc, {})["stats"]
    np.testing.assert_allclose(st["basal_u"], o["basal_u"], rtol=1e-11 if precision == "fp64" else 1e-4)
    sc = W.scenario(20, meal_minute=(), bolus=False, basal_scale=0.8)
    _, y = _run(vct, gp, sc, {"precision": precision}, trace="f64", trace_kind="cgm")
    np.testing.assert_allclose(y[:, -1], pop["g_sp"], atol=1e-6 if precision == "fp64" else 1e-3)


def test_zero_rates_and_sensitivities_from_host(vct):
    """Cohorts given by the caller may hold a zero absorption rate or insulin
    sensitivity (a drawn cohort never does): the kernel's state variables that
    are held divided by such a coefficient keep a floor, so the run must still
    follow the oracle, which integrates the unscaled states."""
    pop = W.population(6, 17)
    people = O.create_population(pop)
    rows = people["rows"].copy()
    names = W.PARAM_NAMES
    rows[1, names.index("ka1")] = 0.0   # x1 frozen at its start value
    rows[2, names.index("SIT")] = 0.0   # x1 never driven
    rows[3, names.index("ka3")] = 0.0
    rows[4, names.index("SIE")] = 0.0
    gp = vct.Population.from_host(pop, rows, people["u_b"], people["x0"])
    people["rows"] = rows
    sc = W.scenario(1)
    o = O.simulate(pop, people, sc, {})["stats"]
    for precision, tol in (("fp64", 1e-11), ("fp32", 1e-4)):
        st, _ = _run(vct, gp, sc, {"precision": precision})
        np.testing.assert_array_equal(st["status"], o["status"])
        np.testing.assert_array_equal(st["n_samples"], o["n_samples"])
        ok = o["status"] == 0
        np.testing.assert_allclose(st["g_mean"][ok], o["g_mean"][ok], rtol=tol)
        np.testing.assert_allclose(st["basal_u"][ok], o["basal_u"][ok], rtol=tol)


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_range_edges_on_the_gpu(vct, precision, rel):
    """Sec. IV-A's range edges (54, 70, 180, 250 mg/dL = 3, 3.9, 10, 13.9 mmol/L
    as printed): patients at rest just below and just above each edge land in
    the ranges on either side, as in the oracle (lower-closed ranges)."""
    names = W.PARAM_NAMES
    base = np.array([W.NOMINAL[k] for k in names] + [80.0])
    base[names.index("VG")] = 0.125                      # V_G BW = 10 L
    gs, expect = [], []
    for j, mg in enumerate((54.0, 70.0, 180.0, 250.0)):
        e = mg / 18.0
        gs += [e * (1 - rel), e * (1 + rel)]
        expect += [j, j + 1]
    rows, ubs, x0s = [], [], []
    for g in gs:
        rc, ub, x0 = O.basal(base, g)
        assert rc == 0
        rows.append(base)
        ubs.append(ub)
        x0s.append(x0)
    pop = W.population(len(gs), 63, sigma_q1=0.0, cgm_sd=0.0)
    people = {"rows": np.array(rows), "u_b": np.array(ubs), "x0": np.array(x0s), "first": 0}
    gp = vct.Population.from_host(pop, people["rows"], people["u_b"], people["x0"])
    sc = W.scenario(0, horizon_periods=1, meal_minute=())
    st, _ = _run(vct, gp, sc, {"precision": precision})
    o = O.simulate(pop, people, sc, {})["stats"]
    np.testing.assert_array_equal(o["tir"].argmax(axis=1), expect)
    np.testing.assert_array_equal(st["tir"], o["tir"])


def test_nonfinite_parameters_are_flagged(vct):
    pop = W.population(8, 16)
    people = O.create_population(pop)
    rows = people["rows"].copy()
    rows[3, 2] = np.nan
    rows[6, 2] = 1e38          # k12: finite, but Q2 overflows within the first day
    gp = vct.Population.from_host(pop, rows, people["u_b"], people["x0"])
    people["rows"] = rows
    o = O.simulate(pop, people, W.scenario(1), {})["stats"]
    assert o["status"][6] == 1 and 0 < o["n_samples"][6] < 288   # dies during the run
    for precision in ("fp32", "fp64"):
        st, _ = _run(vct, gp, W.scenario(1), {"precision": precision})
        np.testing.assert_array_equal(st["status"], o["status"])
        np.testing.assert_array_equal(st["n_samples"], o["n_samples"])
        assert st["status"][3] == vct.PATIENT_NONFINITE
        if precision == "fp32":
            # the packed two-patient form: a lane that dies leaves its partner's
            # sums untouched, bit for bit the one-patient records
            for reg in (192, 168):
                pk, _ = _run(vct, gp, W.scenario(1), {"precision": "fp32", "patients_per_thread": 2,
                                                      "reg_cap": reg, "block_size": 64})
                assert pk.tobytes() == st.tobytes(), reg


def test_patients_turning_nonfinite_mid_run_give_the_same_records_in_every_variant(vct):
    """Patients whose FP32 state overflows at different periods of a three-day
    run (k12 beyond the Euler step's stability limit, so Q2 grows by
    |1 - h k12| per step) and one with a NaN parameter: the lean and full
    kernels, the packed kernel (per lane, dead and live patients in one
    thread), chunked runs (the state through the blob) and the natural
    register allocation write the same records, bit for bit."""
    pop = W.population(200, 23)
    people = O.create_population(pop)
    rows = people["rows"].copy()
    # in the FP64 oracle these overflow FP32's range near periods 611, 52, 175,
    # 185 and 252 (k12 just above the stability limit of the Q1-Q2 exchange)
    k12 = {3: 3.91, 67: 3.99, 10: 3.93, 140: 3.96, 75: 3.93, 199: 1e38, 5: np.nan}
    for i, v in k12.items():
        rows[i, 2] = v
    gp = vct.Population.from_host(pop, rows, people["u_b"], people["x0"])
    sc = [W.scenario(3), W.scenario(2, kp_mult=0.5)]
    base = {"precision": "fp32", "persistent": True}
    ref, _ = _run(vct, gp, sc, dict(base, reg_cap=128, block_size=64, patients_per_thread=1))
    H = 3 * W.PERIODS_PER_DAY
    st0 = ref[:200]
    died = set(np.flatnonzero((st0["status"] & vct.PATIENT_NONFINITE) != 0).tolist())
    assert len(died & set(k12)) >= 5 and died <= set(k12), (died, st0["n_samples"][list(k12)])
    mid = [i for i in died if 0 < st0["n_samples"][i] < H]
    assert len(set(st0["n_samples"][mid].tolist())) >= 4, st0["n_samples"][list(k12)]
    assert st0["n_samples"][5] == 0
    hist = torch.zeros((2, vct.BG_BINS), dtype=torch.int32, device="cuda")
    variants = [dict(reg_cap=112, block_size=128, patients_per_thread=1),
                dict(reg_cap=128, block_size=64, patients_per_thread=1, bg_hist=hist.data_ptr()),
                dict(reg_cap=128, block_size=64, patients_per_thread=1, steps_per_chunk=97),
                dict(reg_cap=128, block_size=64, patients_per_thread=1, steps_per_chunk=288),
                dict(reg_cap=192, block_size=64, patients_per_thread=2),
                dict(reg_cap=168, block_size=64, patients_per_thread=2),
                dict(reg_cap=192, block_size=64, patients_per_thread=2, steps_per_chunk=97),
                dict(reg_cap=0, block_size=64, patients_per_thread=1)]
    for v in variants:
        st, _ = _run(vct, gp, sc, dict(base, **v))
        assert st.tobytes() == ref.tobytes(), (v, np.flatnonzero(
            (np.frombuffer(st.tobytes(), np.uint8).reshape(len(st), -1)
             != np.frombuffer(ref.tobytes(), np.uint8).reshape(len(ref), -1)).any(1))[:10])


# --------------------------------------------------------------------------- launch shapes, chunks, plans
def test_register_caps_and_chunks_are_bitwise_invariant(vct):
    pop = W.population(1000, 21)
    gp = vct.Population.create(pop)
    scs = [W.scenario(2), W.scenario(1, kp_mult=0.5)]
    ref, _ = _run(vct, gp, scs, {"precision": "fp32"})
    for ppt, reg in ((1, 128), (1, 112), (1, 96), (1, 80), (2, 192), (2, 168), (2, 128)):
        for block in (64, 128):
            st, _ = _run(vct, gp, scs, {"precision": "fp32", "reg_cap": reg, "block_size": block,
                                        "patients_per_thread": ppt, "persistent": True})
            assert st.tobytes() == ref.tobytes(), (ppt, reg, block)
    for chunk in (1, 97, 288, 400):
        st, _ = _run(vct, gp, scs, {"precision": "fp32", "steps_per_chunk": chunk, "persistent": True})
        assert st.tobytes() == ref.tobytes(), chunk
    # the packed two-patient form across chunks (state through the blob) and in
    # a plain launch
    for chunk in (0, 97, 288):
        st, _ = _run(vct, gp, scs, {"precision": "fp32", "steps_per_chunk": chunk, "persistent": True,
                                    "patients_per_thread": 2, "reg_cap": 192, "block_size": 64})
        assert st.tobytes() == ref.tobytes(), ("packed", chunk)
    # a run with no trace, BG histogram or protocol takes the lean kernel; asking
    # for a histogram takes the full one: the records agree bit for bit
    hist = torch.zeros((2, vct.BG_BINS), dtype=torch.int32, device="cuda")
    for reg in (128, 112, 96, 80):
        for extra in ({}, {"bg_hist": hist.data_ptr()}):
            st, _ = _run(vct, gp, scs, dict(extra, precision="fp32", reg_cap=reg, block_size=128,
                                            patients_per_thread=1, persistent=True))
            assert st.tobytes() == ref.tobytes(), (reg, extra)
    st64, _ = _run(vct, gp, scs, {"precision": "fp64"})
    st64c, _ = _run(vct, gp, scs, {"precision": "fp64", "steps_per_chunk": 150})
    assert st64.tobytes() == st64c.tobytes()


def test_autotune_and_graph_plan(vct):
    pop = W.population(5000, 22)
    gp = vct.Population.create(pop)
    scs = [W.scenario(2), W.scenario(3, basal_scale=0.5)]
    ref, _ = _run(vct, gp, scs, {"precision": "fp32"})
    best, ms = vct.autotune(gp, scs, {"precision": "fp32", "persistent": True, "steps_per_chunk": -1})
    assert best["block_size"] in (64, 128, 256) and best["patients_per_thread"] in (1, 2)
    assert best["reg_cap"] in (0, 144, 128, 112, 96, 80, 168) and ms > 0 and best["steps_per_chunk"] >= 288
    plan = vct.Plan(gp, scs, {"precision": "fp32", "persistent": True})   # autotunes itself
    assert plan.opts()["block_size"] in (64, 128, 256)
    for _ in range(2):
        plan.out.zero_()
        plan.launch()
        vct.sync()
        assert vct.stats_to_numpy(plan.out).tobytes() == ref.tobytes()
    chunked = vct.Plan(gp, scs, dict(best, persistent=True, steps_per_chunk=200))
    chunked.launch()
    vct.sync()
    assert vct.stats_to_numpy(chunked.out).tobytes() == ref.tobytes()
    plan.close()
    chunked.close()


def test_redraw_feeds_an_existing_plan(vct):
    pop = W.population(700, 23)
    gp = vct.Population.create(pop)
    sc = W.scenario(1)
    plan = vct.Plan(gp, sc, {"precision": "fp32", "persistent": True, "block_size": 128})
    gp.redraw(99)
    plan.launch()
    vct.sync()
    fresh = vct.Population.create(W.with_changes(pop, seed=99))
    np.testing.assert_array_equal(gp.export()["rows"], fresh.export()["rows"])
    assert gp.info().n_rejected == 0
    one, _ = _run(vct, fresh, sc, {"precision": "fp32"})
    assert vct.stats_to_numpy(plan.out).tobytes() == one.tobytes()
    plan.close()


def test_redraw_rekeys_every_chunk_of_a_plan(vct):
    """A chunked plan (several captured kernel launches) follows each redraw:
    every chunk runs on the new seed, and drawing the first seed again gives
    back the first result bit for bit."""
    pop = W.population(500, 24)
    gp = vct.Population.create(pop)
    sc = W.scenario(3)
    plan = vct.Plan(gp, sc, {"precision": "fp32", "persistent": True, "block_size": 64,
                             "steps_per_chunk": W.PERIODS_PER_DAY})
    plan.launch()
    vct.sync()
    first = vct.stats_to_numpy(plan.out).copy()
    gp.redraw(7)
    plan.launch()
    vct.sync()
    second = vct.stats_to_numpy(plan.out).copy()
    one, _ = _run(vct, vct.Population.create(W.with_changes(pop, seed=7)), sc, {"precision": "fp32"})
    assert second.tobytes() == one.tobytes()
    assert second.tobytes() != first.tobytes()
    gp.redraw(pop["seed"])
    plan.launch()
    vct.sync()
    assert vct.stats_to_numpy(plan.out).tobytes() == first.tobytes()
    plan.close()


def test_batched_uneven_horizons_one_persistent_launch(vct):
    """Many scenarios of uneven horizon in one persistent graph-captured launch
    equal the scenarios run one by one, and agree with the oracle: twelve
    scenarios of 1-7 days (five patients each against the oracle) and one of
    52 weeks (eight patients spread over the cohort against the oracle, per
    statistic)."""
    pop, scs = W.batched_uneven(n_scen=13, n_patients=300, seed=4, max_weeks=1)
    for j, sc in enumerate(scs):   # horizons of 1..7 days, independent noise per scenario
        sc["horizon_periods"] = (1 + j % 7) * W.PERIODS_PER_DAY
        sc["stream_id"] = j
    scs[-1]["horizon_periods"] = 364 * W.PERIODS_PER_DAY
    gp = vct.Population.create(pop)
    plan = vct.Plan(gp, scs, {"precision": "fp32", "persistent": True, "block_size": 64})
    plan.launch()
    vct.sync()
    batched = vct.stats_to_numpy(plan.out)
    n = pop["n_patients"]
    people = O.create_population(pop, n=5)
    for j, sc in enumerate(scs[:-1]):
        one, _ = _run(vct, gp, sc, {"precision": "fp32"})
        assert batched[j * n:(j + 1) * n].tobytes() == one.tobytes(), j
        o = O.simulate(pop, people, sc, {})["stats"]
        g = batched[j * n:j * n + 5]
        np.testing.assert_array_equal(g["n_samples"], o["n_samples"])
        np.testing.assert_allclose(g["g_mean"], o["g_mean"], rtol=1e-4)
        np.testing.assert_allclose(g["bolus_u"], o["bolus_u"], rtol=1e-5)
    # the 52-week scenario
    j = len(scs) - 1
    one, _ = _run(vct, gp, scs[j], {"precision": "fp32"})
    assert batched[j * n:(j + 1) * n].tobytes() == one.tobytes()
    ids = np.array([0, 1, 63, 64, 150, 222, 298, 299])
    o = np.concatenate([O.simulate(pop, O.create_population(pop, n=1, first=int(i)), scs[j], {})["stats"]
                        for i in ids])
    g = batched[j * n + ids]
    np.testing.assert_array_equal(g["status"], o["status"])
    np.testing.assert_array_equal(g["n_samples"], o["n_samples"])
    assert np.all(o["n_samples"] == 364 * W.PERIODS_PER_DAY)
    frac_g = g["tir"] / g["n_samples"][:, None]
    frac_o = o["tir"] / o["n_samples"][:, None]
    assert np.abs(frac_g - frac_o).max() <= 1e-3          # 0.1 pp per patient
    np.testing.assert_allclose(g["g_mean"], o["g_mean"], rtol=1e-4)
    np.testing.assert_allclose(g["g_var"], o["g_var"], rtol=1e-3)
    np.testing.assert_allclose(g["g_min"], o["g_min"], rtol=1e-3, atol=1e-3)
    np.testing.assert_allclose(g["g_max"], o["g_max"], rtol=1e-4)
    np.testing.assert_allclose(g["basal_u"], o["basal_u"], rtol=1e-4)
    np.testing.assert_allclose(g["bolus_u"], o["bolus_u"], rtol=1e-5)
    # over the whole year, every range-count and episode difference still lies
    # at samples the oracle has within 1e-4 x edge of an edge
    near = o["near_edge"][:, 0, :]
    assert edge_count_excess(g["tir"], o["tir"], near).size == 0
    assert hypo_excess(g["hypo_episodes"], o["hypo_episodes"], near[:, 1]).size == 0
    summ = vct.population_stats(plan.out, len(scs), n, [s["horizon_periods"] for s in scs])
    assert [s["horizon_periods"] for s in summ] == [s["horizon_periods"] for s in scs]
    plan.close()


# --------------------------------------------------------------------------- population reductions
def _to_device_stats(vct, o_stats):
    """Oracle per-patient indicators in the library's vct_patient_stats layout."""
    n = o_stats.shape[0]
    a = np.zeros(n, vct.PATIENT_STATS_DTYPE)
    for f in ("tir", "hypo_episodes", "q1_clamps", "status", "n_samples", "g_mean", "g_var",
              "g_min", "g_max", "basal_u", "bolus_u", "glucagon_ug"):
        a[f] = o_stats[f]
    return torch.from_numpy(a.view(np.uint8).copy()).cuda()


def _check_popstats(got, exp):
    assert got["n_patients"] == exp["n_patients"] and got["n_flagged"] == exp["n_flagged"]
    np.testing.assert_array_equal(got["below_min"], exp["below_min"])
    np.testing.assert_array_equal(got["below_max"], exp["below_max"])
    np.testing.assert_array_equal(got["tir_total"], exp["tir_total"])
    np.testing.assert_allclose(got["tir_mean"], exp["tir_mean"], rtol=1e-15)
    np.testing.assert_array_equal(got["tir_quantile"], exp["tir_quantile"])
    assert got["worst_patient"] == exp["worst_patient"]
    assert got["worst_g_min"] == exp["worst_g_min"]
    for k in ("g_mean_mean", "basal_u_mean", "bolus_u_mean", "glucagon_ug_mean"):
        assert got[k] == pytest.approx(exp[k], rel=1e-14)
    assert got["g_mean_var"] == pytest.approx(exp["g_mean_var"], rel=1e-10, abs=1e-15)


def test_population_reductions_match_numpy_oracle(vct):
    pop = W.population(1500, 17)
    sc = W.scenario(2)
    people = O.create_population(pop)
    o = O.simulate(pop, people, sc, {})["stats"]
    o["status"][[5, 77]] = 1          # flagged patients are left out
    o["g_min"][[10, 11]] = o["g_min"].min() - 1.0   # a tie: the lower id wins
    dev = _to_device_stats(vct, o)
    got = vct.population_stats(dev, 1, 1500, [sc["horizon_periods"]], first_patient=1000)[0]
    exp = OP.population_stats(o["tir"], o["status"], o["g_mean"], o["g_min"], o["basal_u"],
                              o["bolus_u"], sc["horizon_periods"], first_patient=1000,
                              glucagon_ug=o["glucagon_ug"])
    _check_popstats(got, exp)
    assert got["worst_patient"] == 1010


def test_population_reductions_synthetic_multi_scenario(vct):
    rng = np.random.default_rng(18)
    S, n = 3, 4099
    horizons = [1, 17, 300]
    arrs = []
    for s in range(S):
        a = np.zeros(n, vct.PATIENT_STATS_DTYPE)
        H = horizons[s]
        cuts = np.sort(rng.integers(0, H + 1, size=(n, 4)), axis=1)
        a["tir"] = np.diff(np.concatenate([np.zeros((n, 1), int), cuts, np.full((n, 1), H)], axis=1), axis=1)
        a["n_samples"] = H
        a["g_mean"] = rng.normal(7, 1, n)
        a["g_min"] = np.round(rng.uniform(2, 5, n), 1)  # many ties
        a["basal_u"] = rng.uniform(5, 30, n)
        a["bolus_u"] = rng.uniform(0, 20, n)
        a["glucagon_ug"] = rng.uniform(0, 500, n) * (rng.uniform(size=n) < 0.3)
        a["status"] = (rng.uniform(size=n) < 0.01).astype(np.uint32)
        arrs.append(a)
    dev = torch.from_numpy(np.concatenate(arrs).view(np.uint8).copy()).cuda()
    got = vct.population_stats(dev, S, n, horizons)
    for s in range(S):
        a = arrs[s]
        exp = OP.population_stats(a["tir"], a["status"], a["g_mean"], a["g_min"], a["basal_u"],
                                  a["bolus_u"], horizons[s], glucagon_ug=a["glucagon_ug"])
        _check_popstats(got[s], exp)


# --------------------------------------------------------------------------- year protocol
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_year_protocol_against_oracle(vct, precision):
    pop = W.population(200, 92)
    gp = vct.Population.create(pop)
    people = O.create_population(pop)
    sc = W.protocol_scenario(10, meal_cv=0.1)          # standard and active days, snacks
    short = W.scenario(5, meal_minute=())              # a two-day protocol, cycled
    short["day_plans"] = [{"minute": [0.0, 435.0, 1435.0], "g_per_kg": [0.29, 1.29, 0.57]},
                          {"minute": [], "g_per_kg": []}]
    short["meal_cv"] = 0.3
    for s in (sc, short):
        st, g = _run(vct, gp, s, {"precision": precision}, trace="f64" if precision == "fp64" else "f32")
        ora = O.simulate(pop, people, s, {}, trace_g=True)
        o = ora["stats"]
        err = rel_err(g, ora["g"], floor=1e-6 if precision == "fp64" else 1.0)
        assert err.max() <= (1e-12 if precision == "fp64" else 1e-4), err.max()
        np.testing.assert_allclose(st["bolus_u"], o["bolus_u"], rtol=1e-12 if precision == "fp64" else 1e-5)
        np.testing.assert_array_equal(st["n_samples"], o["n_samples"])
    one, _ = _run(vct, gp, sc, {"precision": precision})
    chunked, _ = _run(vct, gp, sc, {"precision": precision, "steps_per_chunk": 200})
    assert one.tobytes() == chunked.tobytes()


# --------------------------------------------------------------------------- BG curves (Fig. 3)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bg_histogram_matches_oracle(vct, precision):
    pop = W.population(500, 81)
    sc = W.scenario(2)
    gp = vct.Population.create(pop)
    hist = torch.zeros((2, vct.BG_BINS), dtype=torch.int32, device="cuda")
    vct.simulate(gp, [sc, W.scenario(1, basal_scale=0.5)],
                 {"precision": precision, "bg_hist": hist.data_ptr(), "persistent": True,
                  "block_size": 64})
    vct.sync()
    h = hist.cpu().numpy().view(np.uint32).astype(np.int64)
    ora = O.simulate(pop, O.create_population(pop), sc, {}, trace_g=True)
    ho = OP.bg_histogram(ora["g"], ora["stats"]["n_samples"])
    assert h[0].sum() == ho.sum() == 500 * sc["horizon_periods"]
    assert h[1].sum() == 500 * 288
    # a sample may change bins only when the oracle's 10 G lies near an integer
    x = ora["g"].ravel() * 10.0
    window = 1e-9 if precision == "fp64" else 1e-4 * np.maximum(x, 1.0)
    near = int((np.abs(x - np.round(x)) <= window).sum())
    assert np.abs(h[0] - ho).sum() <= 2 * near, (np.abs(h[0] - ho).sum(), near)
    # Fig. 3's mean curve in the library: the oracle's running share of the
    # same histogram exactly, and of the oracle's own samples up to the
    # near-integer ones
    cdf = vct.bg_cdf(hist, 2)
    assert cdf.shape == (2, vct.BG_BINS)
    np.testing.assert_array_equal(cdf, OP.cdf_of_histogram(h))
    assert cdf[0, -1] == 1.0 and np.all(np.diff(cdf[0]) >= 0)
    ref = OP.bg_cdf_from_trace(ora["g"], ora["stats"]["n_samples"])
    assert np.abs(cdf[0] - ref).max() * ho.sum() <= near
    empty = torch.zeros(vct.BG_BINS, dtype=torch.int32, device="cuda")
    assert np.all(vct.bg_cdf(empty, 1) == 0.0)


def test_worst_patient_replay_is_exact(vct):
    pop = W.population(400, 82)
    sc = W.scenario(2)
    gp = vct.Population.create(pop)
    buf = vct.simulate(gp, sc, {"precision": "fp32"})
    vct.sync()
    summ = vct.population_stats(buf, 1, 400, [sc["horizon_periods"]])[0]
    w = summ["worst_patient"]
    row, trace = vct.replay(pop, sc, w, {"precision": "fp32"}, trace_dtype="f32")
    full = vct.stats_to_numpy(buf)[w]
    assert row.tobytes() == full.tobytes()
    assert trace.min() == full["g_min"] == summ["worst_g_min"]
    assert np.sum(trace < 70.0 / 18.0) == full["tir"][0] + full["tir"][1]


# --------------------------------------------------------------------------- full size
def test_four_week_cohort_first_thousand_against_oracle(vct):
    """100,000 patients x 28 days, FP32 persistent: the first 1,000 patients
    re-simulated by the oracle, per statistic and for the population's range
    fractions over those patients."""
    pop, sc, _ = W.workload("fp32_4w")
    gp = vct.Population.create(pop)
    buf = vct.simulate(gp, sc, {"precision": "fp32", "persistent": True})
    vct.sync()
    st = vct.stats_to_numpy(buf)
    people = O.create_population(pop, n=1000, first=0)
    o = O.simulate(pop, people, sc, {})["stats"]
    g = st[:1000]
    assert np.all(g["status"] == o["status"])
    np.testing.assert_array_equal(g["n_samples"], o["n_samples"])
    ok = o["status"] == 0
    frac_g = g["tir"][ok] / g["n_samples"][ok, None]
    frac_o = o["tir"][ok] / o["n_samples"][ok, None]
    assert np.abs(frac_g - frac_o).max() <= 1e-3                     # 0.1 pp per patient
    assert np.abs(frac_g.mean(axis=0) - frac_o.mean(axis=0)).max() <= 1e-4
    np.testing.assert_allclose(g["g_mean"][ok], o["g_mean"][ok], rtol=1e-4)
    np.testing.assert_allclose(g["g_var"][ok], o["g_var"][ok], rtol=1e-3)
    np.testing.assert_allclose(g["basal_u"][ok], o["basal_u"][ok], rtol=1e-4)
    np.testing.assert_allclose(g["bolus_u"][ok], o["bolus_u"][ok], rtol=1e-5, atol=1e-9)
    # range counts and hypoglycaemia episodes differ only at near-edge samples
    near = o["near_edge"][ok][:, 0, :]
    assert edge_count_excess(g["tir"][ok], o["tir"][ok], near).size == 0
    assert hypo_excess(g["hypo_episodes"][ok], o["hypo_episodes"][ok], near[:, 1]).size == 0
    # the whole cohort: every patient sampled in every period, fractions sum to one
    assert np.all(st["tir"].sum(axis=1) == st["n_samples"])


def test_paper_scale_launch_on_sampled_patients(vct):
    """1,000,000 patients x 52 weeks in the FP32 persistent launch the benchmark
    times; 24 patients spread over the population are re-simulated by the
    oracle and compared per statistic."""
    pop, sc, _ = W.workload("paper_scale")
    gp = vct.Population.create(pop)
    buf = vct.simulate(gp, sc, {"precision": "fp32", "persistent": True})
    vct.sync()
    st = vct.stats_to_numpy(buf)
    ids = np.unique(np.concatenate([[0, 1, 127, 128, 999_999], np.linspace(0, 999_999, 19).astype(int)]))
    people = [O.create_population(pop, n=1, first=int(i)) for i in ids]
    assert all(p["status"][0] == 0 for p in people)
    o = np.concatenate([O.simulate(pop, p, sc, {})["stats"] for p in people])
    g = st[ids]
    assert np.all(g["status"] == o["status"])
    np.testing.assert_array_equal(g["n_samples"], o["n_samples"])
    frac_g = g["tir"] / g["n_samples"][:, None]
    frac_o = o["tir"] / o["n_samples"][:, None]
    assert np.abs(frac_g - frac_o).max() <= 1e-3          # 0.1 pp per patient
    np.testing.assert_allclose(g["g_mean"], o["g_mean"], rtol=1e-4)
    np.testing.assert_allclose(g["g_min"], o["g_min"], rtol=1e-3, atol=1e-3)
    np.testing.assert_allclose(g["basal_u"], o["basal_u"], rtol=1e-4)
    np.testing.assert_allclose(g["bolus_u"], o["bolus_u"], rtol=1e-5)
    # over the whole year, range counts and episodes differ only at near-edge samples
    near = o["near_edge"][:, 0, :]
    assert edge_count_excess(g["tir"], o["tir"], near).size == 0
    assert hypo_excess(g["hypo_episodes"], o["hypo_episodes"], near[:, 1]).size == 0
    # properties that hold at any size
    assert np.all(st["n_samples"] == sc["horizon_periods"])
    assert np.all(st["tir"].sum(axis=1) == st["n_samples"])
    assert np.all((st["g_min"] <= st["g_mean"]) & (st["g_mean"] <= st["g_max"]))
