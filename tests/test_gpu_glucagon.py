"""Glucagon compartments and the AP's glucagon mode on the GPU (Sec. IV-B:
two-state s.c. glucagon model; Sec. IV-C: glucagon mode, no insulin, glucagon
microboli) against the FP64 oracle.

The mode is a floating-point decision (y_k below the threshold) that switches
the controller, so each side's decision sequence is compared first: periods
where the two sides decide differently must have an oracle CGM value within
the precision's window of the threshold, and patients whose decisions all
agree are held to the usual trajectory tolerances (FP64 1e-12, FP32 1e-4).
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import popstats as OP
from paper_2202_13927_gb300 import workloads as W

from tests._parity import compare_bins, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vct():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2202_13927_gb300 import vct as V
    V.load()
    return V


def _run(vct, gp, scs, opts, trace=None, kind="bg"):
    scs = scs if isinstance(scs, list) else [scs]
    kw = dict(opts)
    tr = None
    if trace:
        total = sum(int(s["horizon_periods"]) for s in scs)
        dt = {"f64": torch.float64, "f32": torch.float32}[trace]
        tr = torch.full((total, gp.n), float("nan"), dtype=dt, device="cuda")
        kw.update(trace_ptr=tr.data_ptr(), trace_patients=gp.n, trace_dtype=trace, trace_kind=kind)
    buf = vct.simulate(gp, scs, kw)
    vct.sync()
    return vct.stats_to_numpy(buf), (tr.cpu().numpy().astype(np.float64).T if tr is not None else None)


@pytest.fixture(scope="module")
def hypo_case(vct):
    # the controller believes the basal 50 % too high: patients go low and the
    # glucagon mode engages
    pop = W.population(400, 51)
    sc = W.scenario(2, basal_scale=1.5, glucagon=True)
    gp = vct.Population.create(pop)
    people = O.create_population(pop)
    ora = O.simulate(pop, people, sc, {}, trace_g=True, trace_y=True)
    return pop, sc, gp, people, ora


@pytest.mark.parametrize("precision,window,tol", [("fp64", 1e-9, 1e-12), ("fp32", 2e-3, 1e-4)])
def test_glucagon_mode_matches_oracle(vct, hypo_case, precision, window, tol):
    pop, sc, gp, people, ora = hypo_case
    trace = "f64" if precision == "fp64" else "f32"
    st, g = _run(vct, gp, sc, {"precision": precision}, trace=trace)
    _, y = _run(vct, gp, sc, {"precision": precision}, trace=trace, kind="cgm")
    o = ora["stats"]
    thr = sc["gg_threshold"]
    ok = people["status"] == 0
    mode_gpu = y < thr
    mode_ora = ora["y"] < thr
    differ = (mode_gpu != mode_ora) & ok[:, None]
    # every differing decision sits at the threshold (within the precision's window)
    assert np.all(np.abs(ora["y"][differ] - thr) <= window), np.abs(ora["y"][differ] - thr).max()
    same = ok & ~differ.any(axis=1)
    assert same.sum() >= 0.8 * ok.sum()
    assert mode_ora[same].sum() > 100       # the case exercises the glucagon mode
    np.testing.assert_array_equal(st["status"], o["status"])
    floor = 1e-6 if precision == "fp64" else 1.0
    assert rel_err(g[same], ora["g"][same], floor=floor).max() <= tol
    s, t = st[same], o[same]
    edge_win = 1e-3 / 18.0 if precision == "fp64" else 1e-4 * np.array([54.0, 70.0, 180.0, 250.0]) / 18.0
    _, bad = compare_bins(s["tir"], t["tir"], ora["g"][same], edge_win)
    assert bad.size == 0
    np.testing.assert_allclose(s["glucagon_ug"], t["glucagon_ug"], rtol=10 * tol, atol=10 * tol)
    np.testing.assert_allclose(s["basal_u"], t["basal_u"], rtol=10 * tol)
    np.testing.assert_allclose(s["bolus_u"], t["bolus_u"], rtol=10 * tol, atol=1e-12)
    assert t["glucagon_ug"].sum() > 0.0
    # glucagon mode withheld insulin: no bolus in a glucagon period, none of the basal
    assert np.all(st["glucagon_ug"][~ok] == 0.0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_scenarios_without_glucagon_are_bit_identical_in_the_glucagon_variant(vct, precision):
    pop = W.population(600, 52)
    gp = vct.Population.create(pop)
    plain = W.scenario(2, stream_id=3)
    alone, _ = _run(vct, gp, plain, {"precision": precision})
    mixed, _ = _run(vct, gp, [W.scenario(2, basal_scale=1.5, glucagon=True), plain],
                    {"precision": precision})
    n = gp.n
    assert mixed[n:].tobytes() == alone.tobytes()
    assert mixed[:n]["glucagon_ug"].sum() > 0.0


def test_glucagon_checkpoint_resume_is_bitwise(vct):
    pop = W.population(300, 53)
    gp = vct.Population.create(pop)
    sc = W.scenario(3, basal_scale=1.5, glucagon=True)
    full, _ = _run(vct, gp, sc, {"precision": "fp32"})
    nbytes = vct.state_bytes(1, 300)
    s1 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    out = vct.stats_buffer(1, 300)
    vct.simulate(gp, sc, {"precision": "fp32", "period_end": 437, "state_out": s1.data_ptr()}, out=out)
    vct.simulate(gp, sc, {"precision": "fp32", "period_begin": 437, "state_in": s1.data_ptr()}, out=out)
    vct.sync()
    assert vct.stats_to_numpy(out).tobytes() == full.tobytes()
    assert full["glucagon_ug"].sum() > 0.0


def test_glucagon_plan_autotune_and_population_mean(vct):
    pop = W.population(2000, 54)
    gp = vct.Population.create(pop)
    sc = W.scenario(2, basal_scale=1.5, glucagon=True)
    one, _ = _run(vct, gp, sc, {"precision": "fp32", "persistent": True, "block_size": 128,
                                "reg_cap": 128})
    plan = vct.Plan(gp, sc, {"precision": "fp32", "persistent": True})   # library shape
    plan.launch()
    vct.sync()
    assert vct.stats_to_numpy(plan.out).tobytes() == one.tobytes()
    plan.close()
    tuned = vct.Plan(gp, sc, {"precision": "fp32", "persistent": True, "block_size": 0,
                              "steps_per_chunk": -1})
    assert tuned.opts()["patients_per_thread"] == 1 and tuned.opts()["reg_cap"] in (0, 128, 144)
    tuned.launch()
    vct.sync()
    assert vct.stats_to_numpy(tuned.out).tobytes() == one.tobytes()
    tuned.close()
    got = vct.population_stats(plan.out, 1, gp.n, [sc["horizon_periods"]])[0]
    exp = OP.population_stats(one["tir"], one["status"], one["g_mean"], one["g_min"],
                              one["basal_u"], one["bolus_u"], sc["horizon_periods"],
                              glucagon_ug=one["glucagon_ug"])
    assert got["glucagon_ug_mean"] == pytest.approx(exp["glucagon_ug_mean"], rel=1e-14)
    assert got["glucagon_ug_mean"] > 0.0


def test_glucagon_needs_the_compartment_model(vct):
    gp = vct.Population.create(W.with_changes(W.population(10, 55), tau_gg_min=0.0))
    with pytest.raises(vct.VctError):
        vct.simulate(gp, W.scenario(1, glucagon=True), {"precision": "fp32"})
    with pytest.raises(vct.VctError):
        vct.simulate(vct.Population.create(W.population(10, 55)), W.scenario(1, glucagon=True),
                     {"precision": "fp32", "block_size": 64, "patients_per_thread": 2})


def _dose_hist_from_oracle(vct, day_doses, ok):
    """Histograms of the oracle's whole-day doses (finite days of counted patients)."""
    widths = [vct.DOSE_BIN_WIDTHS[k] for k in ("basal_u", "bolus_u", "glucagon_ug")]
    h = np.zeros((3, vct.DOSE_BINS), np.int64)
    near = np.zeros(3, np.int64)
    for j, w in enumerate(widths):
        x = day_doses[ok][:, :, j].ravel()
        x = x[np.isfinite(x)]
        b = np.minimum(np.floor(x / w), vct.DOSE_BINS - 1).astype(np.int64)
        np.add.at(h[j], b, 1)
        q = x / w
        near[j] = int((np.abs(q - np.round(q)) <= 1e-4 * np.maximum(q, 1.0)).sum())
    return h, near


@pytest.mark.parametrize("precision,glucagon", [("fp64", True), ("fp32", False)])
def test_daily_dose_histograms_match_oracle(vct, precision, glucagon):
    # FP64 with the glucagon mode (its decisions agree with the oracle's);
    # FP32 without it, so that only the bin edges can differ
    pop = W.population(500, 56)
    gp = vct.Population.create(pop)
    people = O.create_population(pop)
    sc = W.scenario(3, basal_scale=1.5, glucagon=glucagon)
    ora = O.simulate(pop, people, sc, {}, day_doses=True)
    hist = torch.zeros(3 * vct.DOSE_BINS, dtype=torch.int32, device="cuda")
    st, _ = _run(vct, gp, sc, {"precision": precision, "dose_hist": hist.data_ptr()})
    got = hist.cpu().numpy().astype(np.int64).reshape(3, vct.DOSE_BINS)
    ok = (people["status"] == 0) & (ora["stats"]["status"] == 0)
    exp, near = _dose_hist_from_oracle(vct, ora["day_doses"], ok)
    assert got.sum(axis=1).tolist() == [3 * int(ok.sum())] * 3      # every whole day, once
    for j in range(3):
        assert np.abs(got[j] - exp[j]).sum() <= 2 * near[j], (j, np.nonzero(got[j] - exp[j]))
    if glucagon:
        assert exp[2, 1:].sum() > 0                                  # some days with glucagon
    # Fig. 5's quantiles in the library: on the oracle's own histograms they are
    # the oracle's order statistics exactly; on the kernel's within one bin
    # where a near-edge dose moved
    qs = (0.0, 0.05, 0.25, 0.5, 0.75, 0.95, 1.0)
    widths = [vct.DOSE_BIN_WIDTHS[k] for k in ("basal_u", "bolus_u", "glucagon_ug")]
    dev_exp = torch.from_numpy(exp.astype(np.int32).reshape(-1)).cuda()
    q_exp = vct.dose_quantiles(dev_exp, 1, qs)[0]
    q_got = vct.dose_quantiles(hist, 1, qs)[0]
    for j, w in enumerate(widths):
        x = ora["day_doses"][ok][:, :, j].ravel()
        want = OP.dose_quantiles(x[np.isfinite(x)], w, qs)
        assert list(q_exp[j]) == want, (j, q_exp[j], want)
        assert np.all(np.abs(q_got[j] - want) <= (w if near[j] else 0.0)), (j, q_got[j], want)
    # a chunked run adds the same counts
    hist2 = torch.zeros_like(hist)
    _run(vct, gp, sc, {"precision": precision, "dose_hist": hist2.data_ptr(),
                       "steps_per_chunk": 100})
    assert torch.equal(hist, hist2)
