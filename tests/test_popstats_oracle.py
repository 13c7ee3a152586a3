"""Pins of the oracle of the population reductions (Sec. IV-D: mean time in
each BG range, the box plot of the per-patient fractions, the worst-case
patient; Fig. 3: the span of time below each range edge and the BG histogram
behind the mean curve).

Every expected value here is worked out by hand from the definitions, on
inputs small enough to check by eye: the inverse-CDF quantile is the smallest
sample whose rank reaches q n, the worst patient is the lowest-id minimiser of
the lowest BG among the counted (unflagged) patients, and the span at an edge
is the fewest and the most periods any counted patient spent below it.
"""
import numpy as np

from oracle import popstats as OP


def _four_patients():
    # horizon 10 periods; rows are (<54, 54-70, 70-180, 180-250, >=250) counts
    tir = np.array([[0, 1, 8, 1, 0],
                    [2, 2, 6, 0, 0],
                    [0, 0, 10, 0, 0],
                    [1, 0, 5, 3, 1]])
    status = np.zeros(4, np.int32)
    g_mean = np.array([6.0, 5.0, 7.0, 8.0])
    g_min = np.array([3.5, 2.5, 4.0, 2.9])
    basal = np.array([10.0, 12.0, 14.0, 16.0])
    bolus = np.array([1.0, 2.0, 3.0, 4.0])
    return tir, status, g_mean, g_min, basal, bolus


def test_hand_worked_four_patient_example():
    tir, status, g_mean, g_min, basal, bolus = _four_patients()
    r = OP.population_stats(tir, status, g_mean, g_min, basal, bolus, horizon=10, first_patient=100)
    assert r["n_patients"] == 4 and r["n_flagged"] == 0
    np.testing.assert_array_equal(r["tir_total"], [3, 3, 29, 4, 1])
    np.testing.assert_allclose(r["tir_mean"], [0.075, 0.075, 0.725, 0.1, 0.025])
    # 70-180 fractions 0.8, 0.6, 1.0, 0.5 -> sorted 0.5, 0.6, 0.8, 1.0: the q-quantile
    # is the k-th smallest with k = ceil(4 q) (k = 1 for q = 0)
    np.testing.assert_allclose(r["tir_quantile"][2], [0.5, 0.5, 0.6, 0.8, 1.0])
    # 180-250 fractions 0.1, 0, 0, 0.3 -> sorted 0, 0, 0.1, 0.3
    np.testing.assert_allclose(r["tir_quantile"][3], [0.0, 0.0, 0.0, 0.1, 0.3])
    # the lowest BG is patient 1's 2.5 mmol/L; ids are global
    assert r["worst_patient"] == 101 and r["worst_g_min"] == 2.5
    # periods below 54, 70, 180, 250 mg/dL per patient: (0,1,9,10), (2,4,10,10),
    # (0,0,10,10), (1,1,6,9)
    np.testing.assert_array_equal(r["below_min"], [0, 0, 6, 9])
    np.testing.assert_array_equal(r["below_max"], [2, 4, 10, 10])
    assert r["g_mean_mean"] == 6.5
    # population variance (divisor n): deviations -0.5, -1.5, 0.5, 1.5 -> 5 / 4
    assert abs(r["g_mean_var"] - 1.25) < 1e-15
    assert r["basal_u_mean"] == 13.0 and r["bolus_u_mean"] == 2.5 and r["glucagon_ug_mean"] == 0.0


def test_flagged_patients_are_left_out_and_ties_go_to_the_lowest_id():
    tir, status, g_mean, g_min, basal, bolus = _four_patients()
    status = np.array([0, 1, 0, 0], np.int32)  # patient 1 (the lowest BG) is flagged
    g_min = g_min.copy()
    g_min[3] = 3.5                              # now patients 0 and 3 tie at 3.5
    r = OP.population_stats(tir, status, g_mean, g_min, basal, bolus, horizon=10)
    assert r["n_patients"] == 3 and r["n_flagged"] == 1
    assert r["worst_patient"] == 0 and r["worst_g_min"] == 3.5
    np.testing.assert_array_equal(r["tir_total"], [1, 1, 23, 4, 1])
    # 70-180 fractions of the counted patients 0.8, 1.0, 0.5 -> sorted 0.5, 0.8, 1.0;
    # k = ceil(3 q): q = 0.25 -> 1, 0.5 -> 2, 0.75 -> 3
    np.testing.assert_allclose(r["tir_quantile"][2], [0.5, 0.5, 0.8, 1.0, 1.0])
    assert r["basal_u_mean"] == (10.0 + 14.0 + 16.0) / 3
    # a flagged patient ahead of the worst one: the id stays the patient's own
    r = OP.population_stats(tir, np.array([1, 0, 0, 0]), g_mean, np.array([2.0, 3.0, 4.0, 2.9]),
                            basal, bolus, horizon=10, first_patient=7)
    assert r["worst_patient"] == 10 and r["worst_g_min"] == 2.9


def test_identical_patients_and_the_all_flagged_case():
    tir = np.tile([[1, 2, 3, 4, 0]], (5, 1))
    r = OP.population_stats(tir, np.zeros(5), np.full(5, 7.0), np.full(5, 3.0), np.ones(5),
                            np.ones(5), horizon=10, glucagon_ug=np.full(5, 20.0))
    np.testing.assert_allclose(r["tir_quantile"], np.tile([[0.1], [0.2], [0.3], [0.4], [0.0]], (1, 5)))
    assert r["g_mean_var"] == 0.0 and r["worst_patient"] == 0 and r["glucagon_ug_mean"] == 20.0
    np.testing.assert_array_equal(r["below_min"], r["below_max"])
    none = OP.population_stats(tir, np.ones(5), np.zeros(5), np.zeros(5), np.zeros(5), np.zeros(5), 10)
    assert none["n_patients"] == 0 and none["n_flagged"] == 5 and none["worst_patient"] == -1


def test_bg_histogram_bins_by_hand():
    # floor(G / 0.1): 2.95 -> 29, 3.0 -> 30 (lower-closed), 10.04 -> 100, 31 -> last bin 300;
    # the second patient's rows after its two samples are ignored
    g = np.array([[2.95, 3.0, 10.04, 31.0], [3.0, 5.55, 99.0, 99.0]])
    h = OP.bg_histogram(g, n_samples=[4, 2])
    expect = np.zeros(301, np.int64)
    for b in (29, 30, 100, 300, 30, 55):
        expect[b] += 1
    np.testing.assert_array_equal(h, expect)


def test_cdf_of_a_histogram_by_hand():
    np.testing.assert_array_equal(OP.cdf_of_histogram([0, 2, 0, 1, 1]), [0.0, 0.5, 0.5, 0.75, 1.0])
    np.testing.assert_array_equal(OP.cdf_of_histogram([0, 0, 0]), [0.0, 0.0, 0.0])
    np.testing.assert_array_equal(OP.cdf_of_histogram([[1, 3], [2, 0]]), [[0.25, 1.0], [1.0, 1.0]])


def test_bg_cdf_from_samples_by_hand():
    # samples 0.05 (bin 0), 0.25 (bin 2), 0.25, 31.0 (open last bin): 4 samples
    g = np.array([[0.05, 0.25], [0.25, 31.0]])
    c = OP.bg_cdf_from_trace(g)
    assert c.shape == (301,)
    np.testing.assert_array_equal(c[:4], [0.25, 0.25, 0.75, 0.75])
    assert c[299] == 0.75 and c[300] == 1.0
    # a patient's samples after it turned non-finite are left out
    c = OP.bg_cdf_from_trace(g, n_samples=[2, 1])
    np.testing.assert_array_equal(c[:3], [1 / 3, 1 / 3, 1.0])


def test_dose_quantiles_by_hand():
    # doses 0.1, 0.3, 0.3, 2.0 U in 0.25 U bins: bins 0, 1, 1, 8
    d = [0.1, 0.3, 0.3, 2.0]
    # q = 0 -> rank 1 (bin 0, upper edge 0.25); 0.3 -> rank ceil(1.2) = 2 (bin 1, 0.5);
    # 0.5 -> rank 2 (bin 1, 0.5); 0.8 -> rank ceil(3.2) = 4 (bin 8, 2.25); 1 -> rank 4
    assert OP.dose_quantiles(d, 0.25, (0.0, 0.3, 0.5, 0.8, 1.0)) == [0.25, 0.5, 0.5, 2.25, 2.25]
    assert OP.dose_quantiles([], 0.25, (0.5,)) == [0.0]
    # a dose beyond the last bin lands in the open last bin: its upper edge is 400 w
    assert OP.dose_quantiles([1e6], 5.0, (1.0,)) == [2000.0]
