"""The parity comparison itself (no GPU): an edge window excuses only what it
should, so the GPU tests that rely on it cannot pass vacuously."""
import numpy as np

from tests._parity import compare_bins, near_edge_samples, near_hypo_edge_samples, rel_err


def _case():
    # three patients, four samples each (mmol/L); edges 3, 3.889, 10, 13.889
    g = np.array([[6.0, 10.0004, 7.0, 8.0],      # one sample 4e-4 above the 180 mg/dL edge
                  [6.0, 6.5, 7.0, 8.0],          # nothing near an edge
                  [3.8885, 3.0, 6.0, 6.0]])      # near 70 mg/dL (5.6e-4 below) and exactly on 54
    ora = np.array([[0, 0, 3, 1, 0], [0, 0, 4, 0, 0], [1, 1, 2, 0, 0]], np.uint32)
    return g, ora


def test_identical_counts_need_no_excuse():
    g, ora = _case()
    excused, bad = compare_bins(ora.copy(), ora, g, 1e-3)
    assert excused == 0 and bad.size == 0


def test_a_count_moved_across_a_nearby_edge_is_excused_elsewhere_not():
    g, ora = _case()
    gpu = ora.copy()
    gpu[0, 3] -= 1
    gpu[0, 2] += 1      # patient 0's near-edge sample binned below 180 mg/dL
    gpu[1, 2] -= 1
    gpu[1, 3] += 1      # patient 1 has no sample near any edge
    excused, bad = compare_bins(gpu, ora, g, 1e-3)
    assert excused == 1 and list(bad) == [1]
    # a window too small for patient 0's sample excuses nothing
    excused, bad = compare_bins(gpu, ora, g, 1e-4)
    assert excused == 0 and list(bad) == [0, 1]


def test_one_near_sample_excuses_one_move_only():
    g, ora = _case()
    gpu = ora.copy()
    gpu[0, 2] -= 2
    gpu[0, 1] += 2      # two counts moved, one near-edge sample to explain them
    assert np.abs(gpu.astype(int) - ora.astype(int)).sum(axis=1)[0] == 4
    _, bad = compare_bins(gpu, ora, g, 1e-3)
    assert list(bad) == [0]


def test_near_edge_counts():
    g, _ = _case()
    np.testing.assert_array_equal(near_edge_samples(g, 1e-3), [1, 0, 2])
    # per-edge windows: the 70 mg/dL edge's window takes patient 2's first sample,
    # and a sample exactly on an edge (3.0) counts even with a zero window
    np.testing.assert_array_equal(near_edge_samples(g, [0.0, 1e-3, 0.0, 0.0]), [0, 0, 2])
    np.testing.assert_array_equal(near_edge_samples(g, [0.0, 0.0, 1e-3, 0.0]), [1, 0, 1])
    np.testing.assert_array_equal(near_hypo_edge_samples(g, 1e-3), [0, 0, 1])
    np.testing.assert_allclose(rel_err([1.0, 0.0], [2.0, 0.0], floor=1e-3), [0.5, 0.0])


def test_per_edge_counts_excuse_only_moves_at_a_near_edge():
    from tests._parity import edge_count_excess
    ora = np.array([[0, 0, 3, 1, 0], [0, 0, 4, 0, 0]], np.uint32)
    near = np.array([[0, 0, 1, 0], [0, 0, 0, 0]])     # patient 0: one sample near 180 mg/dL
    gpu = ora.copy()
    gpu[0, 3] -= 1
    gpu[0, 2] += 1      # moved across 180 mg/dL: excused
    assert edge_count_excess(gpu, ora, near).size == 0
    gpu2 = ora.copy()
    gpu2[0, 2] -= 1
    gpu2[0, 1] += 1     # moved across 70 mg/dL, where patient 0 has no near sample
    assert list(edge_count_excess(gpu2, ora, near)) == [0]
    gpu3 = ora.copy()
    gpu3[0, 2] -= 1
    gpu3[0, 4] += 1     # two edges crossed (180 and 250): only one near sample
    assert list(edge_count_excess(gpu3, ora, near)) == [0]
    gpu4 = ora.copy()
    gpu4[1, 2] -= 1
    gpu4[1, 3] += 1
    assert list(edge_count_excess(gpu4, ora, near)) == [1]


def test_hypo_episode_excuse():
    from tests._parity import hypo_excess
    assert hypo_excess([3, 2, 5], [3, 3, 3], [0, 1, 1]).tolist() == [2]
    assert hypo_excess([3, 2, 5], [3, 3, 3], [0, 1, 2]).size == 0


def test_variance_bound_holds_for_bounded_perturbations():
    """The bound is not loose by orders of magnitude either: a perturbation
    aligned with the deviations reaches half of its perturbation part."""
    from tests._parity import variance_error_bound
    rng = np.random.default_rng(3)
    g = 6.0 + rng.normal(0.0, 1.5, size=(200, 2016))
    eps = 10.0 ** rng.uniform(-6, -3, size=200)
    pert = g + eps[:, None] * rng.uniform(-1.0, 1.0, size=g.shape)
    bound = variance_error_bound(g.var(axis=1), g.mean(axis=1), 6.0, eps)
    assert np.all(np.abs(pert.var(axis=1) - g.var(axis=1)) <= bound)
    aligned = g + eps[:, None] * np.sign(g - g.mean(axis=1, keepdims=True))
    pert_part = variance_error_bound(g.var(axis=1), g.mean(axis=1), 6.0, eps, n_day=0)
    assert np.all(np.abs(aligned.var(axis=1) - g.var(axis=1)) >= 0.5 * pert_part)
