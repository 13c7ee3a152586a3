"""Comparison helpers for GPU-vs-oracle parity tests (test infrastructure)."""
from __future__ import annotations

import numpy as np

EDGES_MMOL = np.array([54.0, 70.0, 180.0, 250.0]) / 18.0


def near_edge_samples(g_trace: np.ndarray, window_mmol) -> np.ndarray:
    """Per patient: samples of the oracle's G(t_k) within `window` of a range edge
    (window may be an array per edge)."""
    w = np.broadcast_to(np.asarray(window_mmol, float), EDGES_MMOL.shape)
    d = np.abs(g_trace[:, :, None] - EDGES_MMOL[None, None, :])
    return (d <= w[None, None, :]).any(axis=2).sum(axis=1)


def near_hypo_edge_samples(g_trace: np.ndarray, window_mmol) -> np.ndarray:
    w = np.broadcast_to(np.asarray(window_mmol, float), EDGES_MMOL.shape)[1]
    return (np.abs(g_trace - EDGES_MMOL[1]) <= w).sum(axis=1)


def compare_bins(gpu_tir, ora_tir, g_trace, window_mmol):
    """Range counts must agree except where an oracle sample lies within the
    window of an edge: each such sample may move one count between adjacent
    ranges.  Returns (excused patients, unexcused patients)."""
    diff = np.abs(gpu_tir.astype(np.int64) - ora_tir.astype(np.int64)).sum(axis=1)
    near = near_edge_samples(g_trace, window_mmol)
    bad = diff > 2 * near
    excused = (diff > 0) & ~bad
    return int(excused.sum()), np.nonzero(bad)[0]


def edge_count_excess(gpu_tir, ora_tir, near_edge):
    """Per edge e, the count of samples at or above it (sum of the ranges above
    e) may differ only by samples the oracle has within the window of e
    (near_edge [n][4], from the oracle's records): a sample farther from the
    edge than both sides' error falls on the same side.  Returns the patients
    where some edge's difference exceeds its near-edge count."""
    g = np.cumsum(np.asarray(gpu_tir, np.int64)[:, ::-1], axis=1)[:, ::-1][:, 1:]
    o = np.cumsum(np.asarray(ora_tir, np.int64)[:, ::-1], axis=1)[:, ::-1][:, 1:]
    excess = np.abs(g - o) - np.asarray(near_edge, np.int64)
    return np.nonzero((excess > 0).any(axis=1))[0]


def hypo_excess(gpu_hypo, ora_hypo, near_hypo_edge):
    """Moving one sample across the 70 mg/dL edge changes the number of
    hypoglycaemia episodes (entries below it) by at most one, so the counts may
    differ by at most the oracle's near-edge samples at that edge.  Returns the
    patients where they differ by more."""
    d = np.abs(np.asarray(gpu_hypo, np.int64) - np.asarray(ora_hypo, np.int64))
    return np.nonzero(d > np.asarray(near_hypo_edge, np.int64))[0]


def variance_error_bound(var_ref, mean_ref, g_sp, eps_max, n_day=288):
    """Largest |var_gpu - var_ref| that the FP32 form can show for a patient
    whose binned samples differ from the oracle's by at most eps_max:
    perturbing every sample by at most eps moves the population variance by at
    most 2 sd eps + eps^2 (Cauchy-Schwarz on the covariance of the samples with
    the perturbation), and the FP32 day partials of (G - G_sp) and its square
    (n_day terms each, folded into FP64 once a day) add at most
    3 n_day 2^-24 E[(G - G_sp)^2]."""
    var_ref = np.asarray(var_ref, float)
    eps = np.asarray(eps_max, float)
    second = var_ref + (np.asarray(mean_ref, float) - g_sp) ** 2
    return 2.0 * np.sqrt(var_ref) * eps + eps ** 2 + 3.0 * n_day * 2.0 ** -24 * second


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)
