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


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)
