"""Population summaries of per-patient indicators -- plain numpy.

TEST INFRASTRUCTURE ONLY (same rule as ``oracle.py``).  Follows Sec. IV-D of
the paper: mean time in each of the five BG ranges over the population, the
box plot of the per-patient range fractions, and the worst-case patient
(lowest BG reached, Sec. III-C "stored only if worse ... lowest BG").
Quantiles are numpy's inverted-CDF quantiles; the worst patient is the first
(lowest id) minimiser of g_min.
"""
from __future__ import annotations

import numpy as np

QUANTILES = (0.0, 0.25, 0.5, 0.75, 1.0)


def population_stats(tir, status, g_mean, g_min, basal_u, bolus_u, horizon: int,
                     first_patient: int = 0, glucagon_ug=None) -> dict:
    tir = np.asarray(tir, np.int64)
    ok = np.asarray(status) == 0
    n = int(ok.sum())
    out = {"n_patients": n, "n_flagged": int((~ok).sum()), "horizon_periods": int(horizon)}
    if n == 0:
        out.update(tir_total=np.zeros(5, np.uint64), tir_mean=np.zeros(5),
                   tir_quantile=np.zeros((5, 5)), worst_patient=-1, worst_g_min=0.0,
                   g_mean_mean=0.0, g_mean_var=0.0, basal_u_mean=0.0, bolus_u_mean=0.0,
                   glucagon_ug_mean=0.0, below_min=np.zeros(4, np.uint32), below_max=np.zeros(4, np.uint32))
        return out
    t = tir[ok]
    out["tir_total"] = t.sum(axis=0).astype(np.uint64)
    out["tir_mean"] = t.sum(axis=0) / (n * horizon) if horizon else np.zeros(5)
    frac = t / horizon if horizon else np.zeros_like(t, dtype=float)
    out["tir_quantile"] = np.stack([np.quantile(frac[:, b], QUANTILES, method="inverted_cdf")
                                    for b in range(5)])
    gmin = np.asarray(g_min)[ok]
    ids = np.nonzero(ok)[0]
    j = int(np.argmin(gmin))
    out["worst_patient"] = int(ids[j]) + first_patient
    out["worst_g_min"] = float(gmin[j])
    cum = np.cumsum(t[:, :4], axis=1)          # periods below 54, 70, 180, 250 mg/dL
    out["below_min"] = cum.min(axis=0).astype(np.uint32)
    out["below_max"] = cum.max(axis=0).astype(np.uint32)
    gm = np.asarray(g_mean)[ok]
    out["g_mean_mean"] = float(gm.mean())
    out["g_mean_var"] = float(gm.var())
    out["basal_u_mean"] = float(np.asarray(basal_u)[ok].mean())
    out["bolus_u_mean"] = float(np.asarray(bolus_u)[ok].mean())
    gg = np.zeros(len(ok)) if glucagon_ug is None else np.asarray(glucagon_ug)
    out["glucagon_ug_mean"] = float(gg[ok].mean())
    return out


def bg_histogram(g_trace, n_samples=None, bins: int = 301, width: float = 0.1) -> np.ndarray:
    """Counts of the binned samples G(t_k) per `width` mmol/L bin, bin floor(G/width)
    with everything above the last edge in the last bin (Fig. 3's curves are the
    running sums of this histogram).  Rows of g_trace beyond n_samples[i] (a patient
    that turned non-finite) are ignored."""
    g = np.asarray(g_trace, np.float64)
    if n_samples is not None:
        mask = np.arange(g.shape[1])[None, :] < np.asarray(n_samples)[:, None]
        g = g[mask]
    b = np.minimum(np.floor(g.ravel() * (1.0 / width)).astype(np.int64), bins - 1)
    return np.bincount(b, minlength=bins)


def cdf_of_histogram(hist) -> np.ndarray:
    """Running share of a histogram's counts: entry j is the fraction of the
    samples in bins 0..j (Fig. 3's mean BG curve when the histogram is the
    population's BG histogram); all zero for an empty histogram."""
    h = np.asarray(hist, np.int64)
    c = np.cumsum(h, axis=-1)
    total = c[..., -1:]
    return np.where(total > 0, c / np.maximum(total, 1), 0.0)


def bg_cdf_from_trace(g_trace, n_samples=None, bins: int = 301, width: float = 0.1) -> np.ndarray:
    """Fig. 3's mean BG curve straight from the samples: entry j is the fraction
    of binned samples with floor(G / width) <= j (the last bin open)."""
    g = np.asarray(g_trace, np.float64)
    if n_samples is not None:
        mask = np.arange(g.shape[1])[None, :] < np.asarray(n_samples)[:, None]
        g = g[mask]
    b = np.minimum(np.floor(g.reshape(-1) * (1.0 / width)).astype(np.int64), bins - 1)
    n = b.size
    return np.array([(b <= j).sum() / n if n else 0.0 for j in range(bins)])


def dose_quantiles(doses, width: float, qs, bins: int = 400) -> list:
    """Fig. 5's daily-dose quantiles from the doses themselves: each dose falls
    in bin min(floor(dose / width), bins - 1); quantile q is the upper edge
    (b + 1) width of the bin of the r-th smallest dose, r = max(ceil(q n), 1)
    (inverse-CDF definition); 0 for no doses."""
    d = np.asarray(doses, np.float64).ravel()
    if d.size == 0:
        return [0.0 for _ in qs]
    b = np.sort(np.minimum(np.floor(d * (1.0 / width)), bins - 1))
    out = []
    for q in qs:
        r = max(int(np.ceil(q * d.size)), 1)
        out.append(float((b[r - 1] + 1.0) * width))
    return out
