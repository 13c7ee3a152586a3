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
                     first_patient: int = 0) -> dict:
    tir = np.asarray(tir, np.int64)
    ok = np.asarray(status) == 0
    n = int(ok.sum())
    out = {"n_patients": n, "n_flagged": int((~ok).sum()), "horizon_periods": int(horizon)}
    if n == 0:
        out.update(tir_total=np.zeros(5, np.uint64), tir_mean=np.zeros(5),
                   tir_quantile=np.zeros((5, 5)), worst_patient=-1, worst_g_min=0.0,
                   g_mean_mean=0.0, g_mean_var=0.0, basal_u_mean=0.0, bolus_u_mean=0.0)
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
    gm = np.asarray(g_mean)[ok]
    out["g_mean_mean"] = float(gm.mean())
    out["g_mean_var"] = float(gm.var())
    out["basal_u_mean"] = float(np.asarray(basal_u)[ok].mean())
    out["bolus_u_mean"] = float(np.asarray(bolus_u)[ok].mean())
    return out
