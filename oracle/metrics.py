"""Dose and clinical plan metrics (Sec. 2.A definitions, Sec. 3.B conventions).

Test infrastructure (see oracle/__init__.py).

  dose d = Phi_eval t                     (Sec. 4: sum of dose-rate kernels
                                           weighted by the sector times)
  coverage    = |target AND d >= D| / |target|
  selectivity = |target AND d >= D| / |d >= D|
  GI          = |d >= D/2| / |d >= D|     (only when all prescriptions are equal)
  BOT         = sum over isocenters of the longest sector time
                (sum over the collimators of that sector), in minutes
Multi-target coverage and selectivity use each target's own prescription
(Sec. 3.B); the prescription isodose volume for selectivity is the union over
targets of {d >= D_k}.
"""
from __future__ import annotations

import numpy as np


def dose(phi_eval, t):
    """(E, B) x (B, K) -> (E, K) doses, FP64."""
    return np.asarray(phi_eval, dtype=np.float64) @ np.asarray(t, dtype=np.float64)


def beam_on_time(t, n_iso, n_sectors=8, n_coll=3):
    """Sec. 3.B: per isocenter the longest sector (its collimator times summed),
    summed over isocenters.  t (B, K) -> (K,)."""
    t = np.asarray(t, dtype=np.float64)
    K = t.shape[1]
    per_sector = t.reshape(n_iso, n_sectors, n_coll, K).sum(axis=2)
    return per_sector.max(axis=1).sum(axis=0)


def plan_metrics(d, label, d_presc, t, n_iso, n_sectors=8, n_coll=3):
    """Coverage, selectivity, GI (nan if prescriptions differ) and BOT per
    column.  d (E, K); label (E,) target index or -1; d_presc (n_targets,)."""
    d = np.asarray(d, dtype=np.float64)
    label = np.asarray(label)
    d_presc = np.atleast_1d(np.asarray(d_presc, dtype=np.float64))
    K = d.shape[1]
    cov = np.zeros(K)
    sel = np.zeros(K)
    gi = np.full(K, np.nan)
    inT = label >= 0
    D_vox = np.where(inT, d_presc[np.maximum(label, 0)], np.nan)
    for j in range(K):
        covered = inT & (d[:, j] >= D_vox)
        piv = np.zeros(d.shape[0], dtype=bool)
        for D in np.unique(d_presc):
            piv |= d[:, j] >= D
        cov[j] = covered.sum() / max(inT.sum(), 1)
        sel[j] = covered.sum() / max(piv.sum(), 1)
        if np.all(d_presc == d_presc[0]):
            D = d_presc[0]
            gi[j] = (d[:, j] >= 0.5 * D).sum() / max((d[:, j] >= D).sum(), 1)
    bot = beam_on_time(t, n_iso, n_sectors, n_coll)
    return dict(coverage=cov, selectivity=sel, gi=gi, bot=bot)
