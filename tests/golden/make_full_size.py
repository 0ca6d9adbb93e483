"""Write the stored oracle plans for the full-size GPU tests.

Calls only the oracle (`oracle/`) and the seeded input generator (`synth/`):
for a sample of slider weightings of the 3750 x 41200 case (81 weightings)
and of the 5000 x 61600 case (441 weightings) it runs the FP64 literal ADMM
of Eq. admm to relative residual 5e-5 (the stop the GPU tests solve to:
plans of these degenerate LPs are compared at the same stop; columns still
above it after 40000 iterations are stored with their residuals and
flagged), evaluates the plans' clinical metrics on a regular grid
(Sec. 3.B conventions), the weighted-sum objective of Sec. 2.A at the plans'
multipliers (the LP's dual objective: weak duality brackets the optimum
between it and c^T z1), and stores them as JSON.

    python tests/golden/make_full_size.py --cfg 1     # about 30 min on 4 host cores
    python tests/golden/make_full_size.py --cfg 2     # about 1-2 h (each iteration streams A)
    python tests/golden/make_full_size.py --cfg 3     # hours (A is 8.2 GB in FP64)

The sampled weightings (indices into `synth.cases.slider_weights(grid)`,
row-major over (s_LD, s_BOT)) are, for cfg 1 and 2, the four corners of the
slider grid, its centre and one off-centre point; index 0 (s_LD = s_BOT = 0,
the lowest BOT weight) converges slowest.  For the 9-target cfg 3 case the
lowest BOT weights take over 10^4 iterations, hours per weighting for the
FP64 oracle on the host, so its sample is four weightings of the upper half
of the BOT slider: the two top corners, the centre and one point between.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import admm as AD          # noqa: E402
from oracle import kkt as KK           # noqa: E402
from oracle import lp as L             # noqa: E402
from oracle import metrics as M        # noqa: E402
from synth import cases as SC          # noqa: E402

TOL = 5e-5
GRID_SPACING = {1: 2.0, 2: 2.0, 3: 2.0}    # mm
GRID_MARGIN = 12.0                     # mm


def sample_indices(g: int, cfg: int = 1) -> list[int]:
    c = g // 2
    if cfg == 3:            # upper half of the BOT slider (index = s_LD row * g + s_BOT column)
        return sorted({g - 1, g * g - 1, c * g + c, (c // 2) * g + (c + g) // 2})
    return sorted({0, g - 1, g * (g - 1), g * g - 1, c * g + c, (c // 2) * g + c // 2})


def run_chunked(lp, b, l, u, rho, max_iter, t0, chunk=2000):
    """oracle.admm.admm in chunks of `chunk` iterations on the columns still
    running, each chunk starting from the state the last one left (the
    iteration is the same as one long call; the chunks only report
    progress).  Returns an AdmmResult over all columns."""
    K = len(rho)
    n, m = lp.n, lp.m
    z1, z2, y1, y2 = np.zeros((n, K)), np.zeros((m, K)), np.zeros((n, K)), np.zeros((m, K))
    x1, x2 = np.zeros((n, K)), np.zeros((m, K))
    iters = np.zeros(K, dtype=np.int64)
    conv = np.zeros(K, dtype=bool)
    rp, rd = np.full(K, np.inf), np.full(K, np.inf)
    while (~conv).any() and iters.max() < max_iter:
        a = np.flatnonzero(~conv)
        r = AD.admm(lp.A, lp.c, b[:, a], l[:, a], u[:, a], rho[a], max_iter=chunk, tol=TOL,
                    state=(z1[:, a], z2[:, a], y1[:, a], y2[:, a]))
        z1[:, a], z2[:, a], y1[:, a], y2[:, a] = r.z1, r.z2, r.y1, r.y2
        x1[:, a], x2[:, a] = r.x1, r.x2
        iters[a] += r.iters
        conv[a] = r.converged
        rp[a], rd[a] = r.rel_pri, r.rel_dual
        print(f"  {time.time() - t0:.0f} s: iterations {iters.tolist()} converged {int(conv.sum())}/{K} "
              f"max rel_pri {rp[a].max():.2e} rel_dual {rd[a].max():.2e}", flush=True)
    return AD.AdmmResult(z1=z1, z2=z2, y1=y1, y2=y2, x1=x1, x2=x2, iters=iters, converged=conv,
                         rel_pri=rp, rel_dual=rd, rho=np.asarray(rho, dtype=np.float64))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cfg", type=int, required=True, choices=(1, 2, 3))
    ap.add_argument("--max-iter", type=int, default=40000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                f"full_size_cfg{a.cfg}.json")
    t0 = time.time()
    case = SC.workload_case(a.cfg)
    g = SC.WORKLOADS[a.cfg]["grid"]
    idx = sample_indices(g, a.cfg)
    W = SC.slider_weights(g)[idx]
    lp = L.precondition(L.assemble_case(case))
    rho0 = L.rho0_for(lp)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, rho0)
    b, l, u = L.bounds(lp, W)
    print(f"cfg{a.cfg}: A {lp.m} x {lp.n}, beta {lp.beta:.3f}, K {len(idx)}; "
          f"set-up {time.time() - t0:.0f} s", flush=True)
    res = run_chunked(lp, b, l, u, rho, a.max_iter, t0)
    print(f"ADMM {time.time() - t0:.0f} s, iterations {res.iters.tolist()}, "
          f"converged {res.converged.tolist()}", flush=True)
    lam = res.multipliers()                       # scaled multipliers rho y2 (m x K)
    t, tau = L.times_from_multipliers(lp, lam)
    pts, label, _ = SC.eval_grid(case, spacing=GRID_SPACING[a.cfg], margin=GRID_MARGIN)
    phi_eval = SC.dose_rate(pts, case.iso)
    d = M.dose(phi_eval, t)
    met = M.plan_metrics(d, label, case.d_presc, t, case.n_iso)
    rows = []
    for c, w in enumerate(idx):
        primal = float(lp.c @ res.z1[:, c])
        plan_obj, viol = KK.planning_objective(lp.A, b[:, c], lp.c, u[:, c], lam[:, c])
        rows.append(dict(
            index=int(w), W=W[c].tolist(), rho=float(rho[c]), iters=int(res.iters[c]),
            converged=bool(res.converged[c]), rel_pri=float(res.rel_pri[c]),
            rel_dual=float(res.rel_dual[c]), obj=primal, planning_objective=plan_obj,
            hard_violation=viol, max_lam=float(np.abs(lam[:, c]).max()),
            gap=abs(primal + plan_obj) / max(1.0, abs(primal)),
            coverage=float(met["coverage"][c]), selectivity=float(met["selectivity"][c]),
            gi=None if np.isnan(met["gi"][c]) else float(met["gi"][c]),
            bot=float(met["bot"][c])))
        print(rows[-1], flush=True)
    doc = dict(
        workload=SC.WORKLOADS[a.cfg]["name"], cfg=a.cfg, m=lp.m, n=lp.n, beta=lp.beta,
        rho0=rho0, w0_bot=SC.W0_BOT, tol=TOL, grid=g,
        eval_grid=dict(spacing=GRID_SPACING[a.cfg], margin=GRID_MARGIN, points=int(pts.shape[0])),
        method="oracle.admm.admm (FP64 literal ADMM, Eq. admm) to relative residual 5e-5; "
               "metrics by oracle.metrics.plan_metrics; planning objective by "
               "oracle.kkt.planning_objective",
        seconds=round(time.time() - t0, 1), plans=rows)
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", out, flush=True)


if __name__ == "__main__":
    main()
