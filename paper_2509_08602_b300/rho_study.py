"""Penalty study of Sec. 3.C (Eq. rho_rule), run through the library's public
API on the synthetic workloads.

Two protocols:

  * ``iters`` (default): every weighting of a g x g slider grid is solved to a
    relative residual ``tol`` with rho = mult * rho0 * sqrt(w0 / w_BOT),
    rho0 = 1100 beta, for each multiplier ``mult``; the table gives the
    largest and mean iteration count and the number of converged weightings.
    The largest count sets the time of a batch.
  * ``fixed``: the paper's own protocol -- a fixed number of iterations per
    multiplier, then the total objective and the beam-on-time term (the sum
    of the isocenter times tau) compared with a tight solve of the same
    weighting (tol 1e-6, multiplier 1).  The paper compares with the simplex
    optimum; the tight ADMM solve stands in for it here so that the study
    needs nothing but the library.

Usage (one GPU):

    python -m paper_2509_08602_b300.rho_study --cfgs 0 1 --mults 0.5,1,2
    python -m paper_2509_08602_b300.rho_study --protocol fixed --iters 2000
"""
import argparse
import json
import sys

import numpy as np

from paper_2509_08602_b300 import lgk
from synth import cases as SC

RHO0_PER_BETA = 1.1e3
MULTS = (0.35, 0.5, 0.71, 1.0, 1.41, 2.0, 4.0)


def rule(W, beta, mult):
    """Per-weighting penalty of Eq. rho_rule with the constant 1100 beta."""
    return mult * RHO0_PER_BETA * beta * np.sqrt(SC.W0_BOT / W[:, 3])


def open_case(cfg):
    c = SC.workload_case(cfg)
    cs = lgk.create_case(c.phi, c.kind, c.struct_id, c.n_iso, c.d_presc, c.q_area, c.q_vol,
                         c.d_ld1, c.d_ld2, c.phi_cal)
    return cs, SC.slider_weights(SC.WORKLOADS[cfg]["grid"])


def study_iters(cfg, mults, tol, max_iter):
    cs, W = open_case(cfg)
    rows = []
    for mult in mults:
        res = lgk.solve_weightings(cs, W, rule(W, cs.beta, mult), tol=tol, max_iter=max_iter)
        st = lgk.fetch_stats(res)
        res.close()
        rows.append(dict(cfg=cfg, K=len(W), mult=mult, max_iters=int(st["iters"].max()),
                         mean_iters=float(st["iters"].mean()), converged=int(st["converged"].sum())))
        print(json.dumps(rows[-1]), flush=True)
    cs.close()
    return rows


def study_fixed(cfg, mults, iters):
    cs, W = open_case(cfg)
    ref = lgk.solve_weightings(cs, W, rule(W, cs.beta, 1.0), tol=1e-6, max_iter=100000)
    st_ref = lgk.fetch_stats(ref)
    _, tau_ref = lgk.fetch_times(ref)
    ref.close()
    bot_ref = tau_ref.sum(axis=1)
    rows = []
    for mult in mults:
        res = lgk.solve_weightings(cs, W, rule(W, cs.beta, mult), tol=0.0, max_iter=iters)
        st = lgk.fetch_stats(res)
        _, tau = lgk.fetch_times(res)
        res.close()
        d_obj = np.abs(st["obj"] - st_ref["obj"]) / np.maximum(1.0, np.abs(st_ref["obj"]))
        d_bot = np.abs(tau.sum(axis=1) - bot_ref) / np.maximum(bot_ref, 1e-12)
        rows.append(dict(cfg=cfg, K=len(W), mult=mult, iters=iters,
                         obj_max=float(d_obj.max()), obj_mean=float(d_obj.mean()),
                         bot_max=float(d_bot.max()), bot_mean=float(d_bot.mean()),
                         ref_converged=int(st_ref["converged"].sum())))
        print(json.dumps(rows[-1]), flush=True)
    cs.close()
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--cfgs", type=int, nargs="+", default=[0, 1])
    ap.add_argument("--mults", default=",".join(str(m) for m in MULTS))
    ap.add_argument("--protocol", choices=("iters", "fixed"), default="iters")
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=12000)
    ap.add_argument("--iters", type=int, default=2000, help="iterations of the fixed protocol")
    args = ap.parse_args(argv)
    mults = [float(m) for m in args.mults.split(",")]
    for cfg in args.cfgs:
        if args.protocol == "iters":
            study_iters(cfg, mults, args.tol, args.max_iter)
        else:
            study_fixed(cfg, mults, args.iters)
    return 0


if __name__ == "__main__":
    sys.exit(main())
