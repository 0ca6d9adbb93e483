"""Record how many iterations the FP64 oracle ADMM needs per plan at the
benchmark's tolerance, so that the benchmark's CPU baseline and its
reference arm both extrapolate a timed oracle iteration with the oracle's
own iteration count (not the device's, and not the paper's fixed 3000).

Calls only the oracle (`oracle/`) and the seeded generator (`synth/`):
oracle.admm.admm (FP64 literal ADMM, Eq. admm) with the rho rule of
Eq. rho_rule, the residual test at tol 1e-4 every 10 iterations.

    python tests/golden/make_oracle_iters.py            # cfg0 and cfg1 (the bench's line)
    python tests/golden/make_oracle_iters.py 2          # the cfg2 sample (hours on the host)

cfg0 (9 weightings) and cfg1 (81 weightings) run every weighting of their
slider grid; cfg2 (441 weightings) runs a 21-weighting sample that holds
every BOT weight of its grid once (s_BOT index i with s_LD index 7 i mod 21).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import admm as AD          # noqa: E402
from oracle import lp as L             # noqa: E402
from synth import cases as SC          # noqa: E402

TOL = 1e-4
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iters.json")


def sample(cfg: int):
    g = SC.WORKLOADS[cfg]["grid"]
    if cfg < 2:
        return list(range(g * g)), "every weighting of the grid"
    return [((7 * i) % g) * g + i for i in range(g)], \
        f"{g} weightings: s_BOT index i with s_LD index 7 i mod {g}"


def main():
    cfgs = [int(a) for a in sys.argv[1:]] or [0, 1]
    doc = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            doc = json.load(f)
    for cfg in cfgs:
        t0 = time.time()
        case = SC.workload_case(cfg)
        idx, how = sample(cfg)
        W = SC.slider_weights(SC.WORKLOADS[cfg]["grid"])[idx]
        lp = L.precondition(L.assemble_case(case))
        b, l, u = L.bounds(lp, W)
        rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
        res = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=40000, tol=TOL)
        doc[f"cfg{cfg}"] = dict(
            workload=SC.WORKLOADS[cfg]["name"], tol=TOL, sample=how, K=len(idx),
            mean_iters=float(res.iters.mean()), max_iters=int(res.iters.max()),
            converged=int(res.converged.sum()), iters=res.iters.tolist(),
            seconds=round(time.time() - t0, 1))
        print(cfg, doc[f"cfg{cfg}"]["mean_iters"], doc[f"cfg{cfg}"]["max_iters"],
              doc[f"cfg{cfg}"]["converged"], flush=True)
        with open(OUT, "w") as f:
            json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
