"""Plain, slow FP64 CPU oracle for the batched-ADMM planning path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may use it.  It shares no code with the CUDA path: the two meet only
in the seeded input generator (`synth.cases`), which holds none of the
method's arithmetic.

Modules (each function cites the passage of arXiv 2509.08602 it follows):
  lp       -- dual LP assembly (Appendix A), preprocessing (Sec. 3.C),
              per-weighting bounds, rho rule (Eq. rho_rule), BF16 rounding
  admm     -- literal scaled-form ADMM (Eq. admm, Eq. partial_elimination)
  simplex  -- dense bounded-variable primal simplex (textbook)
  vertex   -- brute-force vertex enumeration for tiny LPs
  kkt      -- optimality (KKT) residuals and the primal objective of Sec. 2.A
  metrics  -- dose and clinical metrics (Sec. 2.A, Sec. 3.B)
  sampling -- second-pass low-dose volumes and Algorithm 1 (Sec. 2.C), with
              the SplitMix64 counter-based draws both sides implement

Parity status: every function here is pinned by `tests/test_oracle_*.py`
against closed forms, brute force, a library LP solver (HiGHS via scipy),
published generator outputs or invariants; none is "parity unpinned".
"""
