"""Dual LP of Appendix A, its preprocessing (Sec. 3.C) and per-weighting data.

Test infrastructure (see oracle/__init__.py).  Plain FP64 numpy.

The dual LP (Eq. dual_problem, Appendix A):

    minimize c^T x  s.t.  A x <= b,  l <= x <= u

Rows of A: the 24 N beam variables (isocenter-major, then sector, then
collimator), then the N isocenter beam-on-time rows.  Columns: one per dose
point, in input order, then one per (isocenter, sector) pair for the
beam-on-time coupling (the block -C_S^T over T^T).  Kind codes of
`synth.cases`: 0 TS, 1 TI, 2 R, 3 LD1, 4 LD2, 5 OAR.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TS, TI, R, LD1, LD2, OAR = 0, 1, 2, 3, 4, 5


@dataclasses.dataclass
class DualLP:
    A: np.ndarray            # (m, n) float64
    c: np.ndarray            # (n,)
    kind: np.ndarray         # (n,) int: point kind, or -1 for the BOT columns
    struct_id: np.ndarray    # (n,) int
    n_iso: int
    n_sectors: int
    n_coll: int
    n_pts: int
    counts: dict             # (kind, struct) -> number of points
    n_targets: int
    row_scale: np.ndarray    # (m,) D_r applied to the rows (ones if unscaled)
    beta: float              # BOT-column scale applied (1 if unscaled)
    q_area: np.ndarray       # (n_targets,) share of total target surface
    q_vol: np.ndarray        # (n_targets,) share of total target volume

    @property
    def m(self):
        return self.A.shape[0]

    @property
    def n(self):
        return self.A.shape[1]

    @property
    def n_beams(self):
        return self.n_iso * self.n_sectors * self.n_coll


def assemble(phi, kind, struct_id, n_iso, d_presc, d_ld1, d_ld2, phi_cal,
             d_oar=(), n_sectors=8, n_coll=3, q_area=None, q_vol=None) -> DualLP:
    """Build A and c of the dual LP exactly as Appendix A states.

    A = [ phi_TS^T/D  phi_TI^T/D  -phi_R^T/D  -phi_LD^T/D_LD  -phi_O^T/D_O  -C_S^T ]
        [    0           0           0             0              0         T^T   ]
    C = I_N (x) I_8 (x) 1_{1x3},  T = I_N (x) 1_{8x1},  C_S = C / (D_T / phi_cal)
    c = (-1, -1, 1, 1, 1, 0) blockwise.  With several targets the TS/TI/R blocks
    are per target with that target's prescription and C_S uses the mean
    prescription (Appendix A, multi-target extension).
    """
    phi = np.asarray(phi, dtype=np.float64)
    kind = np.asarray(kind).astype(int)
    struct_id = np.asarray(struct_id).astype(int)
    d_presc = np.atleast_1d(np.asarray(d_presc, dtype=np.float64))
    d_oar = np.atleast_1d(np.asarray(d_oar, dtype=np.float64))
    P, B = phi.shape
    assert B == n_iso * n_sectors * n_coll
    m = B + n_iso
    NS = n_iso * n_sectors
    n = P + NS
    A = np.zeros((m, n))
    c = np.zeros(n)
    # point columns: sign and threshold per class
    D = np.empty(P)
    sign = np.empty(P)
    for p in range(P):
        k = kind[p]
        if k in (TS, TI):
            D[p], sign[p], c[p] = d_presc[struct_id[p]], 1.0, -1.0
        elif k == R:
            D[p], sign[p], c[p] = d_presc[struct_id[p]], -1.0, 1.0
        elif k == LD1:
            D[p], sign[p], c[p] = d_ld1, -1.0, 1.0
        elif k == LD2:
            D[p], sign[p], c[p] = d_ld2, -1.0, 1.0
        elif k == OAR:
            D[p], sign[p], c[p] = d_oar[struct_id[p]], -1.0, 1.0
        else:
            raise ValueError(f"unknown point kind {k}")
    A[:B, :P] = (phi * (sign / D)[:, None]).T
    # BOT columns: -C_S^T on beam rows, T^T on isocenter rows
    d_mean = float(np.mean(d_presc))
    Cmat = np.kron(np.eye(NS), np.ones((1, n_coll)))          # (N*8, 24N)
    Tmat = np.kron(np.eye(n_iso), np.ones((n_sectors, 1)))    # (N*8, N)
    A[:B, P:] = -(Cmat / (d_mean / phi_cal)).T
    A[B:, P:] = Tmat.T
    counts = {}
    for k, s in zip(kind, struct_id):
        counts[(int(k), int(s))] = counts.get((int(k), int(s)), 0) + 1
    col_kind = np.concatenate([kind, -np.ones(NS, int)])
    col_sid = np.concatenate([struct_id, np.zeros(NS, int)])
    nT = len(d_presc)
    q_area = np.ones(nT) / nT if q_area is None else np.asarray(q_area, float)
    q_vol = np.ones(nT) / nT if q_vol is None else np.asarray(q_vol, float)
    return DualLP(A=A, c=c, kind=col_kind, struct_id=col_sid, n_iso=n_iso,
                  n_sectors=n_sectors, n_coll=n_coll, n_pts=P, counts=counts,
                  n_targets=nT, row_scale=np.ones(m), beta=1.0,
                  q_area=q_area, q_vol=q_vol)


def assemble_case(case, n_sectors=8, n_coll=3) -> DualLP:
    return assemble(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                    case.d_ld1, case.d_ld2, case.phi_cal, case.d_oar, n_sectors, n_coll,
                    q_area=case.q_area, q_vol=case.q_vol)


def beta_factor(lp: DualLP) -> float:
    """BOT column scale of Sec. 3.C: (N_TS + N_TI + N_R + N_1LD + N_2LD) / 2000
    (OAR points excluded)."""
    n_cost = sum(v for (k, _), v in lp.counts.items() if k != OAR)
    return n_cost / 2000.0


def precondition(lp: DualLP, *, normalize_rows=True, scale_bot=True) -> DualLP:
    """Sec. 3.C: normalise the rows of A to unit Euclidean norm (D_r, which also
    scales b), then multiply the BOT columns by beta.  c, l and u are unchanged:
    the BOT columns have c = 0, l = 0, u = inf, so scaling them is a change of
    variables mu' = mu / beta that leaves the optimum value unchanged."""
    A = lp.A.copy()
    m = A.shape[0]
    d_r = np.ones(m)
    if normalize_rows:
        norms = np.sqrt(np.sum(A * A, axis=1))
        d_r = np.where(norms > 0, 1.0 / np.where(norms > 0, norms, 1.0), 1.0)
        A = A * d_r[:, None]
    beta = 1.0
    if scale_bot:
        beta = beta_factor(lp)
        A[:, lp.n_pts:] *= beta
    return dataclasses.replace(lp, A=A, row_scale=d_r, beta=beta)


def bounds(lp: DualLP, W, select=None) -> tuple:
    """Per-weighting (b, l, u) columns (Appendix A), each (m or n) x K.

    u = (w_TS/N_TS, w_TI/N_TI, w_R/N_R, w_LD/N_LD, inf, inf); with several
    targets w_kTS = q_kA w_T, w_kTI = q_kV w_T, w_kR = w_R / n_targets, each
    normalised by that target's own point count.  Each low-dose volume (LD1,
    LD2) gets w_LD over its own point count.  b = (0, w_BOT), times the row
    scale D_r when the rows were normalised.

    select (n_pts, K) bool, optional: the dose points each weighting keeps
    (Sec. 2.C, second pass); the others get u = 0, and each class's point
    count is the count of its selected points in that weighting.
    """
    W = np.atleast_2d(np.asarray(W, dtype=np.float64))
    K = W.shape[0]
    qa, qv = lp.q_area, lp.q_vol
    nT = lp.n_targets
    u = np.full((lp.n, K), np.inf)
    if select is None:
        select = np.ones((lp.n_pts, K), dtype=bool)
    select = np.asarray(select, dtype=bool)
    counts = {}
    for j in range(lp.n_pts):
        key = (int(lp.kind[j]), int(lp.struct_id[j]))
        counts[key] = counts.get(key, 0) + select[j].astype(np.int64)
    for j in range(lp.n):
        k, s = int(lp.kind[j]), int(lp.struct_id[j])
        if k < 0 or k == OAR:
            continue
        cnt = counts[(k, s)].astype(np.float64)
        cnt[cnt == 0] = np.inf       # a class with no selected point: u = 0
        wT, wR, wLD = W[:, 0], W[:, 1], W[:, 2]
        if k == TS:
            u[j] = qa[s] * wT / cnt
        elif k == TI:
            u[j] = qv[s] * wT / cnt
        elif k == R:
            u[j] = (wR / nT) / cnt
        else:  # LD1, LD2
            u[j] = wLD / cnt
        u[j] = np.where(select[j], u[j], 0.0)
    l = np.zeros((lp.n, K))
    b = np.zeros((lp.m, K))
    b[lp.n_beams:, :] = W[:, 3][None, :]
    b *= lp.row_scale[:, None]
    return b, l, u


RHO0_PAPER = 2.5e-3
RHO0_PER_BETA = 1.1e3


def rho0_for(lp: DualLP) -> float:
    """Constant of Eq. rho_rule for this case: RHO0_PER_BETA * beta.

    The paper's constant rho0 = 2.5e-3 was tuned (Sec. 3.C) for its kernels'
    units, which it does not state.  The bounds u = w / N_alpha make the dual
    variables scale as 1 / (number of points) while the multipliers (sector
    times) do not, so the balancing penalty grows with the point count; beta =
    (#non-OAR points) / 2000 of Sec. 3.C is that count.  Re-running the paper's
    tuning procedure (grid of rho values, objective against the simplex
    optimum, iterations to tolerance) on three synthetic case sizes puts the
    best constant at 1.1e3 * beta on all three."""
    return RHO0_PER_BETA * lp.beta


def rho_rule(w_bot, w0_bot: float, rho0: float) -> np.ndarray:
    """Eq. rho_rule: rho = rho0 * sqrt(w_0,BOT / w_BOT)."""
    return rho0 * np.sqrt(w0_bot / np.asarray(w_bot, dtype=np.float64))


def times_from_multipliers(lp: DualLP, lam_scaled) -> tuple:
    """Sector times t and isocenter BOT tau from the multipliers of the scaled
    constraints A'x' <= b' (Sec. 2.B: the primal solution is rho*y2; undoing the
    row scaling gives lambda = D_r * lambda').  Returns (t (B x K), tau (N x K))."""
    lam = np.asarray(lam_scaled, dtype=np.float64)
    if lam.ndim == 1:
        lam = lam[:, None]
    lam = lam * lp.row_scale[:, None]
    return lam[:lp.n_beams], lam[lp.n_beams:]


def bf16_round(x) -> np.ndarray:
    """Round FP64 values to the nearest bfloat16 (8 significant bits, ties to
    even, exponent range of FP32, subnormals down to 2^-133), returned as
    float64.  Plain definition of IEEE round-to-nearest-even on that format."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = (x != 0) & np.isfinite(x)
    ax = np.abs(x[nz])
    _, e = np.frexp(ax)                 # ax = f * 2^e, f in [0.5, 1)
    e = e - 1                           # ax in [2^e, 2^(e+1))
    e = np.maximum(e, -126)             # below 2^-126 the spacing is fixed
    q = np.ldexp(1.0, e - 7)            # spacing of 8-bit significands
    r = np.rint(ax / q) * q             # rint: ties to even
    r = np.where(r >= np.ldexp(1.0, 128), np.inf, r)
    out[nz] = np.sign(x[nz]) * r
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    return out
