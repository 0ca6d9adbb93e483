"""Seeded synthetic Gamma Knife planning cases: the method's INPUTS only.

This module holds no arithmetic of the planning method (no LP assembly, no
scaling, no ADMM).  It produces what a treatment-planning system would export
and what the paper takes as given (Sec. 2.A, Sec. 3.B): dose points sampled
from volumes of interest, their class (target surface / interior, ring,
low-dose volumes, OAR), isocenter positions, dose-rate kernels phi at the dose
points, threshold doses, multi-target area/volume fractions (Appendix A) and
the weight vectors of a slider grid.  Both the CPU oracle and the CUDA path
consume these arrays.

The paper's kernels are exported from a proprietary planning system and its
patient data are not public, so the dose-rate kernel is a synthetic stand-in:

    phi(p; i, s, c) = (phi_cal / 8) * exp(-4 ln2 |p - x_i|^2 / F_c^2)
                      * (1 + gamma * cos(theta - theta_s))

with collimator FWHM F_c in {4, 8, 16} mm, sector angle theta_s = 2 pi (s+1/2)/8,
theta the azimuth of p - x_i, gamma = 0.5.  Beam variables are ordered
isocenter-major, then sector, then collimator, matching the Kronecker order of
C = I_N (x) I_8 (x) 1_{1x3} in Appendix A.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage

KIND_TS, KIND_TI, KIND_R, KIND_LD1, KIND_LD2, KIND_OAR = 0, 1, 2, 3, 4, 5
KIND_NAMES = ("TS", "TI", "R", "LD1", "LD2", "OAR")
N_SECTORS = 8
N_COLLIMATORS = 3
FWHM_MM = (4.0, 8.0, 16.0)
GAMMA_ANISO = 0.5
PHI_CAL = 3.0          # calibration dose rate, Gy/min (Sec. 3.B)
D_PRESC = 20.0         # prescription dose, Gy
D_LD1 = 10.0           # first low-dose threshold, Gy
D_LD2 = 5.0            # second low-dose threshold, Gy
W0_BOT = 1e-4          # lowest beam-on-time weight of the slider grid


@dataclasses.dataclass
class Case:
    """One planning case.  Arrays are C-contiguous numpy arrays."""
    name: str
    n_iso: int
    points: np.ndarray        # (P, 3) float64, mm
    kind: np.ndarray          # (P,) uint8, KIND_*
    struct_id: np.ndarray     # (P,) uint16, target index (TS/TI/R), OAR index (OAR), 0 (LD)
    iso: np.ndarray           # (N, 3) float64, mm
    phi: np.ndarray           # (P, 24 N) float64, Gy/min
    d_presc: np.ndarray       # (n_targets,) float64, Gy
    q_area: np.ndarray        # (n_targets,) fraction of total target surface
    q_vol: np.ndarray         # (n_targets,) fraction of total target volume
    d_oar: np.ndarray         # (n_oars,) float64, Gy
    d_ld1: float
    d_ld2: float
    phi_cal: float
    targets: list             # [(centre(3,), semi_axes(3,))]
    seed: int

    @property
    def n_pts(self) -> int:
        return int(self.points.shape[0])

    @property
    def n_beams(self) -> int:
        return 24 * self.n_iso

    @property
    def n_targets(self) -> int:
        return int(self.d_presc.shape[0])

    @property
    def n_oars(self) -> int:
        return int(self.d_oar.shape[0])


def dose_rate(points: np.ndarray, iso: np.ndarray, *, n_sectors: int = N_SECTORS,
              fwhm=FWHM_MM, gamma: float = GAMMA_ANISO, phi_cal: float = PHI_CAL,
              dtype=np.float64, chunk: int = 8192) -> np.ndarray:
    """Synthetic dose-rate kernels phi (P x N*n_sectors*len(fwhm)), Gy/min."""
    points = np.asarray(points, dtype=np.float64)
    iso = np.asarray(iso, dtype=np.float64)
    P, N = points.shape[0], iso.shape[0]
    C = len(fwhm)
    out = np.empty((P, N * n_sectors * C), dtype=dtype)
    theta_s = 2.0 * math.pi * (np.arange(n_sectors) + 0.5) / n_sectors
    inv_f2 = np.array([4.0 * math.log(2.0) / (f * f) for f in fwhm])
    for p0 in range(0, P, chunk):
        p1 = min(P, p0 + chunk)
        d = points[p0:p1, None, :] - iso[None, :, :]              # (p, N, 3)
        r2 = np.einsum("pnk,pnk->pn", d, d)
        theta = np.arctan2(d[..., 1], d[..., 0])                  # (p, N)
        radial = np.exp(-r2[..., None] * inv_f2[None, None, :])   # (p, N, C)
        aniso = 1.0 + gamma * np.cos(theta[..., None] - theta_s)  # (p, N, S)
        blk = (phi_cal / 8.0) * aniso[..., :, None] * radial[..., None, :]  # (p,N,S,C)
        out[p0:p1] = blk.reshape(p1 - p0, -1)
    return out


# ---------------------------------------------------------------- geometry

def _grid(targets, margin: float, h: float):
    lo = np.min([c - a for c, a in targets], axis=0) - margin
    hi = np.max([c + a for c, a in targets], axis=0) + margin
    axes = [np.arange(lo[d], hi[d] + 0.5 * h, h) for d in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return axes, np.stack([X, Y, Z], axis=-1)


def _labels(xyz, targets):
    lab = np.full(xyz.shape[:3], -1, dtype=np.int32)
    for k, (c, a) in enumerate(targets):
        q = ((xyz - c) / a) ** 2
        lab[q.sum(-1) <= 1.0] = k
    return lab


def _sample(rng, idx: np.ndarray, count: int, xyz_flat: np.ndarray, h: float):
    """`count` points uniform over the union of the voxels `idx` (voxel drawn
    uniformly with replacement, then a uniform position inside it)."""
    if count <= 0:
        return np.zeros((0, 3))
    pick = idx[rng.integers(0, idx.size, size=count)]
    return xyz_flat[pick] + rng.uniform(-0.5 * h, 0.5 * h, size=(count, 3))


def make_case(targets, *, n_target_pts: int, n_ring: int, n_ld1: int, n_ld2: int,
              n_iso: int, seed: int, name: str = "case", d_presc=None,
              oars=None, n_oar: int = 0,
              with_phi: bool = True, phi_dtype=np.float64) -> Case:
    """Sample dose points by class (Sec. 2.A) and build the inputs.

    Classes on a 1 mm voxel grid: TS = target voxels with a 6-neighbour outside
    their target, TI = other target voxels, R = 0 < dist <= 2 mm outside,
    LD1 = 3 <= dist < 10 mm, LD2 = 10 <= dist <= 25 mm (dist = distance to the
    nearest target voxel).  Target points are split between targets and
    between TS/TI by voxel share; ring points between targets by ring-voxel
    share.  Isocenters are distinct target voxels drawn uniformly.
    oars: optional list of (centre, semi-axes, maximum dose D_O) organs at
    risk (Appendix A); n_oar points are sampled in each, from its voxels
    outside the targets, and appended after the other classes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    targets = [(np.asarray(c, float), np.asarray(a, float)) for c, a in targets]
    h = 1.0
    _, xyz = _grid(targets, 26.0, h)
    lab = _labels(xyz, targets)
    inside = lab >= 0
    # surface: target voxel with a 6-neighbour not in the same target
    surf = np.zeros_like(inside)
    for ax in range(3):
        for sh in (-1, 1):
            nb = np.roll(lab, sh, axis=ax)
            surf |= inside & (nb != lab)
    dist, ind = ndimage.distance_transform_edt(~inside, sampling=h, return_indices=True)
    nearest = lab[tuple(ind)]
    xyz_flat = xyz.reshape(-1, 3)
    labf, surff, distf, nearf = lab.ravel(), surf.ravel(), dist.ravel(), nearest.ravel()

    nT = len(targets)
    pts, kinds, sids = [], [], []
    tvox = np.array([(labf == k).sum() for k in range(nT)], float)
    svox = np.array([((labf == k) & surff).sum() for k in range(nT)], float)
    alloc_t = _split(n_target_pts, tvox)
    for k in range(nT):
        ts_idx = np.flatnonzero((labf == k) & surff)
        ti_idx = np.flatnonzero((labf == k) & ~surff)
        n_ts, n_ti = _split(alloc_t[k], np.array([ts_idx.size, ti_idx.size], float))
        for kind, idx, cnt in ((KIND_TS, ts_idx, n_ts), (KIND_TI, ti_idx, n_ti)):
            pts.append(_sample(rng, idx, cnt, xyz_flat, h))
            kinds.append(np.full(cnt, kind, np.uint8))
            sids.append(np.full(cnt, k, np.uint16))
    ring = (labf < 0) & (distf > 0) & (distf <= 2.0)
    rvox = np.array([(ring & (nearf == k)).sum() for k in range(nT)], float)
    alloc_r = _split(n_ring, rvox)
    for k in range(nT):
        idx = np.flatnonzero(ring & (nearf == k))
        pts.append(_sample(rng, idx, alloc_r[k], xyz_flat, h))
        kinds.append(np.full(alloc_r[k], KIND_R, np.uint8))
        sids.append(np.full(alloc_r[k], k, np.uint16))
    for kind, cnt, sel in ((KIND_LD1, n_ld1, (distf >= 3.0) & (distf < 10.0)),
                           (KIND_LD2, n_ld2, (distf >= 10.0) & (distf <= 25.0))):
        idx = np.flatnonzero((labf < 0) & sel)
        pts.append(_sample(rng, idx, cnt, xyz_flat, h))
        kinds.append(np.full(cnt, kind, np.uint8))
        sids.append(np.zeros(cnt, np.uint16))
    points = np.ascontiguousarray(np.concatenate(pts))
    kind = np.ascontiguousarray(np.concatenate(kinds))
    struct_id = np.ascontiguousarray(np.concatenate(sids))

    tidx = np.flatnonzero(labf >= 0)
    iso = xyz_flat[rng.choice(tidx, size=n_iso, replace=False)].copy()
    d_oar = np.zeros(0)
    if oars:
        o_pts, o_kind, o_sid = [], [], []
        for o, (c, a, _) in enumerate(oars):
            c, a = np.asarray(c, float), np.asarray(a, float)
            idx = np.flatnonzero(((((xyz_flat - c) / a) ** 2).sum(1) <= 1.0) & (labf < 0))
            if idx.size == 0:
                raise ValueError(f"OAR {o} has no voxel outside the targets inside the grid")
            o_pts.append(_sample(rng, idx, n_oar, xyz_flat, h))
            o_kind.append(np.full(n_oar, KIND_OAR, np.uint8))
            o_sid.append(np.full(n_oar, o, np.uint16))
        points = np.ascontiguousarray(np.concatenate([points] + o_pts))
        kind = np.ascontiguousarray(np.concatenate([kind] + o_kind))
        struct_id = np.ascontiguousarray(np.concatenate([struct_id] + o_sid))
        d_oar = np.array([float(d) for _, _, d in oars])
    phi = dose_rate(points, iso, dtype=phi_dtype) if with_phi else None
    if d_presc is None:
        d_presc = np.full(nT, D_PRESC)
    return Case(name=name, n_iso=n_iso, points=points, kind=kind, struct_id=struct_id,
                iso=iso, phi=phi, d_presc=np.asarray(d_presc, float),
                q_area=svox / svox.sum(), q_vol=tvox / tvox.sum(),
                d_oar=d_oar, d_ld1=D_LD1, d_ld2=D_LD2, phi_cal=PHI_CAL,
                targets=targets, seed=seed)


def _split(total: int, share: np.ndarray) -> list:
    """Integer split of `total` proportional to `share` (largest remainder)."""
    share = np.asarray(share, float)
    if total <= 0 or share.sum() <= 0:
        return [0] * len(share)
    raw = total * share / share.sum()
    base = np.floor(raw).astype(int)
    rem = total - base.sum()
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rem]] += 1
    return [int(x) for x in base]


def _spheres(rng, count, rmin, rmax, box, first=None, gap=4.0, tries=10000):
    out = [] if first is None else [first]
    while len(out) < count + (0 if first is None else 1):
        for _ in range(tries):
            r = rng.uniform(rmin, rmax)
            c = rng.uniform(-box / 2, box / 2, size=3)
            if all(np.linalg.norm(c - c2) > r + a2[0] + gap for c2, a2 in out):
                out.append((c, np.full(3, r)))
                break
        else:
            raise RuntimeError("could not place non-overlapping spheres")
    return out


# ---------------------------------------------------------------- workloads

WORKLOADS = {
    # one sphere r=8 mm; 1500 target + 3 x 1000 shell points; 20 isocenters; 3x3 sliders
    0: dict(name="sphere8_p4500_iso20_k9", grid=3, n_iso=20,
            n_target_pts=1500, n_ring=1000, n_ld1=1000, n_ld2=1000),
    # ellipsoid 30 x 22 x 18.8 mm (52 cm^3); 12000 target + 28000 shell; 150 iso; 9x9
    1: dict(name="ellipsoid52cc_p40000_iso150_k81", grid=9, n_iso=150,
            n_target_pts=12000, n_ring=9334, n_ld1=9333, n_ld2=9333),
    # sphere r=8 + 3 spheres r in U[5,15]; 60000 points (30 % target); 200 iso; 21x21
    2: dict(name="4targets_p60000_iso200_k441", grid=21, n_iso=200,
            n_target_pts=18000, n_ring=14000, n_ld1=14000, n_ld2=14000),
    # 9 spheres r in U[3,12] in a 60 mm cube; 120000 points; 333 iso; 21x21
    3: dict(name="9targets_p120000_iso333_k441", grid=21, n_iso=333,
            n_target_pts=36000, n_ring=28000, n_ld1=28000, n_ld2=28000),
}


def workload_targets(cfg: int, rng):
    if cfg == 0:
        return [(np.zeros(3), np.full(3, 8.0))]
    if cfg == 1:
        return [(np.zeros(3), np.array([30.0, 22.0, 18.8]))]
    if cfg == 2:
        return _spheres(rng, 3, 5.0, 15.0, 70.0, first=(np.zeros(3), np.full(3, 8.0)))
    if cfg == 3:
        return _spheres(rng, 9, 3.0, 12.0, 60.0)
    raise ValueError(cfg)


def workload_case(cfg: int, *, with_phi: bool = True, phi_dtype=np.float64,
                  seed: int | None = None) -> Case:
    """The synthetic stand-in for one of the paper's case sizes (Table 1 shapes)."""
    spec = dict(WORKLOADS[cfg])
    seed = 1000 + cfg if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    targets = workload_targets(cfg, rng)
    name = spec.pop("name")
    spec.pop("grid")
    return make_case(targets, seed=seed, name=name, with_phi=with_phi,
                     phi_dtype=phi_dtype, **spec)


def slider_weights(grid: int, w0_bot: float = W0_BOT) -> np.ndarray:
    """Weight vectors (w_T, w_R, w_LD, w_BOT) for a grid x grid slider grid.

    The paper does not state the slider-to-weight map (Sec. 3.B); this reading
    keeps w_T = w_R = 1, sets w_LD = s_LD and w_BOT = w0 * 10^(3 s_BOT), so the
    lowest allowed BOT weight is w0 = 1e-4 and the grid spans the range over
    which the synthetic plans trade beam-on time for coverage (about 60 to 14
    minutes on the r = 8 mm sphere).  Row-major over (s_LD, s_BOT).
    """
    s = np.linspace(0.0, 1.0, grid) if grid > 1 else np.array([0.5])
    W = []
    for s_ld in s:
        for s_bot in s:
            W.append((1.0, 1.0, s_ld, w0_bot * 10.0 ** (3.0 * s_bot)))
    return np.ascontiguousarray(np.array(W, dtype=np.float64))


def eval_grid(case: Case, spacing: float = 1.0, margin: float = 12.0):
    """Regular evaluation grid over the targets' bounding box + margin.

    Returns (points (E,3), target_label (E,) int32 with -1 outside all
    targets, voxel volume mm^3).
    """
    _, xyz = _grid(case.targets, margin, spacing)
    lab = _labels(xyz, case.targets)
    return (np.ascontiguousarray(xyz.reshape(-1, 3)), lab.ravel().astype(np.int32),
            spacing ** 3)
