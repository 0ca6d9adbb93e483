"""Second-pass low-dose volumes and non-redundant point sampling (Sec. 2.C,
Algorithm 1).

Test infrastructure (see oracle/__init__.py).  Plain Python sets and exact
integer / rational arithmetic.

The second pass of the two-pass optimisation replaces the first pass's
low-dose points (a geometric expansion of the targets) by points of the
low-dose volume of each weighting's first-pass plan: the part of the
candidate region whose first-pass dose lies in [D_LD, D_LD + Delta).  As the
volumes differ per weighting, Algorithm 1 samples them so that overlapping
volumes share points: volumes are visited by decreasing sampling density
omega_j = N_j / |V_j|; at each, the union's current points are thinned to
omega_j |V_union| points, those inside V_j are reused, and omega_j times the
part of V_j outside the union is drawn fresh.  A weighting's second-pass LP
keeps its own sample p_j of the union P (the other union points get u = 0).

Readings where the paper is silent:
  * counts omega_j |X| are rounded to nearest, halves up (exact rationals);
  * a draw of k items takes the k with the smallest random keys (ties:
    smaller index), i.e. a uniformly random k-subset, and asks for at most
    the whole set;
  * the keys come from a counter-based generator, SplitMix64 (Steele, Lea
    and Flood, "Fast splittable pseudorandom number generators", OOPSLA
    2014), so both implementations draw the same points:
        key(i) = f(f(f(f(seed) ^ level) ^ (2 j + s)) ^ i)
    with f the generator's output for state x (x + golden gamma, mixed),
    s = 0 for the thinning draw, 1 for the fresh draw, i the candidate;
  * N_j is capped at |V_j| (omega_j <= 1); empty volumes are skipped.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(x: int) -> int:
    """Output of a SplitMix64 generator in state x (its first output when
    seeded with x)."""
    z = (x + GOLDEN_GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw_key(seed: int, level: int, j: int, s: int, i: int) -> int:
    f = splitmix64
    return f(f(f(f(seed & MASK64) ^ level) ^ (2 * j + s)) ^ i)


def draw(items, k: int, seed: int, level: int, j: int, s: int) -> set:
    """k items of `items` chosen uniformly without replacement (all if k >= |items|)."""
    items = sorted(items)
    if k >= len(items):
        return set(items)
    ranked = sorted(items, key=lambda i: (draw_key(seed, level, j, s, i), i))
    return set(ranked[:k])


def round_half_up(x: Fraction) -> int:
    return int((x + Fraction(1, 2)).__floor__())


def low_dose_volume(dose, d_lo: float, delta: float):
    """Indices of the candidates with dose in [d_lo, d_lo + delta) (Sec. 2.C)."""
    hi = d_lo + delta
    d = np.asarray(dose, dtype=np.float64)
    return set(np.flatnonzero((d >= d_lo) & (d < hi)).tolist())


def algorithm1(volumes, n_desired, seed: int, level: int = 0):
    """Algorithm 1 on the volumes V_j (sets of candidate indices).

    Returns (P, samples): P the sorted union of the samples, samples[j] = p_j
    (a set; empty for an empty volume)."""
    K = len(volumes)
    V = [set(v) for v in volumes]
    N = [min(max(int(n_desired[j]), 0), len(V[j])) for j in range(K)]
    order = sorted((j for j in range(K) if V[j]), key=lambda j: (-Fraction(N[j], len(V[j])), j))
    V_union, p_union = set(), set()
    samples = [set() for _ in range(K)]
    for j in order:
        omega = Fraction(N[j], len(V[j]))
        p_tilde = draw(p_union, round_half_up(omega * len(V_union)), seed, level, j, 0)
        p_in = p_tilde & V[j]
        fresh = V[j] - V_union
        p_out = draw(fresh, round_half_up(omega * len(fresh)), seed, level, j, 1)
        samples[j] = p_in | p_out
        p_union = p_tilde | p_out
        V_union = V[j] | V_union
    P = sorted(set().union(*samples))
    return P, samples
