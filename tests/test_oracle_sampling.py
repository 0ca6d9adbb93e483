"""Pins of the second-pass sampling oracle (Sec. 2.C, Algorithm 1) and CPU
parity of the library's Algorithm 1 with it (host code: no GPU needed)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import sampling as SA

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_splitmix64_reference_outputs():
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    state, got = 1234567, []
    for _ in range(len(want)):
        got.append(SA.splitmix64(state))
        state = (state + SA.GOLDEN_GAMMA) & SA.MASK64
    assert got == want


def test_draw_is_a_uniform_subset():
    """All C(5, 2) = 10 subsets appear equally often over seeds (chi-square)."""
    counts = {}
    n_seeds = 4000
    for seed in range(n_seeds):
        s = frozenset(SA.draw(range(5), 2, seed, 0, 0, 1))
        assert len(s) == 2
        counts[s] = counts.get(s, 0) + 1
    assert len(counts) == 10
    e = n_seeds / 10
    chi2 = sum((c - e) ** 2 / e for c in counts.values())
    assert chi2 < 27.9          # 9 degrees of freedom, p = 0.001
    assert SA.draw(range(5), 9, 1, 0, 0, 0) == set(range(5))


def test_low_dose_volume_half_open_range():
    d = np.array([9.999, 10.0, 10.5, 11.0, 11.0000001, 4.0])
    assert SA.low_dose_volume(d, 10.0, 1.0) == {1, 2}


def test_disjoint_volumes_sample_exactly_their_targets():
    V = [set(range(0, 100)), set(range(100, 400)), set(range(400, 450))]
    P, p = SA.algorithm1(V, [40, 90, 80], seed=3)
    assert [len(x) for x in p] == [40, 90, 50]          # 80 capped at |V_3| = 50
    for j in range(3):
        assert p[j] <= V[j]
    assert P == sorted(p[0] | p[1] | p[2])


def test_identical_volumes_share_every_point():
    V = [set(range(500))] * 4
    P, p = SA.algorithm1(V, [120] * 4, seed=11)
    assert all(x == p[0] for x in p) and len(p[0]) == 120 and len(P) == 120


def test_nested_volumes_reuse_and_top_up():
    """V_2 inside V_1, same desired count: V_2 is denser, drawn first; V_1
    reuses omega_1 |V_2| of those points and draws omega_1 |V_1 \\ V_2| fresh."""
    V1, V2 = set(range(1000)), set(range(200, 400))
    P, p = SA.algorithm1([V1, V2], [250, 250], seed=5)
    assert len(p[1]) == 200                               # omega_2 = 1 (capped)
    w1 = Fraction(250, 1000)
    k_in = SA.round_half_up(w1 * 200)
    assert len(p[0] & V2) == k_in and len(p[0] - V2) == SA.round_half_up(w1 * 800)
    assert p[0] & V2 <= p[1]                              # reused, not redrawn
    assert len(P) == len(p[0] | p[1])


def test_empty_and_zero_requests():
    V = [set(), set(range(10)), set(range(5, 30))]
    P, p = SA.algorithm1(V, [5, 0, 10], seed=1)
    assert p[0] == set() and p[1] == set()
    assert len(p[2]) == 10                  # p_union was emptied by omega = 0: all fresh


def test_relative_std_bound_over_seeds():
    """Sec. 2.C: |p_j ∩ union| is (about) binomial with standard deviation
    sqrt(|p~| r (1 - r)); relative to omega_j |V_j| it stays below
    1 / sqrt(omega_j |V_j|).  Two overlapping volumes of a 1-D line, the
    denser first: the second's reused count varies with the seed."""
    V1 = set(range(0, 2000))             # density 400 / 2000 = 0.2, drawn second
    V2 = set(range(1500, 2300))          # density 400 / 800 = 0.5, drawn first
    n = 400
    reused = []
    for seed in range(300):
        _, p = SA.algorithm1([V1, V2], [n, n], seed=seed)
        reused.append(len(p[0] & V2))
    reused = np.array(reused, float)
    w1 = n / len(V1)
    k_tilde = SA.round_half_up(Fraction(n, len(V1)) * len(V2))        # |p~| from the union's 400 points
    r = len(V1 & V2) / len(V2)
    std_binom = math.sqrt(k_tilde * r * (1 - r))
    assert reused.std(ddof=1) <= 1.2 * std_binom
    assert abs(reused.mean() - k_tilde * r) <= 4 * std_binom / math.sqrt(len(reused))
    assert reused.std(ddof=1) / (w1 * len(V1)) < 1 / math.sqrt(w1 * len(V1))


# --------------------------------------------------------- library parity (CPU)
@pytest.fixture(scope="module")
def lgk():
    from paper_2509_08602_b300 import build
    build.build()
    from paper_2509_08602_b300 import lgk as mod
    return mod


def _random_volumes(rng, K, n_cand):
    """Shell-like overlapping volumes: intervals of a shuffled candidate order
    (so that bit positions are scattered), a few empty, one full."""
    perm = rng.permutation(n_cand)
    vols = []
    for j in range(K):
        if j % 11 == 5:
            vols.append(np.zeros(n_cand, bool))
            continue
        a = int(rng.integers(0, n_cand // 2))
        b = int(min(n_cand, a + rng.integers(1, n_cand // 2)))
        m = np.zeros(n_cand, bool)
        m[perm[a:b]] = True
        vols.append(m)
    vols[-1][:] = True
    return np.array(vols)


@pytest.mark.parametrize("K,n_cand,seed", [(1, 40, 0), (12, 3001, 7), (33, 2048, 2 ** 63 + 5),
                                           (70, 517, 123)])
def test_library_algorithm1_matches_oracle(lgk, K, n_cand, seed):
    rng = np.random.default_rng(K * 1000 + n_cand)
    member = _random_volumes(rng, K, n_cand)
    n_desired = rng.integers(0, n_cand // 3 + 2, size=K)
    n_desired[0] = 10 ** 6            # more than any volume: capped
    for level in (0, 1):
        idx, sel = lgk.sample_low_dose(member, n_desired, seed=seed, level=level)
        P, p = SA.algorithm1([set(np.flatnonzero(m).tolist()) for m in member], n_desired,
                             seed=seed, level=level)
        assert idx.tolist() == P
        for j in range(K):
            assert set(idx[sel[:, j]].tolist()) == p[j], j


def test_library_algorithm1_rejects_bad_arguments(lgk):
    with pytest.raises(lgk.LgkError) as e:
        lgk.sample_low_dose(np.zeros((0, 10), bool), [], seed=0)
    assert e.value.code == 1
