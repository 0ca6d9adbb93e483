"""Group solve (lgk_solve_group): cases of different sizes, each with its own
weighting set, iterated together, every tensor-core product of an iteration
one persistent launch over all of them.

Each case's products are cut into the same stream-K runs and summed in the
same order as in a solve of that case alone, so a group member's plan is
bitwise the plan of lgk_solve_weightings with the same arguments: the test
compares the q-form states, iteration counts and objectives exactly, for the
default iteration form and with one refinement step of the x-update's solve.
A member that cannot take 256-row tiles (more than 128 weightings) moves the
group to 128-row tiles; those members are then compared with their solo
plans at the objective bar (1e-3) instead, since the sums run in another
order.  Bad groups are refused on the host.
"""
import numpy as np
import pytest

from synth import cases as SC

pytestmark = pytest.mark.gpu

W0 = SC.W0_BOT


@pytest.fixture(scope="module")
def lgk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_08602_b300 import build
    build.build()
    from paper_2509_08602_b300 import lgk as mod
    return mod


def small_case(seed, n_iso, n_target):
    rng = np.random.default_rng(seed)
    r = float(rng.uniform(5.0, 9.0))
    return SC.make_case([(np.zeros(3), np.full(3, r))], n_target_pts=n_target, n_ring=300, n_ld1=300,
                        n_ld2=300, n_iso=n_iso, seed=seed)


def create(lgk, case, **kw):
    return lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area,
                           case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                           params=lgk.default_params(refine_after=0, **kw))


def members(lgk, **kw):
    """Three cases of different shapes (m x n: 500 x 4660, 300 x 1596,
    400 x 2220) with 9, 17 and 40 weightings."""
    specs = [(SC.workload_case(0), SC.slider_weights(3)),
             (small_case(5, 12, 600), SC.slider_weights(5)[:17]),
             (small_case(6, 16, 800), SC.slider_weights(7)[:40])]
    cases = [create(lgk, c, **kw) for c, _ in specs]
    return cases, [w for _, w in specs]


def rule(cs):
    return 1100.0 * cs.beta


@pytest.mark.parametrize("refine", [0, 1], ids=["default", "refined_solve"])
def test_group_members_equal_their_solo_solves_bitwise(lgk, refine):
    cases, Ws = members(lgk, solve_refine=refine)
    kw = dict(w0_bot=W0, tol=1e-4, max_iter=1500)
    solo = [lgk.solve_weightings(c, W, None, rho0=rule(c), **kw) for c, W in zip(cases, Ws)]
    group = lgk.solve_group(cases, Ws, None, rho0=[rule(c) for c in cases], **kw)
    for a, b in zip(solo, group):
        sa, sb = lgk.fetch_stats(a), lgk.fetch_stats(b)
        np.testing.assert_array_equal(sb["iters"], sa["iters"])
        np.testing.assert_array_equal(sb["obj"], sa["obj"])
        np.testing.assert_array_equal(sb["converged"], sa["converged"])
        qa, qb = lgk.fetch_state(a), lgk.fetch_state(b)
        np.testing.assert_array_equal(qb[0], qa[0])
        np.testing.assert_array_equal(qb[1], qa[1])
        ta, _ = lgk.fetch_times(a)
        tb, _ = lgk.fetch_times(b)
        np.testing.assert_array_equal(tb, ta)
    for r in solo + group:
        r.close()
    for c in cases:
        c.close()


def test_members_stop_on_their_own(lgk):
    """The first member stops long before the second (three fast weightings
    of the sphere case against 40 of another case): the later launches skip
    it, and both members still equal their solo solves bit for bit."""
    cases, Ws = members(lgk)
    cases[1].close()
    cases = [cases[0], cases[2]]
    Ws = [Ws[0][[2, 5, 8]], Ws[2]]                    # the sphere's fastest weightings first
    kw = dict(w0_bot=W0, tol=1e-4, max_iter=3000)
    group = lgk.solve_group(cases, Ws, None, rho0=[rule(c) for c in cases], **kw)
    solo = [lgk.solve_weightings(c, W, None, rho0=rule(c), **kw) for c, W in zip(cases, Ws)]
    its = [int(lgk.fetch_stats(r)["iters"].max()) for r in group]
    assert its[0] + 100 <= its[1], its
    for a, b in zip(solo, group):
        sa, sb = lgk.fetch_stats(a), lgk.fetch_stats(b)
        np.testing.assert_array_equal(sb["iters"], sa["iters"])
        np.testing.assert_array_equal(sb["obj"], sa["obj"])
        np.testing.assert_array_equal(lgk.fetch_state(b)[0], lgk.fetch_state(a)[0])
    for r in solo + group:
        r.close()
    for c in cases:
        c.close()


def test_a_wide_member_moves_the_group_to_128_row_tiles(lgk):
    cases, Ws = members(lgk)
    big = SC.slider_weights(13)[:150]                 # 150 weightings: no 256-row tiles
    Ws = [Ws[0], big]
    cases[2].close()
    cases = cases[:2]
    # both sides stop at 5e-5, as the converged parity tests do: two plans
    # stopped at 1e-4 on differently rounded paths can sit just over 1e-3
    # apart in objective on these degenerate LPs
    # (past 8000 iterations both switch to the literal iteration at the same
    # boundary: the 150-weighting member is then the oldest one running)
    kw = dict(w0_bot=W0, tol=5e-5, max_iter=30000)
    group = lgk.solve_group(cases, Ws, None, rho0=[rule(c) for c in cases], **kw)
    solo = [lgk.solve_weightings(c, W, None, rho0=rule(c), **kw) for c, W in zip(cases, Ws)]
    for a, b in zip(solo, group):
        sa, sb = lgk.fetch_stats(a), lgk.fetch_stats(b)
        both = sa["converged"] & sb["converged"]
        assert both.mean() >= 0.98, (sa["converged"].sum(), sb["converged"].sum())
        gap = np.abs(sb["obj"] - sa["obj"])[both] / np.maximum(1.0, np.abs(sa["obj"][both]))
        assert gap.max() <= 1e-3, gap.max()
    # the 150-weighting member ran on the same tiles alone: bitwise equal
    np.testing.assert_array_equal(lgk.fetch_stats(group[1])["obj"], lgk.fetch_stats(solo[1])["obj"])
    for r in solo + group:
        r.close()
    for c in cases:
        c.close()


def test_bad_groups_are_refused(lgk):
    cases, Ws = members(lgk)
    kw = dict(w0_bot=W0, tol=1e-4, max_iter=10)
    r0 = [rule(c) for c in cases]
    with pytest.raises(lgk.LgkError) as e:                     # a case twice
        lgk.solve_group([cases[0], cases[0]], [Ws[0], Ws[0]], None, rho0=r0[:2], **kw)
    assert e.value.code == 1
    fp32 = create(lgk, SC.workload_case(0), precision=lgk.PREC_FP32)
    with pytest.raises(lgk.LgkError) as e:                     # the FP32 form
        lgk.solve_group([cases[0], fp32], [Ws[0], Ws[0]], None, rho0=[r0[0], 1100.0 * fp32.beta], **kw)
    assert e.value.code == 1
    refined = create(lgk, SC.workload_case(0), solve_refine=1)
    with pytest.raises(lgk.LgkError) as e:                     # mixed iteration forms
        lgk.solve_group([cases[1], refined], [Ws[1], Ws[0]], None, rho0=[r0[1], 1100.0 * refined.beta], **kw)
    assert e.value.code == 1
    with pytest.raises(lgk.LgkError) as e:                     # more than four
        lgk.solve_group(cases + cases[:2], Ws + Ws[:2], None, rho0=r0 + r0[:2], **kw)
    assert e.value.code == 1
    for c in cases + [fp32, refined]:
        c.close()
