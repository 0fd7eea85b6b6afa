"""Invariants of the oracle that its pins on end states cannot see.

* R10's stop test is relative, so Lanczos is scale-invariant: on c M it takes
  the steps it takes on M and returns c times the value.
* The start point is projected (x onto X, y onto Y) before the first
  iteration: a start outside X or Y gives the iterates of its projection.
* relKKT is measured on the original problem (R6): every check's recorded
  relKKT equals that of the traced iterate, unscaled, on the original data."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R


@pytest.mark.parametrize("c", [1e-4, 1e6])
def test_lanczos_is_scale_invariant(c):
    rng = np.random.default_rng(5)
    B = rng.standard_normal((60, 40))
    M = B.T @ B
    R.lanczos_max_eig(lambda v: M @ v, 40, tol=1e-6, name="M")
    steps, val = R.NORM_STEPS["M"], R.lanczos_max_eig(lambda v: M @ v, 40, tol=1e-6, name="M")
    val_c = R.lanczos_max_eig(lambda v: (c * M) @ v, 40, tol=1e-6, name="cM")
    assert R.NORM_STEPS["cM"] == steps
    assert val_c == pytest.approx(c * val, rel=1e-12)


def test_start_point_is_projected():
    inst = qpgen.tiny_qp(61, n=6, m=4, m_eq=2, bounds="box")
    rng = np.random.default_rng(6)
    x0 = rng.uniform(-30, 30, inst.n)                    # far outside the box
    y0 = rng.uniform(-3, 3, inst.m)                      # inequality entries of both signs
    xp = np.clip(x0, inst.l, inst.u)
    yp = y0.copy()
    yp[inst.m_eq:] = np.maximum(yp[inst.m_eq:], 0.0)
    o = R.Options(max_iter=20, eps=0.0, check_period=8)
    a = R.solve(inst, o, x0=x0, y0=y0, trace_at=range(1, 21))
    b = R.solve(inst, o, x0=xp, y0=yp, trace_at=range(1, 21))
    for t in range(1, 21):
        for key in ("x", "y", "xbar", "ybar"):
            np.testing.assert_array_equal(a.trace[t][key], b.trace[t][key])


def test_checks_measure_the_original_problem():
    inst = qpgen.tiny_qp(62, n=8, m=5, m_eq=2, bounds="mixed")
    p = R.problem_from_instance(inst)
    r = R.solve(inst, R.Options(eps=1e-9, check_period=16), trace_at=range(16, 2000, 16))
    D = r.D1, r.D2
    assert np.max(np.abs(D[0] - 1)) > 1e-3 or np.max(np.abs(D[1] - 1)) > 1e-3     # scaling is active
    for c in r.checks:
        st = r.trace.get(c["total"])
        if st is None:
            continue
        assert c["kkt_cur"] == pytest.approx(R.rel_kkt(p, st["x"], st["y"]), rel=1e-12)
        assert c["kkt_avg"] == pytest.approx(R.rel_kkt(p, st["xbar"], st["ybar"]), rel=1e-12)


def test_iteration_limit_checks_at_max_iter():
    """R7: a check also runs at max_iter when it is not a multiple of the
    check period, and the solve stops there."""
    inst = qpgen.tiny_qp(63, n=6, m=4, m_eq=1, bounds="box")
    r = R.solve(inst, R.Options(max_iter=100, check_period=64, eps=1e-14))
    assert r.status == "iteration_limit" and r.iterations == 100
    assert [c["total"] for c in r.checks] == [64, 100]


def test_termination_is_relkkt_at_most_eps():
    """eq. (terminate) is relKKT <= eps: min 1/2 x^2 + 5x on [0, 10] from x = 1
    reaches its bound x* = 0 exactly (the projection clips), where relKKT is
    exactly 0, so eps = 0 terminates."""
    p = R.Problem(sp.csr_matrix(np.array([[1.0]])), sp.csr_matrix((0, 1)), np.array([5.0]), np.zeros(0),
                  np.array([0.0]), np.array([10.0]), 0)
    r = R.solve(p, R.Options(eps=0.0, max_iter=640, check_period=64, scaling=False), x0=np.array([1.0]))
    assert r.status == "optimal" and r.x[0] == 0.0 and r.kkt["rel_kkt"] == 0.0


def test_certificate_order():
    """R18's order: within the dual-ray tests the current iterate's ray before
    the average's, and dual rays (primal infeasibility) before primal rays.
    Rows x1 >= 3, x2 >= 3 on x1 in [0, 5], x2 in [0, 1], x3 >= 0 (c3 = -1):
    y = (s, t) has Farkas value 3s + 3t - (5s + t) = 2t - 2s, so y = (0, 2) (value
    4) and y = (1, 2) (value 2) both prove infeasibility, in different
    directions; d = (0, 0, 1) is an unbounded direction."""
    p = R.Problem(sp.csr_matrix((3, 3)), sp.csr_matrix(np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])),
                  np.array([0.0, 0.0, -1.0]), np.array([3.0, 3.0]), np.zeros(3), np.array([5.0, 1.0, np.inf]), 0)
    one3, one2, z3, z2 = np.ones(3), np.ones(2), np.zeros(3), np.zeros(2)
    y_cur, y_avg = np.array([0.0, 2.0]), np.array([1.0, 2.0])
    assert R.dual_ray_value(p, y_cur, 1e-8) == 4.0 and R.dual_ray_value(p, y_avg, 1e-8) == 2.0
    st, x, y = R.find_certificate(p, p, one2, one3, ((z3, y_cur), (z3, y_avg)), (z3, z2), 1e-8)
    assert st == "primal_infeasible"
    np.testing.assert_array_equal(y, y_cur / 4.0)
    d_cur = np.array([0.0, 0.0, 1.0])
    assert R.primal_ray_value(p, d_cur, 1e-8) == 1.0
    st, x, y = R.find_certificate(p, p, one2, one3, ((d_cur, z2), (z3, y_cur)), (z3, z2), 1e-8)
    assert st == "primal_infeasible"
    np.testing.assert_array_equal(y, y_cur / 4.0)
