"""A saddle point of L(x, y) is a fixed point of Algorithm 1 for any step
sizes: started there (x = x_prev = x_bar = x*, y = y_bar = y*), every
iterate stays there.  Pinned on three exact solutions -- an LP solved by
hand (with an inactive row, whose zero dual the projection must keep, and a
variable held at its bound by a positive reduced cost), an equality QP from
its KKT linear system, and a diagonal box QP's closed form -- with and
without the Section 5 scaling.  Sign and dropped-term mistakes of the
iteration break it."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R
from tests.test_oracle_mutations import _load


def _lp():
    """min -x1 - x2 + x3 s.t. x1 + 2 x2 <= 4, 3 x1 + x2 <= 6, x1 + x2 >= 1/2,
    x >= 0, x3 <= 5.  Rows 1-2 are active at x* = (8/5, 6/5, 0) with duals
    y = (2/5, 1/5) from c = A'y on (x1, x2); row 3 is inactive (x1 + x2 = 14/5),
    its dual 0; x3 sits at 0 with reduced cost 1."""
    A = sp.csr_matrix(np.array([[-1.0, -2.0, 0.0], [-3.0, -1.0, 0.0], [1.0, 1.0, 0.0]]))
    p = R.Problem(sp.csr_matrix((3, 3)), A, np.array([-1.0, -1.0, 1.0]), np.array([-4.0, -6.0, 0.5]),
                  np.zeros(3), np.array([np.inf, np.inf, 5.0]), 0)
    return p, np.array([8 / 5, 6 / 5, 0.0]), np.array([2 / 5, 1 / 5, 0.0])


def _equality_qp():
    inst = qpgen.tiny_qp(11, n=8, m=3, m_eq=3, bounds="free")
    Q, A = inst.Q.toarray(), inst.A.toarray()
    K = np.block([[Q, -A.T], [A, np.zeros((3, 3))]])
    sol = np.linalg.solve(K, np.concatenate([-inst.c, inst.b]))
    return R.problem_from_instance(inst), sol[:8], sol[8:]


def _box_qp():
    inst = qpgen.diagonal_box_qp(31, 12)
    return R.problem_from_instance(inst), np.clip(-inst.c / inst.Q.diagonal(), inst.l, inst.u), np.zeros(0)


CASES = {"lp": _lp, "equality_qp": _equality_qp, "box_qp": _box_qp}


def _stays(R_, p, xs, ys, scaling):
    res = R_.solve(p, R_.Options(max_iter=40, eps=0.0, check_period=8, scaling=scaling), x0=xs, y0=ys,
                   trace_at=range(1, 41))
    worst = 0.0
    for st in res.trace.values():
        for k, ref in (("x", xs), ("xbar", xs), ("y", ys), ("ybar", ys)):
            if ref.size:
                worst = max(worst, float(np.max(np.abs(st[k] - ref) / (1 + np.abs(ref)))))
    return worst


@pytest.mark.parametrize("scaling", [False, True], ids=["unscaled", "scaled"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_saddle_point_is_a_fixed_point(name, scaling):
    p, xs, ys = CASES[name]()
    kkt = R.kkt_parts(p, xs, ys)
    assert kkt["rel_kkt"] <= 1e-13          # the point is a KKT point
    assert _stays(R, p, xs, ys, scaling) <= 1e-13


@pytest.mark.parametrize("mutation", ["dual_sign", "drop_ATy", "xmd_from_x", "no_dual_projection"])
def test_iteration_mistakes_break_the_fixed_point(mutation):
    """dual_sign pushes the inactive row's dual up, drop_ATy leaves the
    primal step without A'y, no_dual_projection lets the inactive row's dual
    go negative; xmd_from_x is invisible here (x_md = x at a fixed point), so
    it must pass -- the pin separates what it can see from what it cannot."""
    M = _load(mutation)
    p, xs, ys = _lp()
    pm = M.Problem(p.Q, p.A, p.c, p.b, p.l, p.u, p.m_eq)
    moved = _stays(M, pm, xs, ys, False)
    if mutation == "xmd_from_x":
        assert moved <= 1e-13
    else:
        assert moved > 1e-6
