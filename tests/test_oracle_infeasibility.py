"""Pins of the oracle's infeasibility certificates (optional, not in the paper).

Each infeasible instance is classified independently by scipy's HiGHS linear
programming solver (status 2: infeasible, 3: unbounded) or, for a QP, by hand;
each returned certificate is checked against its defining inequalities with
the box's support function taken by brute force over the box's vertices (and
its limits where a bound is infinite).  Feasible problems solve to the same
iterates with detection on as with it off.  Planted mistakes in the
certificate tests are caught."""
import itertools
import os
import sys
import types

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import qpgen
from oracle import rapdhg as R

INF = np.inf
ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "rapdhg.py")


def _inst(Q, A, c, b, l, u, m_eq):
    n = len(c)
    A = np.asarray(A, float).reshape(-1, n)
    return qpgen.QPInstance("hand", n, A.shape[0], m_eq, sp.csr_matrix(np.asarray(Q, float)), sp.csr_matrix(A),
                            np.asarray(c, float), np.asarray(b, float), np.asarray(l, float), np.asarray(u, float))


# primal infeasible (no x satisfies the rows and the box)
BOX_LP = _inst(np.zeros((2, 2)), [[1, 1]], [1, 1], [3], [0, 0], [1, 1], 0)                 # x1 + x2 >= 3 in [0,1]^2
EQ_FREE = _inst(np.eye(2), [[1, 1], [1, 1]], [0, 0], [1, 2], [-INF, -INF], [INF, INF], 2)   # x1+x2 = 1 and = 2
EQ_BOX = _inst(np.eye(2), [[1, 1], [1, 1]], [0, 0], [1, 2], [-5, -5], [5, 5], 2)
MIXED = _inst(np.diag([1, 0, 2]), [[1, 1, 0], [-1, -1, 0], [0, 1, 1]], [1, -1, 0], [2, -1, 0],
              [0, -INF, -1], [INF, INF, 1], 0)                                                 # x1+x2 >= 2 and <= 1
# dual infeasible (objective unbounded below)
RAY_NO_ROWS = _inst(np.diag([1, 0]), np.zeros((0, 2)), [0, -1], [], [-INF, 0], [INF, INF], 0)
RAY_LP = _inst(np.zeros((2, 2)), [[1, -2]], [-1, -1], [-1], [0, 0], [INF, INF], 0)
RAY_BOXED = _inst(np.diag([0, 1]), np.zeros((0, 2)), [-1, -1], [], [0, 0], [INF, 1], 0)   # x2 moves to its bound
EQ_SCALED = _inst(np.eye(2), [[1, 1], [10, 10]], [0, 0], [1, 20], [-INF, -INF], [INF, INF], 2)   # rows of unequal scale
PRIMAL_INFEASIBLE = {"box_lp": BOX_LP, "eq_free": EQ_FREE, "eq_box": EQ_BOX, "mixed": MIXED, "eq_scaled": EQ_SCALED}
DUAL_INFEASIBLE = {"ray_no_rows": RAY_NO_ROWS, "ray_lp": RAY_LP, "ray_boxed": RAY_BOXED}


def _support(g, l, u):
    """sup over the box of g'x by brute force: the maximum over the box's
    vertices, +inf when g pushes towards an infinite bound."""
    if np.any((g > 0) & ~np.isfinite(u)) or np.any((g < 0) & ~np.isfinite(l)):
        return INF
    lo = np.where(np.isfinite(l), l, 0.0)
    hi = np.where(np.isfinite(u), u, 0.0)
    return max(float(g @ np.array(v)) for v in itertools.product(*zip(lo, hi)))


def _check_farkas(inst, y):
    """y proves primal infeasibility: y_I >= 0 and b'y - sup_box (A'y)'x = 1
    (to rounding), the support finite up to eps in A'y."""
    assert np.all(y[inst.m_eq:] >= 0)
    g = inst.A.T @ y
    # components of A'y that push towards an infinite bound must vanish (eps)
    lo_inf, up_inf = ~np.isfinite(inst.l), ~np.isfinite(inst.u)
    leak = np.concatenate([g[up_inf & (g > 0)], -g[lo_inf & (g < 0)]])
    assert leak.size == 0 or leak.max() <= 1e-8
    g_clean = np.where((up_inf & (g > 0)) | (lo_inf & (g < 0)), 0.0, g)
    assert float(inst.b @ y) - _support(g_clean, inst.l, inst.u) == pytest.approx(1.0, abs=1e-9)


def _check_ray(inst, d):
    """d proves unboundedness: in the box's recession cone, c'd = -1, Qd = 0,
    A_E d = 0, A_I d >= 0 (to 1e-8)."""
    assert np.all(d[np.isfinite(inst.l) & np.isfinite(inst.u)] == 0)
    assert np.all(d[np.isfinite(inst.l)] >= 0) and np.all(d[np.isfinite(inst.u)] <= 0)
    assert float(inst.c @ d) == pytest.approx(-1.0, abs=1e-12)
    assert np.abs(inst.Q @ d).max() <= 1e-8
    Ad = inst.A @ d
    assert np.all(np.abs(Ad[:inst.m_eq]) <= 1e-8) and np.all(Ad[inst.m_eq:] >= -1e-8)


def _linprog_status(inst):
    """HiGHS on the LP with the same rows and box (objective c; feasibility
    does not depend on it)."""
    A, b = inst.A.toarray(), inst.b
    kw = dict(bounds=list(zip(np.where(np.isfinite(inst.l), inst.l, None),
                              np.where(np.isfinite(inst.u), inst.u, None))), method="highs")
    if inst.m_eq:
        kw.update(A_eq=A[:inst.m_eq], b_eq=b[:inst.m_eq])
    if inst.m > inst.m_eq:
        kw.update(A_ub=-A[inst.m_eq:], b_ub=-b[inst.m_eq:])
    return linprog(inst.c, **kw).status


def _solve(R_, inst, **kw):
    return R_.solve(inst, R_.Options(detect_infeasibility=True, max_iter=5000, **kw))


@pytest.mark.parametrize("name", sorted(PRIMAL_INFEASIBLE))
def test_primal_infeasible_certificates(name):
    inst = PRIMAL_INFEASIBLE[name]
    assert _linprog_status(inst) == 2
    r = _solve(R, inst)
    assert r.status == "primal_infeasible"
    assert np.all(r.x == 0)
    _check_farkas(inst, r.y)


def test_box_lp_certificate_is_exact():
    """x1 + x2 >= 3 on [0,1]^2: b'y - sup(A'y)'x = 3y - 2y, so the normalised
    certificate is y = 1, found at the first check."""
    r = _solve(R, BOX_LP)
    assert r.iterations == 64
    assert r.y == pytest.approx([1.0], abs=1e-12)


@pytest.mark.parametrize("name", sorted(DUAL_INFEASIBLE))
def test_dual_infeasible_certificates(name):
    inst = DUAL_INFEASIBLE[name]
    if not np.any(inst.Q.diagonal()):
        assert _linprog_status(inst) == 3
    r = _solve(R, inst)
    assert r.status == "dual_infeasible"
    assert np.all(r.y == 0)
    _check_ray(inst, r.x)


def test_ray_without_rows_is_exact():
    """x1 stays at its minimiser 0 and x2 grows with nothing to stop it: the
    ray is (0, 1) exactly."""
    r = _solve(R, RAY_NO_ROWS)
    assert r.iterations == 64
    np.testing.assert_array_equal(r.x, [0.0, 1.0])


FEASIBLE = [
    qpgen.tiny_qp(5, n=12, m=8, m_eq=3, bounds="mixed", density=0.6),
    qpgen.tiny_qp(6, n=9, m=5, m_eq=0, bounds="free"),
    _inst(np.diag([1, 1]), np.zeros((0, 2)), [0, -1], [], [0, 0], [INF, INF], 0),     # bounded along c
    _inst(np.zeros((2, 2)), [[-1, -2], [-3, -1]], [-1, -1], [-4, -6], [0, 0], [INF, INF], 0),   # LP vertex (1.6, 1.2)
]


@pytest.mark.parametrize("k", range(len(FEASIBLE)))
def test_detection_leaves_feasible_solves_alone(k):
    inst = FEASIBLE[k]
    a = R.solve(inst, R.Options())
    b = _solve(R, inst, **{})
    assert a.status == b.status == "optimal"
    assert a.iterations == b.iterations
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.y, b.y)


@pytest.mark.parametrize("s", [1e-6, 1.0, 1e6])
def test_certificate_tests_are_scale_free(s):
    """A ray has no natural length: both tests are positively homogeneous,
    test(s ray) = s test(ray).  The rays here leave a residual 1e-12 of their
    objective term, far inside eps = 1e-8 relatively but not absolutely once
    scaled by 1e6."""
    free2 = R.Problem(sp.csr_matrix((1, 1)), sp.csr_matrix(np.array([[1.0], [1.0]])), np.zeros(1),
                      np.array([1.0, 2.0]), np.array([-INF]), np.array([INF]), 2)
    rho = np.array([-1.0 + 1e-12, 1.0])                  # A'rho = 1e-12, b'rho = 1 + 1e-12
    v1 = R.dual_ray_value(free2, rho, 1e-8)
    assert v1 == pytest.approx(1.0, rel=1e-11)
    assert R.dual_ray_value(free2, s * rho, 1e-8) == pytest.approx(s * v1, rel=1e-12)
    ray = R.Problem(sp.csr_matrix(np.diag([0.0, 1.0])), sp.csr_matrix((0, 2)), np.array([-1.0, 0.0]),
                    np.zeros(0), np.array([0.0, -INF]), np.array([INF, INF]), 0)
    d = np.array([1.0, 1e-12])                           # Qd = 1e-12, c'd = -1
    w1 = R.primal_ray_value(ray, d, 1e-8)
    assert w1 == 1.0
    assert R.primal_ray_value(ray, s * d, 1e-8) == pytest.approx(s * w1, rel=1e-15)


CLASSES = [qpgen.random_sparse_qp(seed=qpgen.SEED_BASE), *qpgen.mpc_batch(3, seed=qpgen.SEED_BASE + 3),
           qpgen.lasso_qp(), qpgen.huber_qp(), qpgen.svm_qp()]


@pytest.mark.parametrize("k", range(len(CLASSES)), ids=[i.name for i in CLASSES])
def test_no_certificate_on_the_feasible_classes(k):
    """With detection on, the bench's problem classes (random sparse, control,
    Lasso, Huber, SVM) solve exactly as without it: no ray of theirs passes."""
    inst = CLASSES[k]
    a = R.solve(inst, R.Options())
    b = R.solve(inst, R.Options(detect_infeasibility=True))
    assert a.status == b.status == "optimal" and a.iterations == b.iterations
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.y, b.y)


# ---------------------------------------------------------------------------
# planted mistakes in the certificate tests
# ---------------------------------------------------------------------------
MUTATIONS = {
    "farkas_sign": ("value = float(p.b @ rho) + float(", "value = -float(p.b @ rho) + float("),
    "no_Q_test": ("worst = max(_inf_norm(viol), _inf_norm(p.Qmul(d)))", "worst = _inf_norm(viol)"),
    "no_cone_projection": ("d = D2 * recession_project(xs - anchor[0], ps.l, ps.u)", "d = D2 * (xs - anchor[0])"),
    "ineq_rows_two_sided": ("viol[p.m_eq:] = np.maximum(-Ad[p.m_eq:], 0.0)", "pass"),
    "no_unscaling": ("rho = D1 * proj_Y(ys - anchor[1], p.m_eq)", "rho = proj_Y(ys - anchor[1], p.m_eq)"),
    "farkas_residual_absolute": ("return value if (value > 0 and _inf_norm(g - lam) <= eps * value) else 0.0",
                                 "return value if (value > 0 and _inf_norm(g - lam) <= eps) else 0.0"),
    "ray_residual_absolute": ("return -cd if worst <= eps * (-cd) else 0.0", "return -cd if worst <= eps else 0.0"),
}


def _mutant(name):
    src = open(ORACLE_SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle_infeas_mutant_" + name)
    sys.modules[mod.__name__] = mod
    exec(compile(src.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    return mod


def _pins_pass(R_):
    try:
        for inst in PRIMAL_INFEASIBLE.values():
            r = _solve(R_, inst)
            assert r.status == "primal_infeasible"
            _check_farkas(inst, r.y)
        for inst in DUAL_INFEASIBLE.values():
            r = _solve(R_, inst)
            assert r.status == "dual_infeasible"
            _check_ray(inst, r.x)
        for inst in FEASIBLE:
            assert _solve(R_, inst).status == "optimal"
        free2 = R_.Problem(sp.csr_matrix((1, 1)), sp.csr_matrix(np.array([[1.0], [1.0]])), np.zeros(1),
                           np.array([1.0, 2.0]), np.array([-INF]), np.array([INF]), 2)
        rho = np.array([-1.0 + 1e-12, 1.0])
        assert R_.dual_ray_value(free2, 1e6 * rho, 1e-8) > 0
        ray = R_.Problem(sp.csr_matrix(np.diag([0.0, 1.0])), sp.csr_matrix((0, 2)), np.array([-1.0, 0.0]),
                         np.zeros(0), np.array([0.0, -INF]), np.array([INF, INF]), 0)
        assert R_.primal_ray_value(ray, 1e6 * np.array([1.0, 1e-12]), 1e-8) > 0
    except (AssertionError, FloatingPointError, ZeroDivisionError, ValueError):
        return False
    return True


def test_pins_pass_on_the_oracle():
    assert _pins_pass(R)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    assert not _pins_pass(_mutant(name))
