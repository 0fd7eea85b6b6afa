"""Pins of R10's Lanczos start vector on the operators the all-ones vector
fails on: a regularised path-graph Laplacian Q = L + 0.01 I (the all-ones
vector is its eigenvector of the smallest eigenvalue) and a difference-
constraint A whose rows sum to zero (the all-ones vector spans part of A's
null space).  Norms against dense eigen-solves; a difference-constraint LP
solved to HiGHS's optimum; the all-ones start planted back is caught."""
import os
import sys
import types

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import qpgen
from oracle import rapdhg as R
from oracle.warmstart import _mix64

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "rapdhg.py")


def laplacian_qp(n=50, shift=0.01):
    """min 1/2 x'(L + shift I)x + c'x on a box, L the path graph's Laplacian."""
    main = np.full(n, 2.0)
    main[[0, -1]] = 1.0
    L = sp.diags([main + shift, -np.ones(n - 1), -np.ones(n - 1)], [0, 1, -1], format="csr")
    rng = np.random.default_rng(71)
    return qpgen.QPInstance("laplacian", n, 0, 0, sp.csr_matrix(L), sp.csr_matrix((0, n)),
                            rng.standard_normal(n), np.zeros(0), -np.ones(n), np.ones(n))


def difference_lp(n=30, m=40):
    """min c'x s.t. x_i - x_j >= d_k (rows summing to zero), 0 <= x <= 10."""
    rng = np.random.default_rng(72)
    pairs = [tuple(rng.choice(n, 2, replace=False)) for _ in range(m)]
    rows = np.repeat(np.arange(m), 2)
    cols = np.array([c for p in pairs for c in p])
    vals = np.tile([1.0, -1.0], m)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    A.sum_duplicates()
    A.sort_indices()
    b = rng.uniform(-3.0, 1.0, m)
    c = rng.uniform(0.5, 2.0, n)
    return qpgen.QPInstance("difference_lp", n, m, 0, sp.csr_matrix((n, n)), A, c, b, np.zeros(n),
                            np.full(n, 10.0))


def test_start_vector_is_splitmix_signs():
    for dim in (1, 7, 1000):
        v = R.lanczos_start(dim)
        want = np.array([-1.0 if _mix64(j) >> 63 else 1.0 for j in range(dim)]) / np.sqrt(dim)
        np.testing.assert_array_equal(v, want)
        assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-15)


def test_laplacian_norm_against_dense():
    inst = laplacian_qp()
    p = R.problem_from_instance(inst)
    assert np.allclose(p.Q @ np.ones(p.n), 0.01)          # all-ones: the smallest eigenvalue's vector
    dense = np.linalg.eigvalsh(p.Q.toarray())[-1]
    assert R.norm_Q(p) == pytest.approx(dense, rel=1e-6)


def test_zero_row_sum_norm_against_dense():
    inst = difference_lp()
    p = R.problem_from_instance(inst)
    assert np.abs(p.A @ np.ones(p.n)).max() == 0.0         # all-ones: in A's null space
    dense = np.linalg.svd(p.A.toarray(), compute_uv=False)[0]
    assert R.norm_A(p) == pytest.approx(dense, rel=1e-6)


def test_difference_lp_solves_to_highs_optimum():
    inst = difference_lp()
    res = linprog(inst.c, A_ub=-inst.A.toarray(), b_ub=-inst.b, bounds=[(0, 10)] * inst.n, method="highs")
    assert res.status == 0
    r = R.solve(inst, R.Options())
    assert r.status == "optimal" and r.kkt["rel_kkt"] <= 1e-6
    assert r.kkt["primal_obj"] == pytest.approx(res.fun, rel=1e-5, abs=1e-6)


def test_laplacian_qp_solves():
    inst = laplacian_qp()
    r = R.solve(inst, R.Options())
    assert r.status == "optimal" and r.kkt["rel_kkt"] <= 1e-6


def test_all_ones_start_planted_back_is_caught():
    src = open(ORACLE_SRC).read()
    old = "    v = lanczos_start(dim)\n"
    assert src.count(old) == 1
    mod = types.ModuleType("oracle_allones_mutant")
    sys.modules[mod.__name__] = mod
    exec(compile(src.replace(old, "    v = np.full(dim, 1.0 / math.sqrt(dim))\n"), mod.__name__, "exec"),
         mod.__dict__)
    p = mod.problem_from_instance(laplacian_qp())
    dense = np.linalg.eigvalsh(p.Q.toarray())[-1]
    assert mod.norm_Q(p) != pytest.approx(dense, rel=1e-6)
