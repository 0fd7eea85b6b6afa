"""The Lasso, Huber and SVM instances as the oracle solves them, against
answers that do not come from the oracle (CPU):

- Lasso with orthonormal design columns: x* = soft(D'd, lam) coordinatewise
  (1/2 |Dx - d|^2 = 1/2 |x - D'd|^2 + const when D'D = I);
- Huber with M above every residual is least squares; with a small M, the
  minimiser of the Huber loss found by an independent quasi-Newton method;
- SVM: the optimality conditions of the hinge-loss problem checked directly
  at the oracle's x (subgradient zero with multipliers in [0, lam]).
The QP rewriting itself is checked too: the QP objective at the solution
equals the class's own loss."""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R

TIGHT = R.Options(eps=1e-9, max_iter=200_000)


def soft(g, lam):
    return np.sign(g) * np.maximum(np.abs(g) - lam, 0.0)


def huber_loss(r, M):
    a = np.abs(r)
    return float(np.sum(np.where(a <= M, r * r, 2.0 * M * a - M * M)))


def test_lasso_with_orthonormal_columns_is_soft_thresholding():
    rng = np.random.default_rng(5)
    m, n = 30, 20
    Qm, _ = np.linalg.qr(rng.standard_normal((m, m)))
    D = sp.csr_matrix(Qm[:, :n])
    d = rng.standard_normal(m)
    lam = 0.5
    inst = qpgen.lasso_qp(D=D, d=d, lam=lam)
    res = R.solve(inst, TIGHT)
    assert res.status == "optimal"
    x, r, t = res.x[:n], res.x[n:n + m], res.x[n + m:]
    np.testing.assert_allclose(x, soft(D.T @ d, lam), atol=1e-6)
    np.testing.assert_allclose(r, D @ x - d, atol=1e-6)
    np.testing.assert_allclose(t, np.abs(x), atol=1e-6)
    # the QP objective is the Lasso objective
    obj = R.kkt_parts(R.problem_from_instance(inst), res.x, res.y)["primal_obj"]
    assert obj == pytest.approx(0.5 * np.sum((D @ x - d) ** 2) + lam * np.abs(x).sum(), rel=1e-6)


def test_huber_with_large_threshold_is_least_squares():
    rng = np.random.default_rng(6)
    m, n = 40, 8
    D = sp.csr_matrix(rng.standard_normal((m, n)))
    d = rng.standard_normal(m)
    inst = qpgen.huber_qp(D=D, d=d, M=1e3)
    res = R.solve(inst, TIGHT)
    assert res.status == "optimal"
    x_ls = np.linalg.lstsq(D.toarray(), d, rcond=None)[0]
    np.testing.assert_allclose(res.x[:n], x_ls, atol=1e-6)


def test_huber_matches_an_independent_minimiser_of_the_loss():
    inst = qpgen.huber_qp(n=10, m=60, density=0.5, M=0.5)
    n, m = 10, 60
    D = inst.A[:, :n].toarray()
    d = inst.b
    res = R.solve(inst, TIGHT)
    assert res.status == "optimal"
    f = lambda x: huber_loss(D @ x - d, 0.5)
    g = lambda x: D.T @ np.where(np.abs(D @ x - d) <= 0.5, 2.0 * (D @ x - d), 2.0 * 0.5 * np.sign(D @ x - d))
    ref = so.minimize(f, np.zeros(n), jac=g, method="BFGS", options={"gtol": 1e-12, "maxiter": 10000})
    assert f(res.x[:n]) == pytest.approx(ref.fun, rel=1e-7)
    np.testing.assert_allclose(res.x[:n], ref.x, atol=1e-5)
    # the QP objective is the Huber loss
    obj = R.kkt_parts(R.problem_from_instance(inst), res.x, res.y)["primal_obj"]
    assert obj == pytest.approx(f(res.x[:n]), rel=1e-6)


def test_svm_solution_satisfies_the_hinge_optimality_conditions():
    inst = qpgen.svm_qp(n=6, m=40, density=1.0, lam=0.7)
    n, m, lam = 6, 40, 0.7
    res = R.solve(inst, TIGHT)
    assert res.status == "optimal"
    x = res.x[:n]
    SD = inst.A[:, :n].toarray()             # rows s_i D_i
    margin = 1.0 - SD @ x
    # 2x = sum_i a_i s_i D_i with a_i = lam (margin > 0), 0 (margin < 0), in [0, lam] (margin = 0)
    free = np.abs(margin) <= 1e-6
    a = np.where(margin > 1e-6, lam, 0.0)
    rhs = 2.0 * x - SD.T @ a
    if free.any():
        af, *_ = np.linalg.lstsq(SD[free].T, rhs, rcond=None)
        assert np.all(af >= -1e-5) and np.all(af <= lam + 1e-5)
        rhs = rhs - SD[free].T @ af
    assert np.abs(rhs).max() <= 1e-5
    # the QP objective is the SVM objective
    obj = R.kkt_parts(R.problem_from_instance(inst), res.x, res.y)["primal_obj"]
    assert obj == pytest.approx(x @ x + lam * np.maximum(margin, 0.0).sum(), rel=1e-6)


@pytest.mark.parametrize("gen", [qpgen.lasso_qp, qpgen.huber_qp, qpgen.svm_qp])
def test_generators_are_seeded_and_well_formed(gen):
    a, b = gen(seed=qpgen.SEED_BASE + 40), gen(seed=qpgen.SEED_BASE + 40)
    assert (a.A != b.A).nnz == 0 and np.array_equal(a.b, b.b)
    assert a.A.shape == (a.m, a.n) and a.Q.shape == (a.n, a.n)
    assert (a.Q != a.Q.T).nnz == 0
    assert np.all(a.l <= a.u)
