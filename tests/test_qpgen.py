"""The seeded generators against the recipes they state: shapes, symmetric
positive (semi)definite Q, the stated nonzero structure, bounds, and
feasibility (HiGHS on the rows and the box, or the generator's own
certificate); the same seed gives the same instance."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import qpgen


def _feasible(inst):
    """HiGHS feasibility of the rows and the box (zero objective)."""
    A, b = inst.A.toarray(), inst.b
    kw = dict(bounds=list(zip(np.where(np.isfinite(inst.l), inst.l, None),
                              np.where(np.isfinite(inst.u), inst.u, None))), method="highs")
    if inst.m_eq:
        kw.update(A_eq=A[:inst.m_eq], b_eq=b[:inst.m_eq])
    if inst.m > inst.m_eq:
        kw.update(A_ub=-A[inst.m_eq:], b_ub=-b[inst.m_eq:])
    return linprog(np.zeros(inst.n), **kw).status == 0


def _symmetric(Q):
    return abs(Q - Q.T).max() == 0


def test_random_sparse_qp_recipe():
    inst = qpgen.random_sparse_qp()
    assert (inst.n, inst.m, inst.m_eq) == (1000, 500, 250)
    assert _symmetric(inst.Q)
    assert np.linalg.eigvalsh(inst.Q.toarray())[0] >= 0.01 - 1e-9      # B'B + 0.01 I
    assert np.all(np.diff(inst.A.indptr) >= 1)                             # no empty row
    assert np.all(inst.l == -10) and np.all(inst.u == 10)
    assert 0.005 < inst.A.nnz / (inst.n * inst.m) < 0.015
    assert _feasible(inst)


def test_large_sparse_qp_recipe_at_reduced_size():
    inst = qpgen.large_sparse_qp(n=20_000)
    assert (inst.n, inst.m, inst.m_eq) == (20_000, 10_000, 5_000)
    per_col = np.diff(inst.A.tocsc().indptr)
    assert np.all(per_col == 10)                                           # 10 distinct rows per column
    Q = inst.Q.tocsr()
    assert _symmetric(Q)
    d = Q.diagonal()
    off = np.asarray(abs(Q).sum(axis=1)).ravel() - np.abs(d)
    assert np.all(d - off >= 0.1 - 1e-12)                                  # diagonally dominant by U(0.1, 10)
    assert 4.0 <= (Q.nnz - inst.n) / inst.n <= 5.0                         # ~5 off-diagonal entries per row
    assert np.all(inst.l == -10) and np.all(inst.u == 10)


def test_portfolio_qp_recipe_and_certificate():
    inst = qpgen.portfolio_qp(n=2_000, r=16)
    assert (inst.n, inst.m, inst.m_eq) == (2_000, 2, 1) and inst.F.shape == (2_000, 16)
    assert inst.F.dtype == np.float32 and np.all(inst.c == 0)
    mu = inst.A.toarray()[1]
    x = np.zeros(inst.n)
    x[np.argsort(mu)[-20:]] = 0.05                                         # the stated certificate
    assert abs(x.sum() - 1.0) < 1e-12 and mu @ x >= 0.05
    assert np.all(x >= inst.l) and np.all(x <= inst.u)


@pytest.mark.parametrize("i", range(4))
def test_mpc_qp_recipe(i):
    inst = qpgen.mpc_batch(4, seed=qpgen.SEED_BASE + 3)[i]
    T = (inst.n - 12) // 16
    assert inst.n == 12 * (T + 1) + 4 * T and inst.m == inst.m_eq == 12 * (T + 1) and 10 <= T <= 100
    assert sp.issparse(inst.Q) and inst.Q.nnz == inst.n and np.all(inst.Q.diagonal() >= 0.1)
    assert np.all(inst.c == 0)
    assert np.allclose(np.abs(inst.l[:12 * (T + 1)]), 5) and np.allclose(np.abs(inst.l[12 * (T + 1):]), 1)
    assert _feasible(inst)


def test_family_members_share_structure():
    fam = qpgen.family_qp(n=2_000, m=1_000)
    C, B = fam.params(0, 3)
    assert C.shape == (3, 2_000) and B.shape == (3, 1_000)
    C2, _ = fam.params(0, 3)
    np.testing.assert_array_equal(C, C2)
    assert _symmetric(fam.base.Q) and np.linalg.eigvalsh(fam.base.Q.toarray())[0] >= 0.01 - 1e-9


def test_seeds_reproduce():
    a, b = qpgen.random_sparse_qp(seed=5), qpgen.random_sparse_qp(seed=5)
    np.testing.assert_array_equal(a.A.toarray(), b.A.toarray())
    np.testing.assert_array_equal(a.b, b.b)
    c = qpgen.random_sparse_qp(seed=6)
    assert not np.array_equal(a.c, c.c)


def _sectors_per_warp(insts):
    """Distinct 32-byte sectors of float32 values touched by each 32 consecutive
    nonzeros of P = [Q | A'] (what one warp of the primal kernel's staging loop
    gathers), averaged."""
    Q = sp.block_diag([i.Q for i in insts], format="csr")
    A = sp.block_diag([i.A for i in insts], format="csr")
    P = sp.hstack([Q, sp.csr_matrix(A.T)], format="csr")
    P.sort_indices()
    col = P.indices.astype(np.int64)
    g = np.sort((col[:col.size - col.size % 32] * 4 // 32).reshape(-1, 32), axis=1)
    return float((1 + (np.diff(g, axis=1) != 0).sum(axis=1)).mean())


def test_gather_locality_of_the_workloads():
    """The random large sparse QP gathers from a new sector for almost every
    nonzero (the kernels' L2 sector bound); the control QPs' banded structure
    coalesces about 8 nonzeros per sector."""
    assert _sectors_per_warp([qpgen.large_sparse_qp(n=100_000)]) > 30.0
    assert _sectors_per_warp(qpgen.mpc_batch(64, seed=qpgen.SEED_BASE + 3)) < 5.0
