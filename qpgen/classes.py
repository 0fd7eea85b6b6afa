"""Seeded instances of three more convex-QP classes, each written as a QP of
the form in qpgen.instances from its textbook formulation:

- lasso_qp:  l1-penalised least squares,   min 1/2 |D x - d|^2 + lam |x|_1
- huber_qp:  Huber fitting,                 min sum_i h_M(D_i x - d_i)
- svm_qp:    soft-margin linear SVM,        min |x|^2 + lam sum_i max(0, 1 - s_i D_i x)

The paper's Section 6.3 draws such classes from another benchmark's
generators, which are not available; the recipes here are this module's own
and are stated per generator.  Each generator also accepts explicit data
(D, d, labels) so that tests can pass special cases with known answers.
Data only: nothing here computes a solution.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import scipy.sparse as sp

from .instances import SEED_BASE, QPInstance, _canon


def _design(rng, rows: int, cols: int, density: float) -> sp.csr_matrix:
    """rows x cols, each entry nonzero with probability `density`, N(0,1) values;
    an empty row gets one entry in a uniform column."""
    M = sp.random(rows, cols, density=density, format="lil", random_state=rng,
                  data_rvs=lambda k: rng.standard_normal(k))
    for i in range(rows):
        if not M.rows[i]:
            M[i, int(rng.integers(cols))] = rng.standard_normal()
    return sp.csr_matrix(M)


def lasso_qp(seed: int = SEED_BASE + 11, n: int = 200, m: int = 100, density: float = 0.15,
             lam: Optional[float] = None, D: Optional[sp.spmatrix] = None,
             d: Optional[np.ndarray] = None) -> QPInstance:
    """min 1/2 |D x - d|^2 + lam |x|_1 with x in R^n, D m x n.

    QP variables z = (x [n], r [m], t [n]):
        D x - r = d                 (m equalities; r is the residual)
        t - x >= 0,  t + x >= 0     (2n inequalities; t >= |x|)
        objective 1/2 r'r + lam 1't:  Q = diag(0, I_m, 0), c = (0, 0, lam 1)
        x, r free, t >= 0.
    Recipe (unless D, d are given): D ~ Bernoulli(density) N(0,1); x_true with
    each entry 0 with probability 1/2, else N(0, 1/n); d = D x_true + N(0, 0.01^2);
    lam = |D'd|_inf / 4 unless given."""
    rng = np.random.default_rng(seed)
    if D is None:
        D = _design(rng, m, n, density)
        x_true = np.where(rng.random(n) < 0.5, 0.0, rng.normal(0.0, 1.0 / np.sqrt(n), n))
        d = D @ x_true + rng.normal(0.0, 0.01, m)
    D = sp.csr_matrix(D, dtype=np.float64)
    m, n = D.shape
    d = np.asarray(d, dtype=np.float64)
    if lam is None:
        lam = float(np.abs(D.T @ d).max()) / 4.0
    I_n, I_m = sp.identity(n, format="csr"), sp.identity(m, format="csr")
    Z_mn = sp.csr_matrix((m, n))
    A = sp.bmat([[D, -I_m, Z_mn],
                 [-I_n, None, I_n],
                 [I_n, None, I_n]], format="csr")
    N = 2 * n + m
    A = _canon(A, (m + 2 * n, N))
    Q = _canon(sp.block_diag([sp.csr_matrix((n, n)), I_m, sp.csr_matrix((n, n))]), (N, N))
    c = np.concatenate([np.zeros(n + m), np.full(n, lam)])
    b = np.concatenate([d, np.zeros(2 * n)])
    l = np.concatenate([np.full(n + m, -np.inf), np.zeros(n)])
    u = np.full(N, np.inf)
    return QPInstance("lasso_qp", N, m + 2 * n, m, Q, A, c, b, l, u)


def huber_qp(seed: int = SEED_BASE + 12, n: int = 100, m: int = 500, density: float = 0.15, M: float = 1.0,
             D: Optional[sp.spmatrix] = None, d: Optional[np.ndarray] = None) -> QPInstance:
    """min sum_i h_M(D_i x - d_i), h_M(r) = r^2 for |r| <= M, else 2M|r| - M^2.

    h_M(r) is the least w^2 + 2M|s| over r = w + s, so with s = s+ - s- the QP
    in z = (x [n], w [m], s+ [m], s- [m]) is
        D x - w - s+ + s- = d          (m equalities)
        objective w'w + 2M 1'(s+ + s-):  Q = diag(0, 2 I_m, 0, 0), c = (0, 0, 2M 1, 2M 1)
        x, w free, s+, s- >= 0.
    Recipe (unless D, d are given): D ~ Bernoulli(density) N(0,1); x_true ~
    N(0, 1/n); d = D x_true + noise, the noise N(0, 0.1^2) on 95% of the rows and
    N(0, 10^2) (outliers) on the others."""
    rng = np.random.default_rng(seed)
    if D is None:
        D = _design(rng, m, n, density)
        x_true = rng.normal(0.0, 1.0 / np.sqrt(n), n)
        out = rng.random(m) < 0.05
        d = D @ x_true + np.where(out, rng.normal(0.0, 10.0, m), rng.normal(0.0, 0.1, m))
    D = sp.csr_matrix(D, dtype=np.float64)
    m, n = D.shape
    d = np.asarray(d, dtype=np.float64)
    I_m = sp.identity(m, format="csr")
    A = _canon(sp.hstack([D, -I_m, -I_m, I_m]), (m, n + 3 * m))
    N = n + 3 * m
    Q = _canon(sp.block_diag([sp.csr_matrix((n, n)), 2.0 * I_m, sp.csr_matrix((2 * m, 2 * m))]), (N, N))
    c = np.concatenate([np.zeros(n + m), np.full(2 * m, 2.0 * M)])
    l = np.concatenate([np.full(n + m, -np.inf), np.zeros(2 * m)])
    u = np.full(N, np.inf)
    return QPInstance("huber_qp", N, m, m, Q, A, c, d.copy(), l, u)


def svm_qp(seed: int = SEED_BASE + 13, n: int = 50, m: int = 200, density: float = 0.3,
           lam: Optional[float] = None, D: Optional[sp.spmatrix] = None,
           labels: Optional[np.ndarray] = None) -> QPInstance:
    """min |x|^2 + lam sum_i max(0, 1 - s_i D_i x), labels s_i in {-1, +1}
    (linear soft-margin SVM through the origin).

    QP variables z = (x [n], t [m]):
        t_i + s_i D_i x >= 1        (m inequalities; with t >= 0, t_i >= the hinge)
        objective x'x + lam 1't:  Q = diag(2 I_n, 0), c = (0, lam 1)
        x free, t >= 0.
    Recipe (unless D, labels are given): the first m/2 points have label +1 and
    features Bernoulli(density) N(+1/n, 1/n), the others label -1 and
    N(-1/n, 1/n) on the same pattern law; lam = 1 unless given."""
    rng = np.random.default_rng(seed)
    if D is None:
        labels = np.where(np.arange(m) < m // 2, 1.0, -1.0)
        mask = _design(rng, m, n, density)
        mask.data[:] = 1.0
        vals = rng.normal(0.0, 1.0 / np.sqrt(n), (m, n)) + labels[:, None] / n
        D = sp.csr_matrix(mask.multiply(vals))
    D = sp.csr_matrix(D, dtype=np.float64)
    m, n = D.shape
    labels = np.asarray(labels, dtype=np.float64)
    lam = 1.0 if lam is None else lam
    A = _canon(sp.hstack([sp.diags(labels) @ D, sp.identity(m, format="csr")]), (m, n + m))
    N = n + m
    Q = _canon(sp.block_diag([2.0 * sp.identity(n, format="csr"), sp.csr_matrix((m, m))]), (N, N))
    c = np.concatenate([np.zeros(n), np.full(m, lam)])
    b = np.ones(m)
    l = np.concatenate([np.full(n, -np.inf), np.zeros(m)])
    u = np.full(N, np.inf)
    return QPInstance("svm_qp", N, m, 0, Q, A, c, b, l, u)
