"""Seeded synthetic convex-QP instances.

Every instance has the form

    min 1/2 x'Qx + c'x   s.t.  A[:m_eq] x  = b[:m_eq]
                                A[m_eq:] x >= b[m_eq:]
                                l <= x <= u

which is the inequality-form QP of the paper's eq. (1) extended with
equality rows and variable bounds (the extension its footnote to eq. (1)
allows).  The workloads mirror the shapes of the paper's large synthetic
classes (Section 6.3: random QP, equality QP, portfolio, control), which
are not shipped with the paper; each generator states its recipe.

This module only *builds data*.  It holds none of the solver's arithmetic
and is the one module that both the CPU oracle and the CUDA path consume.
All matrices are CSR (scipy.sparse, int32 indices, float64 values) with
column indices sorted and unique inside every row; Q is stored in full
(both triangles).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

SEED_BASE = 2311077100


@dataclasses.dataclass
class QPInstance:
    name: str
    n: int
    m: int
    m_eq: int
    Q: sp.csr_matrix          # n x n, symmetric PSD, full storage
    A: sp.csr_matrix          # m x n
    c: np.ndarray             # n
    b: np.ndarray             # m
    l: np.ndarray             # n, may hold -inf
    u: np.ndarray             # n, may hold +inf
    # optional low-rank factor: Q_total = Q + F F'  (F row-major n x r, float32)
    F: Optional[np.ndarray] = None

    @property
    def nnz_Q(self) -> int:
        return int(self.Q.nnz)

    @property
    def nnz_A(self) -> int:
        return int(self.A.nnz)


def _canon(M: sp.spmatrix, shape) -> sp.csr_matrix:
    """CSR with int32 indices, summed duplicates, sorted columns, no explicit zeros."""
    M = sp.csr_matrix(M, shape=shape, dtype=np.float64)
    M.sum_duplicates()
    M.eliminate_zeros()
    M.sort_indices()
    M.indptr = M.indptr.astype(np.int32)
    M.indices = M.indices.astype(np.int32)
    return M


def _bernoulli_sparse(rng, rows, cols, p):
    """rows x cols with each entry nonzero w.p. p, values N(0,1).  Dense draw;
    used only for the small instances."""
    mask = rng.random((rows, cols)) < p
    vals = rng.standard_normal((rows, cols))
    return sp.csr_matrix(np.where(mask, vals, 0.0))


def _fixed_per_row(rng, rows, cols, k):
    """rows x cols, exactly k distinct uniform columns per row, values N(0,1)."""
    idx = _distinct_uniform(rng, rows, cols, k)
    r = np.repeat(np.arange(rows, dtype=np.int64), k)
    v = rng.standard_normal(rows * k)
    return sp.coo_matrix((v, (r, idx.ravel())), shape=(rows, cols))


def _distinct_uniform(rng, count, universe, k):
    """count x k array; each row holds k distinct integers drawn uniformly from
    [0, universe).  Collisions are redrawn until none remain."""
    idx = rng.integers(0, universe, size=(count, k), dtype=np.int64)
    while True:
        idx.sort(axis=1)
        dup = np.zeros_like(idx, dtype=bool)
        dup[:, 1:] = idx[:, 1:] == idx[:, :-1]
        nd = int(dup.sum())
        if nd == 0:
            return idx
        idx[dup] = rng.integers(0, universe, size=nd, dtype=np.int64)


def _fill_empty_rows(rng, A: sp.csr_matrix, n: int) -> sp.csr_matrix:
    """Give every empty row one N(0,1) entry at a uniform column."""
    A = A.tocsr()
    lens = np.diff(A.indptr)
    empty = np.nonzero(lens == 0)[0]
    if empty.size == 0:
        return A
    extra = sp.coo_matrix(
        (rng.standard_normal(empty.size), (empty, rng.integers(0, n, empty.size))),
        shape=A.shape)
    return (A + extra).tocsr()


def _feasible_rhs(rng, A: sp.csr_matrix, m_eq: int, lo: float, hi: float, n: int):
    """b built so that x0 ~ U(lo, hi) is feasible: b_E = A_E x0 and
    b_I = A_I x0 - s with slack s ~ U(0,1) (x0 strictly satisfies A_I x >= b_I)."""
    x0 = rng.uniform(lo, hi, n)
    b = A @ x0
    s = rng.uniform(0.0, 1.0, A.shape[0] - m_eq)
    b[m_eq:] -= s
    return b, x0


# --------------------------------------------------------------------------
# Configuration 0: small random sparse QP (n=1000, m=500, half equality rows)
# --------------------------------------------------------------------------
def random_sparse_qp(seed: int = SEED_BASE + 0, n: int = 1000, m: int = 500,
                     density_A: float = 0.01, density_B: float = 0.005,
                     name: str = "random_sparse_qp") -> QPInstance:
    """A ~ Bernoulli(density_A) x N(0,1) (empty rows get one entry);
    Q = B'B + 0.01 I with B n x n ~ Bernoulli(density_B) x N(0,1);
    c ~ N(0,1); l=-10, u=10; m_eq = m/2; b feasible for x0 ~ U(-1,1)."""
    rng = np.random.default_rng(seed)
    m_eq = m // 2
    A = _fill_empty_rows(rng, _bernoulli_sparse(rng, m, n, density_A), n)
    B = _bernoulli_sparse(rng, n, n, density_B)
    Q = (B.T @ B) + 0.01 * sp.identity(n, format="csr")
    c = rng.standard_normal(n)
    b, _ = _feasible_rhs(rng, A, m_eq, -1.0, 1.0, n)
    return QPInstance(name, n, m, m_eq, _canon(Q, (n, n)), _canon(A, (m, n)), c, b,
                      np.full(n, -10.0), np.full(n, 10.0))


# --------------------------------------------------------------------------
# Configuration 1: large sparse QP (n=1e6, m=5e5, half equality rows)
# --------------------------------------------------------------------------
def large_sparse_qp(seed: int = SEED_BASE + 1, n: int = 1_000_000, m: Optional[int] = None,
                    nnz_per_col: int = 10, offdiag_per_row: int = 5,
                    name: str = "large_sparse_qp") -> QPInstance:
    """A: each column holds nnz_per_col distinct uniform rows, N(0,1) values
    (row lengths ~ Poisson(2*nnz_per_col) when m=n/2).  Q = diag U(0.1,10) + S,
    S symmetric with n*offdiag_per_row/2 uniform strictly-upper positions of
    N(0, 0.1^2) values mirrored to the lower triangle, then Q_ii += sum_j |S_ij|
    (diagonally dominant, hence PD).  c ~ N(0,1), l=-10, u=10, m_eq=m/2, b feasible
    for x0 ~ U(-1,1)."""
    rng = np.random.default_rng(seed)
    if m is None:
        m = n // 2
    m_eq = m // 2
    rows = _distinct_uniform(rng, n, m, min(nnz_per_col, m))
    cols = np.repeat(np.arange(n, dtype=np.int64), rows.shape[1])
    A = sp.coo_matrix((rng.standard_normal(rows.size), (rows.ravel(), cols)), shape=(m, n))
    A = _fill_empty_rows(rng, A.tocsr(), n)
    n_off = (n * offdiag_per_row) // 2
    i = rng.integers(0, n, n_off, dtype=np.int64)
    j = rng.integers(0, n, n_off, dtype=np.int64)
    keep = i != j
    i, j = i[keep], j[keep]
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    v = 0.1 * rng.standard_normal(lo.size)
    S = sp.coo_matrix((np.concatenate([v, v]), (np.concatenate([lo, hi]), np.concatenate([hi, lo]))),
                      shape=(n, n)).tocsr()
    S.sum_duplicates()
    dom = np.asarray(abs(S).sum(axis=1)).ravel()
    Q = S + sp.diags(rng.uniform(0.1, 10.0, n) + dom, format="csr")
    c = rng.standard_normal(n)
    b, _ = _feasible_rhs(rng, A, m_eq, -1.0, 1.0, n)
    return QPInstance(name, n, m, m_eq, _canon(Q, (n, n)), _canon(A, (m, n)), c, b,
                      np.full(n, -10.0), np.full(n, 10.0))


# --------------------------------------------------------------------------
# Configuration 2: portfolio QP with a dense low-rank factor
# --------------------------------------------------------------------------
def portfolio_qp(seed: int = SEED_BASE + 2, n: int = 100_000, r: int = 64,
                 name: str = "portfolio_qp") -> QPInstance:
    """Q = diag U(0.01,0.1) + F F', F n x r ~ N(0, 0.05^2) stored float32 (applied
    as F(F'x)); row 0: sum(x) = 1; row 1: mu'x >= 0.05 with mu ~ N(0.05, 0.02^2);
    0 <= x <= 0.05; c = 0.  Feasible: the 20 assets with the largest mu at 0.05."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.01, 0.1, n)
    F = (0.05 * rng.standard_normal((n, r))).astype(np.float32)
    mu = rng.normal(0.05, 0.02, n)
    A = sp.csr_matrix(np.vstack([np.ones(n), mu]))
    b = np.array([1.0, 0.05])
    return QPInstance(name, n, 2, 1, _canon(sp.diags(d), (n, n)), _canon(A, (2, n)),
                      np.zeros(n), b, np.zeros(n), np.full(n, 0.05), F=F)


# --------------------------------------------------------------------------
# Configuration 3: batches of MPC-shaped QPs of uneven horizon
# --------------------------------------------------------------------------
NX, NU = 12, 4


def mpc_qp(seed: int, T: Optional[int] = None, T_range=(10, 100), name: str = "mpc_qp") -> QPInstance:
    """Variables z = (x_0..x_T in R^12, u_0..u_{T-1} in R^4); equality rows
    x_0 = x_init (x_init ~ U(-1,1)) and x_{t+1} - A_d x_t - B_d u_t = 0 with
    A_d = I + N(0, 0.1^2) scaled by 1/max(1, spectral radius), B_d ~ N(0, 0.1^2);
    |u| <= 1, |x| <= 5; Q diagonal U(0.1, 1); c = 0.  Redrawn until the u = 0
    trajectory stays inside |x| <= 5 (a feasibility certificate)."""
    rng = np.random.default_rng(seed)
    if T is None:
        T = int(rng.integers(T_range[0], T_range[1] + 1))
    while True:
        Ad = np.eye(NX) + 0.1 * rng.standard_normal((NX, NX))
        rho = float(np.max(np.abs(np.linalg.eigvals(Ad))))
        Ad /= max(1.0, rho)
        Bd = 0.1 * rng.standard_normal((NX, NU))
        x_init = rng.uniform(-1.0, 1.0, NX)
        xs, ok = x_init.copy(), True
        for _ in range(T):
            xs = Ad @ xs
            if np.max(np.abs(xs)) > 5.0:
                ok = False
                break
        if ok:
            break
    n = NX * (T + 1) + NU * T
    m = NX * (T + 1)
    # rows 0..11: x_0 = x_init; rows 12(t+1)+i: x_{t+1,i} - A_d[i,:] x_t - B_d[i,:] u_t = 0
    t = np.arange(T)[:, None, None]
    i = np.arange(NX)[None, :, None]
    row = NX * (t + 1) + i                                   # T x 12 x 1
    cols = np.concatenate([np.broadcast_to(NX * (t + 1) + i, (T, NX, 1)),
                           np.broadcast_to(NX * t + np.arange(NX)[None, None, :], (T, NX, NX)),
                           np.broadcast_to(NX * (T + 1) + NU * t + np.arange(NU)[None, None, :], (T, NX, NU))],
                          axis=2)
    vals = np.concatenate([np.ones((T, NX, 1)), np.broadcast_to(-Ad[None], (T, NX, NX)),
                           np.broadcast_to(-Bd[None], (T, NX, NU))], axis=2)
    r_ = np.concatenate([np.arange(NX), np.broadcast_to(row, cols.shape).ravel()])
    c_ = np.concatenate([np.arange(NX), cols.ravel()])
    v_ = np.concatenate([np.ones(NX), vals.ravel()])
    A = sp.coo_matrix((v_, (r_, c_)), shape=(m, n))
    b = np.zeros(m)
    b[:NX] = x_init
    q = rng.uniform(0.1, 1.0, n)
    l = np.concatenate([np.full(NX * (T + 1), -5.0), np.full(NU * T, -1.0)])
    return QPInstance(f"{name}_T{T}", n, m, m, _canon(sp.diags(q), (n, n)), _canon(A, (m, n)),
                      np.zeros(n), b, l, -l)


def mpc_batch(count: int = 4096, seed: int = SEED_BASE + 3, T_range=(10, 100)) -> List[QPInstance]:
    return [mpc_qp(seed * 100003 + i, T_range=T_range) for i in range(count)]


# --------------------------------------------------------------------------
# Configuration 4: parameterised family sharing one sparsity pattern
# --------------------------------------------------------------------------
@dataclasses.dataclass
class QPFamily:
    """One fixed (Q, A, l, u) with per-instance c = c_bar + scale*N(0,1),
    b = b_bar + scale*N(0,1)."""
    base: QPInstance
    scale: float
    seed: int

    def params(self, start: int, count: int):
        """(C, B): count x n and count x m perturbed objective / rhs rows."""
        C = np.empty((count, self.base.n))
        B = np.empty((count, self.base.m))
        for k in range(count):
            rng = np.random.default_rng((self.seed, start + k))
            C[k] = self.base.c + self.scale * rng.standard_normal(self.base.n)
            B[k] = self.base.b + self.scale * rng.standard_normal(self.base.m)
        return C, B


def family_qp(seed: int = SEED_BASE + 4, n: int = 20_000, m: int = 10_000,
              nnz_row_A: int = 10, nnz_row_B: int = 5, scale: float = 0.1) -> QPFamily:
    """The configuration-0 recipe scaled to n x m keeping its nonzeros per row
    (A: nnz_row_A per row, B: nnz_row_B per row, Q = B'B + 0.01 I)."""
    rng = np.random.default_rng(seed)
    m_eq = m // 2
    A = _fixed_per_row(rng, m, n, nnz_row_A).tocsr()
    Bm = _fixed_per_row(rng, n, n, nnz_row_B).tocsr()
    Q = (Bm.T @ Bm) + 0.01 * sp.identity(n, format="csr")
    c = rng.standard_normal(n)
    b, _ = _feasible_rhs(rng, A, m_eq, -1.0, 1.0, n)
    base = QPInstance("family_qp", n, m, m_eq, _canon(Q, (n, n)), _canon(A, (m, n)), c, b,
                      np.full(n, -10.0), np.full(n, 10.0))
    return QPFamily(base, scale, seed)


# --------------------------------------------------------------------------
# Small instances used to pin the oracle
# --------------------------------------------------------------------------
def tiny_qp(seed: int, n: int, m: int, m_eq: int, bounds: str = "box",
            q_rank: Optional[int] = None, density: float = 1.0, name: str = "tiny_qp") -> QPInstance:
    """Small dense-ish QP with a strictly feasible point.  bounds: 'box'
    (finite l,u), 'lower' (l finite, u=+inf), 'upper', 'free', 'mixed'
    (a random mix of the four per variable)."""
    rng = np.random.default_rng(seed)
    k = n if q_rank is None else q_rank
    G = rng.standard_normal((k, n))
    Q = G.T @ G / max(k, 1)
    if q_rank is None:
        Q += 0.1 * np.eye(n)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    for i in range(m):
        if not A[i].any():
            A[i, rng.integers(0, n)] = 1.0
    x0 = rng.uniform(-0.5, 0.5, n)
    b = A @ x0
    b[m_eq:] -= rng.uniform(0.0, 1.0, m - m_eq)
    c = rng.standard_normal(n)
    lo = -1.0 - rng.uniform(0, 1, n)
    hi = 1.0 + rng.uniform(0, 1, n)
    kinds = {"box": np.zeros(n, int), "lower": np.ones(n, int), "upper": np.full(n, 2),
             "free": np.full(n, 3), "mixed": rng.integers(0, 4, n)}[bounds]
    l = np.where((kinds == 0) | (kinds == 1), lo, -np.inf)
    u = np.where((kinds == 0) | (kinds == 2), hi, np.inf)
    return QPInstance(name, n, m, m_eq, _canon(sp.csr_matrix(Q), (n, n)),
                      _canon(sp.csr_matrix(A), (m, n)), c, b, l, u)


def diagonal_box_qp(seed: int, n: int) -> QPInstance:
    """Q = diag(q), q ~ U(0.5, 2); no rows; finite random box; c ~ N(0, 4)."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.5, 2.0, n)
    c = 2.0 * rng.standard_normal(n)
    l = -rng.uniform(0.2, 1.5, n)
    u = rng.uniform(0.2, 1.5, n)
    return QPInstance("diagonal_box_qp", n, 0, 0, _canon(sp.diags(q), (n, n)),
                      _canon(sp.csr_matrix((0, n)), (0, n)), c, np.zeros(0), l, u)
