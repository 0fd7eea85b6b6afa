"""Degenerate and boundary shapes against the oracle: a 1 x 1 problem, only
equalities, only inequalities, free variables, an empty row of A together
with a variable that appears in no row and no entry of Q, rows of exactly
2048, 2049 and 4096 nonzeros (a full row block, one nonzero past it, two
segments), and entries over 24 decades with exact ties and subnormals.  float64 iterates match the oracle's (norms injected) at three
checkpoints; mixed-precision solves reach the oracle's end state; a batch
with a member that has no rows reproduces the standalone solves bit for bit."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
CHECKPOINTS = (1, 33, 100)


def _canon(M, shape):
    M = sp.csr_matrix(M, shape=shape, dtype=np.float64)
    M.sum_duplicates()
    M.eliminate_zeros()
    M.sort_indices()
    M.indptr = M.indptr.astype(np.int32)
    M.indices = M.indices.astype(np.int32)
    return M


def empty_row_and_column():
    base = qpgen.tiny_qp(seed=qpgen.SEED_BASE + 7300, n=10, m=5, m_eq=2)
    A = base.A.toarray()
    A[3, :] = 0.0                              # an inequality row with no entries: 0 >= b_3
    A[:, 7] = 0.0                              # variable 7 in no row ...
    Q = base.Q.toarray()
    Q[7, :] = 0.0
    Q[:, 7] = 0.0                              # ... and in no entry of Q (linear in x_7, boxed)
    b = base.b.copy()
    b[3] = -1.0
    x0 = np.zeros(10)
    b[:2] = A[:2] @ x0                         # keep the equalities consistent with x = 0
    b[2:] = np.minimum(b[2:], A[2:] @ x0 - 0.5)
    b[3] = -1.0
    return qpgen.QPInstance("empty_row_col", 10, 5, 2, _canon(Q, (10, 10)), _canon(A, (5, 10)), base.c, b,
                            base.l, base.u)


def long_rows():
    rng = np.random.default_rng(7301)
    n, lens = 5000, (2048, 2049, 4096, 10)
    rows, cols, vals = [], [], []
    for i, k in enumerate(lens):
        c = rng.choice(n, size=k, replace=False)
        rows += [i] * k
        cols += list(c)
        vals += list(rng.standard_normal(k) / np.sqrt(k))
    A = _canon(sp.coo_matrix((vals, (rows, cols)), shape=(len(lens), n)), (len(lens), n))
    x0 = rng.uniform(-0.5, 0.5, n)
    b = A @ x0
    b[2:] -= 0.5
    Q = _canon(sp.diags(rng.uniform(0.5, 2.0, n)), (n, n))
    return qpgen.QPInstance("long_rows", n, len(lens), 2, Q, A, rng.standard_normal(n), b, np.full(n, -1.0),
                            np.full(n, 1.0))


def wide_magnitudes():
    """A = S G T with row and column factors spread over 1e-12..1e12 (the
    Ruiz passes undo them; their row maxima are formed from bit patterns and
    must be the exact maxima), Q = T Q0 T, c, b, l, u scaled to match; column
    1 is minus column 0 with the same Q entry, so the two have equal factors
    and every row's two products tie exactly; two subnormal entries."""
    rng = np.random.default_rng(7309)
    n, m, m_eq = 60, 30, 10
    s = 10.0 ** rng.uniform(-12, 12, m)
    t = 10.0 ** rng.uniform(-12, 12, n)
    t[1] = t[0]
    G0 = sp.random(m, n, density=0.15, random_state=rng, data_rvs=rng.standard_normal).toarray()
    G0[:, 0] = np.where(G0[:, 0] == 0.0, 1.0, G0[:, 0])
    G0[:, 1] = -G0[:, 0]
    A = (s[:, None] * G0) * t[None, :]
    A[2, 5] = 1e-310
    A[3, 7] = -2e-310
    q0 = rng.uniform(1.0, 2.0, n)
    q0[1] = q0[0]
    Q = sp.diags(q0 * t * t)
    x0 = rng.uniform(-0.5, 0.5, n) / t
    b = A @ x0
    b[m_eq:] -= 0.5 * s[m_eq:]
    return qpgen.QPInstance("wide_magnitudes", n, m, m_eq, _canon(Q, (n, n)), _canon(A, (m, n)),
                            t * rng.standard_normal(n), b, -1.0 / t, 1.0 / t)


CASES = {
    "1x1": lambda: qpgen.tiny_qp(seed=qpgen.SEED_BASE + 7302, n=1, m=1, m_eq=0),
    "all_equality": lambda: qpgen.tiny_qp(seed=qpgen.SEED_BASE + 7303, n=12, m=6, m_eq=6),
    "all_inequality": lambda: qpgen.tiny_qp(seed=qpgen.SEED_BASE + 7304, n=12, m=6, m_eq=0),
    "free_variables": lambda: qpgen.tiny_qp(seed=qpgen.SEED_BASE + 7305, n=10, m=4, m_eq=2, bounds="free"),
    "empty_row_and_column": empty_row_and_column,
    "long_row_boundaries": long_rows,
    "wide_magnitudes": wide_magnitudes,
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_float64_iterates_match_oracle(name):
    G.lib()
    inst = CASES[name]()
    ref = R.solve(inst, R.Options(max_iter=max(CHECKPOINTS), eps=0.0, check_period=32), trace_at=CHECKPOINTS)
    for t in CHECKPOINTS:
        got = G.state_after(inst, t, precision=0, check_period=32, norm_A=ref.norm_A, norm_Q=ref.norm_Q)
        for key in ("x", "y", "xbar", "ybar"):
            assert G.rel_err(got[key], ref.trace[t][key]) <= ITER_TOL, (name, t, key)


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_end_state(name):
    pd = G.lib()
    inst = CASES[name]()
    ref = R.solve(inst, R.Options(eps=1e-6))
    st, info, x, y = G.solve(inst, precision=1)
    assert st == pd.PDQP_OK
    parts = R.kkt_parts(R.problem_from_instance(inst), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6
    obj = ref.kkt["primal_obj"]
    assert abs(parts["primal_obj"] - obj) <= 1e-6 * (1 + abs(obj))


def test_batch_with_a_member_without_rows():
    pd = G.lib()
    insts = [qpgen.diagonal_box_qp(seed=qpgen.SEED_BASE + 7306, n=50),
             qpgen.tiny_qp(seed=qpgen.SEED_BASE + 7307, n=12, m=6, m_eq=3),
             qpgen.random_sparse_qp(seed=qpgen.SEED_BASE + 7308, n=200, m=100)]
    h = pd.batch_from_instances(insts)
    try:
        x, y = np.zeros(sum(i.n for i in insts)), np.zeros(sum(i.m for i in insts))
        pd.pdqp_solve(h, pd.pdqp_default_options(), x_out=x, y_out=y)
        infos = pd.pdqp_batch_info(h)
    finally:
        pd.pdqp_destroy(h)
    xo = yo = 0
    for inst, bi in zip(insts, infos):
        st, info, xs, ys = G.solve(inst)
        assert (bi.iterations, bi.status) == (info.iterations, info.status)
        np.testing.assert_array_equal(x[xo:xo + inst.n], xs)
        np.testing.assert_array_equal(y[yo:yo + inst.m], ys)
        xo += inst.n
        yo += inst.m


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_every_variant_gives_the_same_bits_with_long_rows(precision):
    """Rows past a row block (2049 and 4096 entries, P's rows of those A'
    columns) are summed from the same segment sums by every iteration-kernel
    variant, the pipelined persistent one included, so the autotuner's choice
    never changes the answer there either."""
    pd = G.lib()
    inst = long_rows()
    runs = {nt: G.solve(inst, precision=precision, spmv_threads=nt) for nt in (256, 512, 1)}
    for nt, (st, info, x, y) in runs.items():
        assert st == pd.PDQP_OK and info.spmv_threads == nt
    for nt in (512, 1):
        assert runs[nt][1].iterations == runs[256][1].iterations
        np.testing.assert_array_equal(runs[nt][2], runs[256][2])
        np.testing.assert_array_equal(runs[nt][3], runs[256][3])
