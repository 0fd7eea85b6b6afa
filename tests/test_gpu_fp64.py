"""Parity of the float64 CUDA path with the CPU oracle, through the C ABI.

Bar: iterates agree with the oracle to relative 1e-10 over the first 200
iterations (same inputs, same spectral norms injected); solves end at relative
KKT <= 1e-6 (recomputed by the oracle on the returned point) with the
objective within relative 1e-6 of the oracle's.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G
from tests.qp_truth import active_set_solve

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
CHECKPOINTS = (1, 2, 3, 10, 63, 64, 65, 100, 128, 129, 150, 192, 199, 200)


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


@pytest.fixture(scope="module")
def cfg0():
    return qpgen.random_sparse_qp()


@pytest.fixture(scope="module")
def cfg0_oracle(cfg0):
    return R.solve(cfg0, R.Options(max_iter=200, eps=0.0), trace_at=CHECKPOINTS)


@pytest.fixture(scope="module")
def cfg0_solution(cfg0):
    return R.solve(cfg0, R.Options())


# --------------------------------------------------------------------------- iterate parity
@pytest.mark.parametrize("t", CHECKPOINTS)
def test_iterates_match_oracle(pdqp, cfg0, cfg0_oracle, t):
    ref = cfg0_oracle.trace[t]
    got = G.state_after(cfg0, t, norm_A=cfg0_oracle.norm_A, norm_Q=cfg0_oracle.norm_Q)
    for key in ("x", "y", "xbar", "ybar"):
        assert G.rel_err(got[key], ref[key]) <= ITER_TOL, (t, key, G.rel_err(got[key], ref[key]))


def test_restart_decisions_match_over_600_iterations(pdqp, cfg0):
    ref = R.solve(cfg0, R.Options(max_iter=600, eps=0.0), trace_at=(600,))
    got = G.state_after(cfg0, 600, norm_A=ref.norm_A, norm_Q=ref.norm_Q)
    for key in ("x", "y", "xbar", "ybar"):
        assert G.rel_err(got[key], ref.trace[600][key]) <= 1e-9, key


def test_hand_worked_iterations_on_gpu(pdqp):
    """The three hand-computed iterations (exact fractions) on the GPU."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_three_iterations.json")))
    d = g["problem"]
    inst = qpgen.QPInstance("hand", 1, 1, 0, sp.csr_matrix(np.array(d["Q"], float)),
                            sp.csr_matrix(np.array(d["A"], float)), np.array(d["c"], float),
                            np.array(d["b"], float), np.array(d["l"], float), np.array(d["u"], float))
    inst.Q.indptr = inst.Q.indptr.astype(np.int32); inst.Q.indices = inst.Q.indices.astype(np.int32)
    inst.A.indptr = inst.A.indptr.astype(np.int32); inst.A.indices = inst.A.indices.astype(np.int32)
    for it, want in g["iterates"].items():
        got = G.state_after(inst, int(it), step_rule=1, restart_rule=2, fixed_K=4, scaling=0, norm_Q=2.0,
                            norm_A=1.0, check_period=1000)
        for key in ("x", "y", "xbar", "ybar"):
            assert got[key][0] == pytest.approx(float(Fraction(want[key])), rel=1e-14, abs=1e-15), (it, key)


@pytest.mark.parametrize("variant", ["halving", "fixed", "none_pdhg", "theory", "noscale", "warm"])
def test_variant_iterates_match_oracle(pdqp, variant):
    inst = qpgen.tiny_qp(5, n=37, m=29, m_eq=9, bounds="mixed", density=0.3)
    ro = dict(halving=R.Options(restart_rule="halving"), fixed=R.Options(restart_rule="fixed", fixed_K=64),
              none_pdhg=R.Options(restart_rule="none", accelerate=False),
              theory=R.Options(step_rule="theory", restart_rule="fixed", fixed_K=64),
              noscale=R.Options(scaling=False), warm=R.Options())[variant]
    go = dict(halving=dict(restart_rule=1), fixed=dict(restart_rule=2, fixed_K=64),
              none_pdhg=dict(restart_rule=3, accelerate=0), theory=dict(step_rule=1, restart_rule=2, fixed_K=64),
              noscale=dict(scaling=0), warm={})[variant]
    ro.max_iter, ro.eps, ro.check_period = 300, 0.0, 32
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-1, 1, inst.n) if variant == "warm" else None
    y0 = rng.uniform(-1, 1, inst.m) if variant == "warm" else None
    ref = R.solve(inst, ro, x0=x0, y0=y0, trace_at=(1, 33, 100, 300))
    from paper_2311_07710_gb300 import pdqp as P
    for t in (1, 33, 100, 300):
        h = G.handle(inst)
        try:
            o = P.pdqp_default_options(max_iter=t, eps=0.0, check_period=32, norm_A=ref.norm_A,
                                       norm_Q=ref.norm_Q, **go)
            P.pdqp_solve(h, o, x0=x0, y0=y0)
            out = [np.zeros(inst.n), np.zeros(inst.m), np.zeros(inst.n), np.zeros(inst.m)]
            P.pdqp_get_iterates(h, *out)
        finally:
            P.pdqp_destroy(h)
        for key, v in zip(("x", "y", "xbar", "ybar"), out):
            assert G.rel_err(v, ref.trace[t][key]) <= ITER_TOL, (variant, t, key)


# --------------------------------------------------------------------------- end-to-end
def test_config0_solves_to_1e6(pdqp, cfg0, cfg0_solution):
    st, info, x, y = G.solve(cfg0)
    assert st == pdqp.PDQP_OK
    p = R.problem_from_instance(cfg0)
    parts = R.kkt_parts(p, x, y)
    assert parts["rel_kkt"] <= 1.0001e-6
    assert info.rel_kkt == pytest.approx(parts["rel_kkt"], rel=1e-6, abs=1e-12)
    ref = cfg0_solution.kkt["primal_obj"]
    assert abs(parts["primal_obj"] - ref) <= 1e-6 * (1 + abs(ref))
    assert abs(info.iterations - cfg0_solution.iterations) <= 64
    assert info.norm_A == pytest.approx(cfg0_solution.norm_A, rel=1e-5)
    assert info.norm_Q == pytest.approx(cfg0_solution.norm_Q, rel=1e-5)


def test_device_pointer_path_is_identical(pdqp, cfg0):
    import torch
    a = G.solve(cfg0)
    h = G.handle(cfg0, device=True)
    try:
        x = torch.zeros(cfg0.n, dtype=torch.float64, device="cuda")
        y = torch.zeros(cfg0.m, dtype=torch.float64, device="cuda")
        st, info = pdqp.pdqp_solve(h, pdqp.pdqp_default_options(), x_out=x, y_out=y)
        torch.cuda.synchronize()
    finally:
        pdqp.pdqp_destroy(h)
    assert st == a[0] and info.iterations == a[1].iterations
    np.testing.assert_array_equal(x.cpu().numpy(), a[2])
    np.testing.assert_array_equal(y.cpu().numpy(), a[3])


def test_runs_are_bitwise_reproducible(pdqp, cfg0):
    a, b = G.solve(cfg0), G.solve(cfg0)
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])


@pytest.mark.parametrize("seed,n,m,m_eq,bounds,rank", [
    (21, 4, 3, 1, "box", None), (22, 5, 4, 2, "mixed", None), (23, 6, 3, 0, "lower", None),
    (24, 5, 2, 1, "upper", None), (31, 6, 3, 1, "box", 2), (25, 6, 4, 2, "mixed", None),
])
def test_tiny_qps_match_brute_force(pdqp, seed, n, m, m_eq, bounds, rank):
    inst = qpgen.tiny_qp(seed, n=n, m=m, m_eq=m_eq, bounds=bounds, q_rank=rank)
    truth = active_set_solve(inst.Q.toarray(), inst.A.toarray(), inst.b, inst.c, inst.l, inst.u, m_eq)
    st, info, x, y = G.solve(inst, eps=1e-9)
    assert st == pdqp.PDQP_OK
    assert info.primal_obj == pytest.approx(truth[2], rel=1e-7, abs=1e-7)
    if rank is None:
        np.testing.assert_allclose(x, truth[0], atol=1e-5)


@pytest.mark.parametrize("n", [1, 7, 255, 256, 257, 1000])
def test_box_qp_closed_form_ragged_sizes(pdqp, n):
    """No rows (m = 0): x* = clip(-c/q, l, u); sizes straddle block boundaries."""
    inst = qpgen.diagonal_box_qp(100 + n, n)
    st, info, x, y = G.solve(inst, eps=1e-10)
    assert st == pdqp.PDQP_OK
    np.testing.assert_allclose(x, np.clip(-inst.c / inst.Q.diagonal(), inst.l, inst.u), atol=1e-8)


def test_lp_vertex(pdqp):
    A = sp.csr_matrix(np.array([[-1.0, -2.0], [-3.0, -1.0]]))
    A.indptr = A.indptr.astype(np.int32); A.indices = A.indices.astype(np.int32)
    Q = sp.csr_matrix((2, 2)); Q.indptr = Q.indptr.astype(np.int32); Q.indices = Q.indices.astype(np.int32)
    inst = qpgen.QPInstance("lp", 2, 2, 0, Q, A, np.array([-1.0, -1.0]), np.array([-4.0, -6.0]), np.zeros(2),
                            np.full(2, np.inf))
    st, info, x, y = G.solve(inst, eps=1e-10)
    assert st == pdqp.PDQP_OK
    np.testing.assert_allclose(x, [1.6, 1.2], atol=1e-8)


def test_iteration_limit_returns_candidate(pdqp, cfg0):
    ref = R.solve(cfg0, R.Options(max_iter=100, eps=0.0))
    st, info, x, y = G.solve(cfg0, max_iter=100, eps=0.0, norm_A=ref.norm_A, norm_Q=ref.norm_Q)
    assert st == pdqp.PDQP_ITER_LIMIT and info.iterations == 100
    assert G.rel_err(x, ref.x) <= ITER_TOL and G.rel_err(y, ref.y) <= ITER_TOL


def test_kkt_entry_point_matches_oracle(pdqp):
    rng = np.random.default_rng(9)
    for inst in (qpgen.random_sparse_qp(), qpgen.tiny_qp(8, n=30, m=20, m_eq=5, bounds="mixed")):
        p = R.problem_from_instance(inst)
        h = G.handle(inst)
        try:
            for _ in range(3):
                x = np.clip(rng.normal(size=inst.n), inst.l, inst.u)
                y = rng.normal(size=inst.m)
                y[inst.m_eq:] = np.abs(y[inst.m_eq:])
                got = pdqp.pdqp_kkt(h, x, y)
                ref = R.kkt_parts(p, x, y)
                for k, key in enumerate(("r_primal", "r_dual", "r_gap", "rel_kkt", "primal_obj", "dual_obj")):
                    assert got[k] == pytest.approx(ref[key], rel=1e-12, abs=1e-13), key
        finally:
            pdqp.pdqp_destroy(h)


def test_invalid_inputs(pdqp):
    inst = qpgen.tiny_qp(1, n=4, m=2, m_eq=1)
    Q, A = inst.Q, inst.A
    cases = {
        "unsorted": (Q.indptr, Q.indices[::-1].copy(), Q.data, inst.l, inst.u),
        "nan": (Q.indptr, Q.indices, np.where(np.arange(Q.nnz) == 0, np.nan, Q.data), inst.l, inst.u),
        "l>u": (Q.indptr, Q.indices, Q.data, inst.u + 1, inst.u),
    }
    for name, (rp, ci, v, l, u) in cases.items():
        with pytest.raises(pdqp.PdqpError) as e:
            pdqp.pdqp_create(4, 2, 1, rp, ci, v, A.indptr, A.indices, A.data, inst.c, inst.b, l, u)
        assert e.value.status == pdqp.PDQP_ERR_INVALID, name
    with pytest.raises(pdqp.PdqpError):
        pdqp.pdqp_create(4, 2, 3, Q.indptr, Q.indices, Q.data, A.indptr, A.indices, A.data, inst.c, inst.b,
                         inst.l, inst.u)
    h = G.handle(inst)
    try:
        with pytest.raises(pdqp.PdqpError):
            pdqp.pdqp_solve(h, pdqp.pdqp_default_options(check_period=3))
    finally:
        pdqp.pdqp_destroy(h)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(pdqp, cfg0, precision):
    """A chunk replayed from its captured CUDA graph computes exactly what the
    direct launches compute."""
    a = G.solve(cfg0, precision=precision, no_graphs=0)
    b = G.solve(cfg0, precision=precision, no_graphs=1)
    assert a[1].iterations == b[1].iterations
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])


def test_create_rejects_bad_row_pointers_and_handles_long_columns(pdqp):
    """Row pointers that leave [0, nnz] are rejected before any column is read;
    a column of A longer than the device sort takes (4096) is built on the
    host and solves like the rest."""
    inst = qpgen.tiny_qp(3, n=4, m=2, m_eq=1)
    bad_rp = np.array([0, 50, 3, 4, 4], np.int32)      # row 0 claims 50 entries of 4
    with pytest.raises(pdqp.PdqpError) as e:
        pdqp.pdqp_create(4, 2, 1, bad_rp, inst.Q.indices[:4].copy(), inst.Q.data[:4].copy(), inst.A.indptr,
                         inst.A.indices, inst.A.data, inst.c, inst.b, inst.l, inst.u)
    assert e.value.status == pdqp.PDQP_ERR_INVALID
    rng = np.random.default_rng(5)
    n, m = 30, 5000
    A = sp.random(m, n, density=0.05, random_state=5, format="csr")
    A = sp.csr_matrix(A + sp.csr_matrix((np.ones(m), (np.arange(m), np.zeros(m, int))), shape=(m, n)))
    A.sort_indices()
    x0 = rng.uniform(-0.5, 0.5, n)
    b = A @ x0 - rng.uniform(0, 1, m)
    Q = sp.identity(n, format="csr")
    big = qpgen.QPInstance("long_column", n, m, 0, sp.csr_matrix(Q), A, rng.standard_normal(n), b,
                           -np.ones(n) * 5, np.ones(n) * 5)
    assert np.diff(A.tocsc().indptr).max() > 4096
    st, info, x, y = G.solve(big, eps=1e-6)
    assert st == pdqp.PDQP_OK
    parts = R.kkt_parts(R.problem_from_instance(big), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6


def test_autotuned_variant_gives_the_same_iterates(pdqp, cfg0):
    """The default options autotune the iteration-kernel variant on the first
    chunk; every variant yields bitwise identical iterates, so the choice
    never changes the answer."""
    outs = {}
    for nt in (0, 256, 512, 1, 2):
        st, info, x, y = G.solve(cfg0, spmv_threads=nt)
        outs[nt] = (x, y, info.iterations, info.spmv_threads)
        assert st == pdqp.PDQP_OK
    assert outs[0][3] in (256, 512, 1, 2)
    for nt in (256, 512, 1, 2):
        assert outs[nt][3] == nt
        np.testing.assert_array_equal(outs[nt][0], outs[0][0])
        np.testing.assert_array_equal(outs[nt][1], outs[0][1])
        assert outs[nt][2] == outs[0][2]
