"""The packed batch call: a batch handed over as one block-diagonal problem is
validated, transposed and stacked on the device, and the handle is the one
the per-instance pointer call stacks on the host -- so the solves agree bit
for bit, in both precisions, from host and from device arrays, and through
the host fallback taken for a column of A longer than the device sort."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


def _bag():
    return [qpgen.tiny_qp(50 + k, n=5 + 7 * k, m=3 + 5 * k, m_eq=k, bounds=("box", "mixed", "lower")[k % 3],
                          density=0.5) for k in range(5)] \
        + [qpgen.diagonal_box_qp(98, 13), qpgen.random_sparse_qp()] + qpgen.mpc_batch(6, seed=77)


def _long_column():
    rng = np.random.default_rng(5)
    n, m = 30, 5000
    A = sp.random(m, n, density=0.05, random_state=5, format="csr")
    A = sp.csr_matrix(A + sp.csr_matrix((np.ones(m), (np.arange(m), np.zeros(m, int))), shape=(m, n)))
    A.sort_indices()
    b = A @ rng.uniform(-0.5, 0.5, n) - rng.uniform(0, 1, m)
    return qpgen.QPInstance("long_column", n, m, 0, sp.identity(n, format="csr"), A, rng.standard_normal(n), b,
                            -np.ones(n) * 5, np.ones(n) * 5)


def _packed(pdqp, insts, device=False):
    p = pdqp.pack_instances(insts)
    arrays = [p[k] for k in ("Q_rowptr", "Q_col", "Q_val", "A_rowptr", "A_col", "A_val", "c", "b", "l", "u")]
    if device:
        import torch
        arrays = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]
        torch.cuda.synchronize()
    return pdqp.pdqp_create_batch_packed(p["n"], p["m"], p["m_eq"], *arrays)


def _solve(pdqp, h, insts, **opts):
    try:
        N, M = sum(i.n for i in insts), sum(i.m for i in insts)
        x, y = np.zeros(N), np.zeros(M)
        st, info = pdqp.pdqp_solve(h, pdqp.pdqp_default_options(**opts), x_out=x, y_out=y)
        infos = [(i.status, i.iterations, i.restarts) for i in pdqp.pdqp_batch_info(h)]
        sizes = pdqp.pdqp_get_sizes(h)
    finally:
        pdqp.pdqp_destroy(h)
    return st, infos, x, y, sizes


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
def test_packed_handle_is_the_pointer_batch_handle(pdqp, precision, device):
    insts = _bag()
    a = _solve(pdqp, pdqp.batch_from_instances(insts), insts, precision=precision)
    b = _solve(pdqp, _packed(pdqp, insts, device), insts, precision=precision)
    assert a[0] == b[0] == pdqp.PDQP_OK
    assert a[1] == b[1]
    assert a[4] == b[4]
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])


def test_packed_single_instance_is_pdqp_create(pdqp):
    inst = qpgen.random_sparse_qp()
    st, info, x, y = G.solve(inst)
    b = _solve(pdqp, _packed(pdqp, [inst]), [inst])
    assert b[0] == st and b[1][0][1] == info.iterations
    np.testing.assert_array_equal(b[2], x)
    np.testing.assert_array_equal(b[3], y)


def test_packed_long_column_takes_the_host_stacking(pdqp):
    insts = [qpgen.tiny_qp(61, n=8, m=5, m_eq=2), _long_column(), qpgen.tiny_qp(62, n=9, m=4, m_eq=1)]
    assert np.diff(insts[1].A.tocsc().indptr).max() > 4096
    a = _solve(pdqp, pdqp.batch_from_instances(insts), insts)
    b = _solve(pdqp, _packed(pdqp, insts), insts)
    assert a[0] == b[0] == pdqp.PDQP_OK
    assert a[1] == b[1]
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])


def _expect_invalid(pdqp, p, text):
    with pytest.raises(pdqp.PdqpError) as e:
        pdqp.pdqp_create_batch_packed(p["n"], p["m"], p["m_eq"], p["Q_rowptr"], p["Q_col"], p["Q_val"],
                                      p["A_rowptr"], p["A_col"], p["A_val"], p["c"], p["b"], p["l"], p["u"])
    assert e.value.status == pdqp.PDQP_ERR_INVALID
    assert text in str(e.value)


def test_packed_rejects_malformed_batches(pdqp):
    insts = [qpgen.tiny_qp(71, n=6, m=4, m_eq=1), qpgen.tiny_qp(72, n=5, m=3, m_eq=2)]
    base = pdqp.pack_instances(insts)
    fresh = lambda: {k: np.array(v, copy=True) for k, v in base.items()}
    # a nonzero of instance 1's A pointing at instance 0's variables
    p = fresh()
    k = p["A_rowptr"][4]
    p["A_col"][k] = 0
    _expect_invalid(pdqp, p, "of its instance")
    # the same for Q, and a column past N
    p = fresh()
    p["Q_col"][p["Q_rowptr"][6]] = 2
    _expect_invalid(pdqp, p, "of its instance")
    p = fresh()
    p["A_col"][-1] = 11
    _expect_invalid(pdqp, p, "of its instance")
    # decreasing row pointers, unsorted columns, non-finite data, bad sizes
    p = fresh()
    p["A_rowptr"][2] = p["A_rowptr"][3] + 1
    _expect_invalid(pdqp, p, "rowptr decreases")
    p = fresh()
    r0 = p["Q_rowptr"][0]
    p["Q_col"][r0], p["Q_col"][r0 + 1] = p["Q_col"][r0 + 1], p["Q_col"][r0]
    _expect_invalid(pdqp, p, "strictly increasing")
    p = fresh()
    p["A_val"][3] = np.nan
    _expect_invalid(pdqp, p, "non-finite value")
    p = fresh()
    p["b"][5] = np.inf
    _expect_invalid(pdqp, p, "b: non-finite")
    p = fresh()
    p["l"][7], p["u"][7] = 1.0, -1.0
    _expect_invalid(pdqp, p, "bounds")
    p = fresh()
    p["m_eq"][1] = 4
    _expect_invalid(pdqp, p, "sizes")
    # a handle still builds after the rejections
    b = _solve(pdqp, _packed(pdqp, insts), insts)
    assert b[0] == pdqp.PDQP_OK


def test_device_build_past_the_capped_grid(pdqp):
    """The device build's kernels loop with the grid's stride: a problem of
    2.5M variables (more than the 8192 x 256 threads of a capped grid) is
    assembled whole.  Its iterates after 50 iterations match the oracle's to
    1e-10, and the converged answer is the closed form clip(-c/q, l, u) --
    to 1e-4 only: with both bounds finite a variable just inside its bound has
    a zero dual residual, so at n = 2.5M relKKT bounds its distance to the
    bound through the gap term alone, relative to an objective of about 1e6."""
    from oracle import rapdhg as R
    inst = qpgen.diagonal_box_qp(seed=qpgen.SEED_BASE + 7401, n=2_500_000)
    ref = R.solve(inst, R.Options(max_iter=50, eps=0.0), trace_at=(50,))
    h = G.handle(inst)
    try:
        pdqp.pdqp_solve(h, pdqp.pdqp_default_options(max_iter=50, eps=0.0, norm_A=ref.norm_A, norm_Q=ref.norm_Q))
        x = np.zeros(inst.n)
        pdqp.pdqp_get_iterates(h, x)
    finally:
        pdqp.pdqp_destroy(h)
    assert G.rel_err(x, ref.trace[50]["x"]) <= 1e-10
    st, info, x, y = G.solve(inst, eps=1e-8)
    assert st == pdqp.PDQP_OK
    np.testing.assert_allclose(x, np.clip(-inst.c / inst.Q.diagonal(), inst.l, inst.u), atol=1e-4)


def test_packed_batch_past_the_capped_grid(pdqp):
    """A packed batch of 2600 control QPs (about 2.3M variables, 1.7M rows):
    64 iterations from the packed handle equal those from the per-instance
    pointer handle bit for bit."""
    insts = qpgen.mpc_batch(2600, seed=qpgen.SEED_BASE + 7402)
    N, M = sum(i.n for i in insts), sum(i.m for i in insts)
    assert N > 2_200_000
    outs = []
    for h in (pdqp.batch_from_instances(insts), _packed(pdqp, insts)):
        try:
            pdqp.pdqp_solve(h, pdqp.pdqp_default_options(max_iter=64, eps=0.0))
            st = [np.zeros(N), np.zeros(M), np.zeros(N), np.zeros(M)]
            pdqp.pdqp_get_iterates(h, *st)
            outs.append(st)
        finally:
            pdqp.pdqp_destroy(h)
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    assert np.abs(outs[0][0]).max() > 0
