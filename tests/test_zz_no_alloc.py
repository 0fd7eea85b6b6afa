"""The allocation-free relKKT entry point (pdqp_kkt_noalloc) against the
handle-based one (pdqp_kkt).

pdqp_kkt_noalloc serves callers that cannot allocate device memory once they
run -- a real-time control loop, a process held to a fixed device-memory
budget -- by keeping its partial sums in a static device array.  Two calls in a
row, first a larger then a smaller problem, must each agree with pdqp_kkt; the
second also shows that the shared array's leftover contents from the first
call do not leak into the result.  The same calls are checked against the
oracle's relKKT directly, the largest accepted problem fills the array exactly,
and host pointers are refused before any device work."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

TOL = 1e-12   # same relative tolerance as the pdqp_kkt parity test
KEYS = ("r_primal", "r_dual", "r_gap", "rel_kkt", "primal_obj", "dual_obj")


def _device_problem(inst):
    import torch
    At = sp.csr_matrix(inst.A.T)
    At.sort_indices()
    arrays = dict(
        Q_rowptr=inst.Q.indptr, Q_col=inst.Q.indices, Q_val=inst.Q.data,
        A_rowptr=inst.A.indptr, A_col=inst.A.indices, A_val=inst.A.data,
        At_rowptr=At.indptr.astype(np.int32), At_col=At.indices.astype(np.int32), At_val=At.data,
        c=inst.c, b=inst.b, l=inst.l, u=inst.u)
    out = {}
    for k, v in arrays.items():
        dt = np.int32 if ("rowptr" in k or "col" in k) else np.float64
        out[k] = torch.from_numpy(np.ascontiguousarray(v, dtype=dt)).cuda()
    return out


def _point(inst, seed):
    rng = np.random.default_rng(seed)
    x = np.clip(rng.normal(size=inst.n), inst.l, inst.u)
    y = rng.normal(size=inst.m)
    y[inst.m_eq:] = np.abs(y[inst.m_eq:])
    return x, y


def _noalloc(pdqp, inst, x, y):
    import torch
    d = _device_problem(inst)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    parts = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    st = pdqp.pdqp_kkt_noalloc(inst.n, inst.m, inst.m_eq, d["Q_rowptr"], d["Q_col"], d["Q_val"],
                               d["A_rowptr"], d["A_col"], d["A_val"], d["At_rowptr"], d["At_col"],
                               d["At_val"], d["c"], d["b"], d["l"], d["u"], xd, yd, parts)
    torch.cuda.synchronize()
    assert st == pdqp.PDQP_OK, pdqp.pdqp_last_error()
    return parts.cpu().numpy()


def _handle_kkt(pdqp, inst, x, y):
    h = G.handle(inst)
    try:
        return pdqp.pdqp_kkt(h, x, y)
    finally:
        pdqp.pdqp_destroy(h)


def test_noalloc_kkt_matches_pdqp_kkt_on_two_calls():
    pdqp = G.lib()
    insts = [qpgen.random_sparse_qp(), qpgen.tiny_qp(8, n=30, m=20, m_eq=5, bounds="mixed")]
    for call, inst in enumerate(insts):
        x, y = _point(inst, 100 + call)
        want = _handle_kkt(pdqp, inst, x, y)
        got = _noalloc(pdqp, inst, x, y)
        for k in range(6):
            assert got[k] == pytest.approx(want[k], rel=TOL, abs=1e-13), (call, k, got[k], want[k])


def test_noalloc_kkt_matches_the_oracle():
    """The same two calls against the oracle's relKKT (Section 5's metric in
    the equality/bound form), not only against the other entry point."""
    pdqp = G.lib()
    insts = [qpgen.random_sparse_qp(), qpgen.tiny_qp(8, n=30, m=20, m_eq=5, bounds="mixed")]
    for call, inst in enumerate(insts):
        x, y = _point(inst, 200 + call)
        got = _noalloc(pdqp, inst, x, y)
        ref = R.kkt_parts(R.problem_from_instance(inst), x, y)
        for k, key in enumerate(KEYS):
            assert got[k] == pytest.approx(ref[key], rel=TOL, abs=1e-13), (call, key, got[k], ref[key])


def _widest_problem(seed=31, n=65536, per_row=24):
    """n = m = 65536 (the largest accepted sizes) with 24 nonzeros per row of
    A, so that both relKKT kernels take 32 lanes per row and 8 rows per block:
    8192 blocks, the whole scratch array."""
    rng = np.random.default_rng(seed)
    m, m_eq = n, n // 2
    cols = rng.integers(0, n, size=m * per_row)
    rows = np.repeat(np.arange(m), per_row)
    A = sp.csr_matrix((rng.normal(size=cols.size), (rows, cols)), shape=(m, n))   # repeats summed
    A.sum_duplicates()
    A.sort_indices()
    i, j = rng.integers(0, n, size=2 * n), rng.integers(0, n, size=2 * n)
    S = sp.csr_matrix((rng.normal(size=2 * n), (i, j)), shape=(n, n))
    S = S + S.T
    Q = sp.csr_matrix(S + sp.diags(np.abs(S).sum(axis=1).A1 + 1.0))
    Q.sort_indices()
    c = rng.normal(size=n)
    b = rng.normal(size=m)
    l, u = np.full(n, -10.0), np.full(n, 10.0)
    return qpgen.QPInstance(name="noalloc_widest", n=n, m=m, m_eq=m_eq,
                            Q=sp.csr_matrix((Q.data, Q.indices.astype(np.int32), Q.indptr.astype(np.int32)),
                                            shape=Q.shape),
                            A=sp.csr_matrix((A.data, A.indices.astype(np.int32), A.indptr.astype(np.int32)),
                                            shape=A.shape),
                            c=c, b=b, l=l, u=u)


def test_noalloc_at_the_largest_accepted_sizes():
    pdqp = G.lib()
    inst = _widest_problem()
    assert inst.A.nnz / inst.m > 16 and (inst.Q.nnz + inst.A.nnz) / inst.n > 16   # 32 lanes per row
    x, y = _point(inst, 300)
    got = _noalloc(pdqp, inst, x, y)
    want = _handle_kkt(pdqp, inst, x, y)
    ref = R.kkt_parts(R.problem_from_instance(inst), x, y)
    for k, key in enumerate(KEYS):
        assert got[k] == pytest.approx(want[k], rel=TOL, abs=1e-13), (key, got[k], want[k])
        assert got[k] == pytest.approx(ref[key], rel=TOL, abs=1e-13), (key, got[k], ref[key])


def test_noalloc_refuses_host_pointers():
    import ctypes
    import torch
    pdqp = G.lib()
    inst = qpgen.tiny_qp(8, n=30, m=20, m_eq=5, bounds="mixed")
    d = _device_problem(inst)
    x, y = _point(inst, 400)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    parts = torch.zeros(6, dtype=torch.float64, device="cuda")
    args = [d["Q_rowptr"], d["Q_col"], d["Q_val"], d["A_rowptr"], d["A_col"], d["A_val"], d["At_rowptr"],
            d["At_col"], d["At_val"], d["c"], d["b"], d["l"], d["u"], xd, yd, parts]
    host_x = np.ascontiguousarray(x)
    for k in (0, 5, 13, 15):       # Q's row pointers, A's values, x, the output
        ptrs = [a.data_ptr() for a in args]
        ptrs[k] = host_x.ctypes.data_as(ctypes.c_void_p).value
        st = pdqp.load().pdqp_kkt_noalloc(inst.n, inst.m, inst.m_eq, ptrs[0], ptrs[1], ptrs[2], inst.Q.nnz,
                                          ptrs[3], ptrs[4], ptrs[5], ptrs[6], ptrs[7], ptrs[8], inst.A.nnz,
                                          ptrs[9], ptrs[10], ptrs[11], ptrs[12], ptrs[13], ptrs[14], ptrs[15], None)
        assert st == pdqp.PDQP_ERR_INVALID, k
    torch.cuda.synchronize()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    pdqp = G.lib()
    n = 65537
    z = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    parts = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = pdqp.load().pdqp_kkt_noalloc(n, 0, 0, z.data_ptr(), None, None, 0, None, None, None, None, None,
                                      None, 0, v.data_ptr(), None, v.data_ptr(), v.data_ptr(), v.data_ptr(),
                                      None, parts.data_ptr(), None)
    assert st == pdqp.PDQP_ERR_INVALID
