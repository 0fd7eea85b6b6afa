"""The allocation-free relKKT entry point (pdqp_kkt_noalloc) against the
handle-based one (pdqp_kkt).

pdqp_kkt_noalloc serves callers that cannot allocate device memory once they
run -- a real-time control loop, code under CUDA stream capture, a host with a
fixed device-memory budget -- by keeping its partial sums in a static device
array.  Two calls in a row, first a larger then a smaller problem, must each
agree with pdqp_kkt; the second also shows that the shared array's leftover
contents from the first call do not leak into the result."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

TOL = 1e-12   # same relative tolerance as the pdqp_kkt parity test


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


def test_noalloc_kkt_matches_pdqp_kkt_on_two_calls():
    import torch
    pdqp = G.lib()
    insts = [qpgen.random_sparse_qp(), qpgen.tiny_qp(8, n=30, m=20, m_eq=5, bounds="mixed")]
    for call, inst in enumerate(insts):
        x, y = _point(inst, 100 + call)
        h = G.handle(inst)
        try:
            want = pdqp.pdqp_kkt(h, x, y)
        finally:
            pdqp.pdqp_destroy(h)
        d = _device_problem(inst)
        xd = torch.from_numpy(x).cuda()
        yd = torch.from_numpy(y).cuda()
        parts = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        st = pdqp.pdqp_kkt_noalloc(inst.n, inst.m, inst.m_eq, d["Q_rowptr"], d["Q_col"], d["Q_val"],
                                   d["A_rowptr"], d["A_col"], d["A_val"], d["At_rowptr"], d["At_col"],
                                   d["At_val"], d["c"], d["b"], d["l"], d["u"], xd, yd, parts)
        torch.cuda.synchronize()
        assert st == pdqp.PDQP_OK, pdqp.pdqp_last_error()
        got = parts.cpu().numpy()
        for k in range(6):
            assert got[k] == pytest.approx(want[k], rel=TOL, abs=1e-13), (call, k, got[k], want[k])


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
