"""The one-launch cluster chunk (spmv_threads = 2): a whole chunk of
iterations in one 16-CTA cluster (8 where 16 cannot be resident) with a
cluster barrier after each half-step.  Its iterates are bitwise those of the
per-iteration kernels (the same row arithmetic), in float64 and in mixed
precision, with its row blocks resident in shared memory (at most one of A
and one of P per CTA) and read from global memory (more blocks than CTAs), at
partial chunks, for a batch whose instances stop at different checks, and for
a problem without rows; problems it does not cover are rejected with
PDQP_ERR_INVALID."""
import numpy as np
import pytest

import qpgen
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_cluster_chunk_solve_is_bitwise_the_row_block_solve(precision):
    pd = G.lib()
    inst = qpgen.random_sparse_qp()
    runs = {nt: G.solve(inst, precision=precision, spmv_threads=nt) for nt in (256, 2)}
    for nt, (st, info, x, y) in runs.items():
        assert st == pd.PDQP_OK
        assert info.spmv_threads == nt
    np.testing.assert_array_equal(runs[2][2], runs[256][2])
    np.testing.assert_array_equal(runs[2][3], runs[256][3])
    assert runs[2][1].iterations == runs[256][1].iterations
    assert runs[2][1].rel_kkt == runs[256][1].rel_kkt


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_cluster_chunk_with_more_blocks_than_ctas(precision):
    """n=1500: 46 row blocks of P, more than the cluster's CTAs, so the blocks
    are read from global memory in every half-step (not resident)."""
    pd = G.lib()
    inst = qpgen.random_sparse_qp(n=1500, m=750)
    runs = {nt: G.solve(inst, precision=precision, spmv_threads=nt) for nt in (256, 2)}
    for nt, (st, info, x, y) in runs.items():
        assert st == pd.PDQP_OK
        assert info.spmv_threads == nt
    np.testing.assert_array_equal(runs[2][2], runs[256][2])
    np.testing.assert_array_equal(runs[2][3], runs[256][3])
    assert runs[2][1].iterations == runs[256][1].iterations


def test_cluster_chunk_profile_counts_its_bytes():
    """With the event profiler on, each cluster launch (kind 3, "other") is
    timed and carries the algorithmic bytes of both half-steps of the
    iterations it runs: positive, at most a full chunk's."""
    pd = G.lib()
    inst = qpgen.random_sparse_qp()
    h = G.handle(inst)
    try:
        pd.pdqp_profile_enable(h, True)
        st, info = pd.pdqp_solve(h, pd.pdqp_default_options(spmv_threads=2, precision=0))
        prof = pd.pdqp_profile_read(h)
        pd.pdqp_profile_enable(h, False)
    finally:
        pd.pdqp_destroy(h)
    assert st == pd.PDQP_OK
    other = prof["other"]
    assert other["launches"] > 0 and other["ms"] > 0.0
    per_iter = prof["dual"]["bytes"] + prof["primal"]["bytes"]   # no half-step launches: the whole problem's
    assert 0.0 < other["bytes"] <= 64 * per_iter * (1 + 1e-12)


@pytest.mark.parametrize("iters", [1, 33, 100])
def test_cluster_chunk_state_at_partial_chunks(iters):
    G.lib()
    inst = qpgen.random_sparse_qp()
    a = G.state_after(inst, iters, precision=0, spmv_threads=256)
    b = G.state_after(inst, iters, precision=0, spmv_threads=2)
    for k in a:
        np.testing.assert_array_equal(b[k], a[k])


def test_cluster_chunk_batch_with_instances_stopping_apart():
    pd = G.lib()
    insts = [qpgen.random_sparse_qp(seed=qpgen.SEED_BASE + 7200, n=200, m=100),
             qpgen.mpc_qp(seed=qpgen.SEED_BASE + 7201, T=10),
             qpgen.random_sparse_qp(seed=qpgen.SEED_BASE + 7202, n=600, m=300)]
    N, M = sum(i.n for i in insts), sum(i.m for i in insts)
    res = {}
    for nt in (256, 2):
        h = pd.batch_from_instances(insts)
        try:
            x, y = np.zeros(N), np.zeros(M)
            pd.pdqp_solve(h, pd.pdqp_default_options(spmv_threads=nt), x_out=x, y_out=y)
            res[nt] = (x, y, [(i.iterations, i.status) for i in pd.pdqp_batch_info(h)])
        finally:
            pd.pdqp_destroy(h)
    assert len({it for it, _ in res[2][2]}) > 1          # the instances stop at different checks
    assert res[2][2] == res[256][2]
    np.testing.assert_array_equal(res[2][0], res[256][0])
    np.testing.assert_array_equal(res[2][1], res[256][1])


def test_cluster_chunk_without_rows():
    pd = G.lib()
    inst = qpgen.diagonal_box_qp(seed=qpgen.SEED_BASE + 7203, n=500)
    a = G.solve(inst, spmv_threads=256)
    b = G.solve(inst, spmv_threads=2)
    assert a[0] == b[0] == pd.PDQP_OK
    np.testing.assert_array_equal(b[2], a[2])


def test_cluster_chunk_rejects_a_low_rank_problem():
    pd = G.lib()
    inst = qpgen.diagonal_box_qp(seed=qpgen.SEED_BASE + 7204, n=64)
    h = G.handle(inst)
    try:
        F = np.random.default_rng(0).standard_normal((inst.n, 4)).astype(np.float32)
        pd.pdqp_set_lowrank_Q(h, 4, F)
        with pytest.raises(pd.PdqpError) as e:
            pd.pdqp_solve(h, pd.pdqp_default_options(spmv_threads=2), x_out=np.zeros(inst.n))
        assert e.value.status == pd.PDQP_ERR_INVALID
        assert "spmv_threads = 2" in str(e.value)
    finally:
        pd.pdqp_destroy(h)
