"""Section 5's algorithm comparison through the batched solver: for PDHG,
accelerated PDHG, restarted PDHG, rAPDHG (the halving restart of Section 5),
rAPDHG with a fixed restart length and with the Section 6 rules, every
instance of a batch ends after the iterations and with the status of its
standalone solve, and a standalone solve takes the oracle's number of
iterations (the oracle's spectral norms injected)."""
import numpy as np
import pytest

import bench
import qpgen
from oracle import rapdhg as R
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu

ORACLE_RULE = {0: "pdqp", 1: "halving", 2: "fixed", 3: "none"}
LIMIT = 20000


def small_set():
    return [qpgen.random_sparse_qp(seed=qpgen.SEED_BASE + 7100, n=200, m=100),
            qpgen.random_sparse_qp(seed=qpgen.SEED_BASE + 7101, n=400, m=200),
            qpgen.mpc_qp(seed=qpgen.SEED_BASE + 7102, T=12)]


def options(pd, acc, rule, K, **kw):
    return pd.pdqp_default_options(precision=pd.PDQP_PREC_FP64, eps=1e-3, max_iter=LIMIT, accelerate=acc,
                                   restart_rule=rule, fixed_K=max(K, 1), **kw)


@pytest.mark.parametrize("variant", range(len(bench.ALGORITHMS)), ids=[a[0] for a in bench.ALGORITHMS])
def test_batched_variant_matches_standalone_solves(variant):
    pd = lib()
    _, acc, rule, K = bench.ALGORITHMS[variant]
    insts = small_set()
    h = pd.batch_from_instances(insts)
    try:
        xs, ys = np.zeros(sum(i.n for i in insts)), np.zeros(sum(i.m for i in insts))
        pd.pdqp_solve(h, options(pd, acc, rule, K), x_out=xs, y_out=ys)
        batch = pd.pdqp_batch_info(h)
    finally:
        pd.pdqp_destroy(h)
    for inst, bi in zip(insts, batch):
        hs = pd.create_from_csr(inst.n, inst.m, inst.m_eq, inst.Q, inst.A, inst.c, inst.b, inst.l, inst.u)
        try:
            st, info = pd.pdqp_solve(hs, options(pd, acc, rule, K), x_out=np.zeros(inst.n), y_out=np.zeros(inst.m))
        finally:
            pd.pdqp_destroy(hs)
        assert (bi.iterations, bi.status, bi.restarts) == (info.iterations, info.status, info.restarts)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 5], ids=[bench.ALGORITHMS[v][0] for v in (0, 1, 2, 3, 5)])
def test_standalone_variant_takes_the_oracles_iterations(variant):
    pd = lib()
    _, acc, rule, K = bench.ALGORITHMS[variant]
    inst = small_set()[0]
    ref = R.solve(inst, R.Options(eps=1e-3, max_iter=LIMIT, accelerate=bool(acc), restart_rule=ORACLE_RULE[rule],
                                  fixed_K=max(K, 1)))
    h = pd.create_from_csr(inst.n, inst.m, inst.m_eq, inst.Q, inst.A, inst.c, inst.b, inst.l, inst.u)
    try:
        st, info = pd.pdqp_solve(h, options(pd, acc, rule, K, norm_A=ref.norm_A, norm_Q=ref.norm_Q),
                                 x_out=np.zeros(inst.n), y_out=np.zeros(inst.m))
    finally:
        pd.pdqp_destroy(h)
    assert info.iterations == ref.iterations
    assert info.restarts == ref.restarts
    assert (info.status == pd.PDQP_OK) == (ref.status == "optimal")
