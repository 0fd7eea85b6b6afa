"""The GPU's Lanczos norms on the operators the all-ones start vector fails
on (a regularised path-graph Laplacian Q, a difference-constraint A whose rows
sum to zero): the norms of the scaled matrices against dense eigen-solves of
the same scaled matrices (the oracle's scaling factors), and both problems
solved to the oracle's end state in both precisions; and the chunked partial
sums of the estimates: repeated solves of a handle and a batch of copies give
the same norms bit for bit."""
import numpy as np
import pytest

from oracle import rapdhg as R
from tests import gpu_util as G
from tests.test_oracle_lanczos_start import difference_lp, laplacian_qp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("make", [laplacian_qp, difference_lp], ids=["laplacian", "difference"])
def test_norms_and_end_state(pdqp, make, precision):
    inst = make()
    ref = R.solve(inst, R.Options())
    ps = R.scale_problem(R.problem_from_instance(inst), ref.D1, ref.D2)
    dense_Q = np.linalg.eigvalsh(ps.Q.toarray())[-1]
    dense_A = np.linalg.svd(ps.A.toarray(), compute_uv=False)[0] if inst.m else 0.0
    st, info, x, y = G.solve(inst, precision=precision)
    assert st == pdqp.PDQP_OK
    assert info.norm_Q == pytest.approx(dense_Q, rel=1e-5)
    assert info.norm_A == pytest.approx(dense_A, rel=1e-5)
    parts = R.kkt_parts(R.problem_from_instance(inst), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6
    assert abs(parts["primal_obj"] - ref.kkt["primal_obj"]) <= 1e-6 * (1 + abs(ref.kkt["primal_obj"]))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_norms_repeat_and_match_in_a_batch(pdqp, precision):
    """The norm estimates' block partials are summed per chunk of 32 row
    blocks by the chunk's last block to finish (a ticket that resets itself):
    solving the same handle again gives the same norms bit for bit, and a
    batch holding the problem twice gives each copy the standalone norms.  A
    problem of several chunks."""
    import qpgen
    from paper_2311_07710_gb300 import pdqp as P
    inst = qpgen.random_sparse_qp(seed=qpgen.SEED_BASE + 7410, n=8000, m=4000, density_A=1.25e-3,
                                  density_B=6.25e-4)   # about 140 row blocks of P: 5 chunks
    o = P.pdqp_default_options(precision=precision, max_iter=64, eps=0.0)
    h = G.handle(inst)
    try:
        runs = [P.pdqp_solve(h, o)[1] for _ in range(3)]
    finally:
        P.pdqp_destroy(h)
    keys = [(i.norm_A, i.norm_Q, i.norm_iters) for i in runs]
    assert keys[0][2] > 8 and keys[0] == keys[1] == keys[2]
    hb = P.batch_from_instances([inst, inst])
    try:
        P.pdqp_solve(hb, o)
        infos = P.pdqp_batch_info(hb)
    finally:
        P.pdqp_destroy(hb)
    assert [(i.norm_A, i.norm_Q, i.norm_iters) for i in infos] == [keys[0], keys[0]]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batch_norms_match_standalone_when_estimates_finish_apart(pdqp, precision):
    """Late in a batch's estimates the Lanczos steps run over the row blocks of
    the instances still estimating only; the norms stay bitwise those of the
    standalone solves: control QPs whose estimates stop many steps apart."""
    import qpgen
    from paper_2311_07710_gb300 import pdqp as P
    insts = qpgen.mpc_batch(48, seed=qpgen.SEED_BASE + 7411)
    o = P.pdqp_default_options(precision=precision, max_iter=64, eps=0.0)
    hb = P.batch_from_instances(insts)
    try:
        P.pdqp_solve(hb, o)
        infos = P.pdqp_batch_info(hb)
    finally:
        P.pdqp_destroy(hb)
    steps = [i.norm_iters for i in infos]
    assert max(steps) - min(steps) >= 24          # the batch runs compacted steps at its end
    order = sorted(range(len(insts)), key=lambda k: steps[k])
    for k in (order[0], order[len(order) // 2], order[-1]):
        h = G.handle(insts[k])
        try:
            info = P.pdqp_solve(h, o)[1]
        finally:
            P.pdqp_destroy(h)
        assert (info.norm_A, info.norm_Q, info.norm_iters) == (infos[k].norm_A, infos[k].norm_Q, infos[k].norm_iters)
