"""The GPU's Lanczos norms on the operators the all-ones start vector fails
on (a regularised path-graph Laplacian Q, a difference-constraint A whose rows
sum to zero): the norms of the scaled matrices against dense eigen-solves of
the same scaled matrices (the oracle's scaling factors), and both problems
solved to the oracle's end state in both precisions."""
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
