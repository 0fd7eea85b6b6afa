"""Mixed precision (float32 iteration and SpMVs, float64 relKKT, restarts and
residual correction) against the CPU oracle.  Iterates are not comparable one
to one with the float64 oracle (different arithmetic), so the bar is the end
state: relative KKT <= 1e-6 recomputed by the oracle on the returned point and
the objective within relative 1e-6 of the oracle's."""
import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G
from tests.qp_truth import active_set_solve

pytestmark = pytest.mark.gpu

MIXED = 1


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


def _check_against_oracle(inst, x, y, eps=1e-6):
    p = R.problem_from_instance(inst)
    parts = R.kkt_parts(p, x, y)
    ref = R.solve(inst, R.Options(eps=eps))
    obj = ref.kkt["primal_obj"]
    assert parts["rel_kkt"] <= 1.0001 * eps, parts
    assert abs(parts["primal_obj"] - obj) <= 1e-6 * (1 + abs(obj))
    assert np.all(x >= inst.l) and np.all(x <= inst.u)
    assert np.all(y[inst.m_eq:] >= 0)
    return ref, parts


def test_config0_mixed_reaches_1e6(pdqp):
    inst = qpgen.random_sparse_qp()
    st, info, x, y = G.solve(inst, precision=MIXED)
    assert st == pdqp.PDQP_OK
    ref, parts = _check_against_oracle(inst, x, y)
    assert info.rel_kkt == pytest.approx(parts["rel_kkt"], rel=1e-6, abs=1e-12)
    err = np.max(np.abs(x - ref.x) / (1 + np.abs(ref.x)))
    print(f"mixed vs oracle: max |x - x*|/(1+|x*|) = {err:.2e}, iterations {info.iterations} vs {ref.iterations}")


def test_mixed_reaches_1e8(pdqp):
    """The float64 residual correction carries the float32 iteration below
    float32 resolution."""
    inst = qpgen.random_sparse_qp()
    st, info, x, y = G.solve(inst, precision=MIXED, eps=1e-8)
    assert st == pdqp.PDQP_OK
    assert R.kkt_parts(R.problem_from_instance(inst), x, y)["rel_kkt"] <= 1.0001e-8


@pytest.mark.parametrize("seed,n,m,m_eq,bounds", [
    (21, 4, 3, 1, "box"), (22, 5, 4, 2, "mixed"), (23, 6, 3, 0, "lower"), (25, 6, 4, 2, "mixed"),
])
def test_tiny_mixed_match_brute_force(pdqp, seed, n, m, m_eq, bounds):
    inst = qpgen.tiny_qp(seed, n=n, m=m, m_eq=m_eq, bounds=bounds)
    truth = active_set_solve(inst.Q.toarray(), inst.A.toarray(), inst.b, inst.c, inst.l, inst.u, m_eq)
    st, info, x, y = G.solve(inst, precision=MIXED, eps=1e-9)
    assert st == pdqp.PDQP_OK
    assert info.primal_obj == pytest.approx(truth[2], rel=1e-7, abs=1e-7)
    np.testing.assert_allclose(x, truth[0], atol=1e-5)


@pytest.mark.parametrize("n", [1, 257, 1000])
def test_mixed_box_closed_form(pdqp, n):
    inst = qpgen.diagonal_box_qp(300 + n, n)
    st, info, x, y = G.solve(inst, precision=MIXED, eps=1e-10)
    assert st == pdqp.PDQP_OK
    np.testing.assert_allclose(x, np.clip(-inst.c / inst.Q.diagonal(), inst.l, inst.u), atol=1e-8)


def test_mixed_mpc_instance(pdqp):
    inst = qpgen.mpc_qp(qpgen.SEED_BASE * 100003 + 3 * 100003 + 5)
    st, info, x, y = G.solve(inst, precision=MIXED)
    assert st == pdqp.PDQP_OK
    _check_against_oracle(inst, x, y)


def test_mixed_warm_start_from_solution_is_immediate(pdqp):
    inst = qpgen.random_sparse_qp()
    ref = R.solve(inst, R.Options(eps=1e-9))
    st, info, x, y = G.solve(inst, precision=MIXED, x0=ref.x, y0=ref.y)
    assert st == pdqp.PDQP_OK and info.iterations == 0
