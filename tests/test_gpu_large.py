"""The n = 1e6 large sparse QP at full size, in the launch configuration the
bench times (default options, float64 and mixed precision).

The oracle cannot redo this solve inside a test, so the checks are: the first
iterations element by element (oracle iterations are cheap; preconditioning
off and fixed norms on both sides so the oracle skips its expensive setup),
the relative KKT error the oracle computes on the returned point, and the
objective and sampled entries of the oracle's stored full solve
(tests/golden/large_sparse_qp_reference.json, written by the script beside it)."""
import json
import os

import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

REF = os.path.join(os.path.dirname(__file__), "golden", "large_sparse_qp_reference.json")


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


@pytest.fixture(scope="module")
def inst():
    return qpgen.large_sparse_qp()


@pytest.fixture(scope="module")
def ref():
    return json.load(open(REF))


def test_first_iterations_elementwise_at_full_size(pdqp, inst):
    opts = dict(scaling=False, norm_A=8.0, norm_Q=30.0, check_period=64)
    oref = R.solve(inst, R.Options(max_iter=3, eps=0.0, scaling=False, norm_A=8.0, norm_Q=30.0),
                   trace_at=(1, 2, 3))
    for t in (1, 3):
        got = G.state_after(inst, t, **opts)
        for key in ("x", "y", "xbar", "ybar"):
            assert G.rel_err(got[key], oref.trace[t][key]) <= 1e-10, (t, key)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_full_solve_matches_oracle(pdqp, inst, ref, precision):
    st, info, x, y = G.solve(inst, device=True, precision=precision)
    assert st == pdqp.PDQP_OK
    parts = R.kkt_parts(R.problem_from_instance(inst), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6, parts
    obj = ref["kkt"]["primal_obj"]
    assert abs(parts["primal_obj"] - obj) <= 1e-6 * (1 + abs(obj))
    xs = np.array(ref["x_value"])
    err = np.max(np.abs(x[ref["x_index"]] - xs) / (1 + np.abs(xs)))
    print(f"precision {precision}: {info.iterations} iterations (oracle {ref['iterations']}), "
          f"relKKT {parts['rel_kkt']:.2e}, sampled x error {err:.2e}")
    if precision == 0:
        assert abs(info.iterations - ref["iterations"]) <= 64
        assert info.norm_A == pytest.approx(ref["norm_A"], rel=1e-5)
