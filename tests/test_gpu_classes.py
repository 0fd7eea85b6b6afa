"""Lasso, Huber and SVM instances solved on the GPU in float64 and in mixed
precision: every solve ends at relKKT <= 1e-6 recomputed by the oracle on
the returned point, with the objective of the oracle's solution within
relative 1e-6; float64 solves take the oracle's iterations within one check
period."""
import functools

import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

GENS = {"lasso": qpgen.lasso_qp, "huber": qpgen.huber_qp, "svm": qpgen.svm_qp}


@functools.lru_cache(maxsize=None)
def case(name):
    inst = GENS[name]()
    return inst, R.solve(inst, R.Options(eps=1e-6))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", sorted(GENS))
def test_class_reaches_the_oracles_end_state(name, precision):
    pd = G.lib()
    inst, ref = case(name)
    st, info, x, y = G.solve(inst, precision=precision)
    assert st == pd.PDQP_OK
    parts = R.kkt_parts(R.problem_from_instance(inst), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6
    obj = ref.kkt["primal_obj"]
    assert abs(parts["primal_obj"] - obj) <= 1e-6 * (1 + abs(obj))
    if precision == 0:
        assert abs(info.iterations - ref.iterations) <= 64
