"""Objectives with a low-rank term, Q_total = Q + F F' (F applied as F(F'x)),
against the oracle, which applies the same F F' in float64."""
import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


def _lowrank_tiny(seed=3, n=30, m=6, r=4):
    inst = qpgen.tiny_qp(seed, n=n, m=m, m_eq=2, bounds="mixed", density=0.4)
    rng = np.random.default_rng(seed)
    inst.F = (0.5 * rng.standard_normal((n, r))).astype(np.float32)
    return inst


def test_lowrank_iterates_match_oracle(pdqp):
    inst = _lowrank_tiny()
    ref = R.solve(inst, R.Options(max_iter=200, eps=0.0), trace_at=(1, 64, 65, 200))
    for t in (1, 64, 65, 200):
        got = G.state_after(inst, t, norm_A=ref.norm_A, norm_Q=ref.norm_Q)
        for key in ("x", "y", "xbar", "ybar"):
            assert G.rel_err(got[key], ref.trace[t][key]) <= 1e-10, (t, key)


def test_lowrank_lanczos_norm_includes_the_factor(pdqp):
    inst = _lowrank_tiny()
    ref = R.solve(inst, R.Options(max_iter=1, eps=0.0))
    st, info, x, y = G.solve(inst, max_iter=1, eps=0.0)
    assert info.norm_Q == pytest.approx(ref.norm_Q, rel=1e-9)
    assert info.norm_A == pytest.approx(ref.norm_A, rel=1e-9)


def test_lowrank_kkt_entry_point(pdqp):
    inst = _lowrank_tiny()
    rng = np.random.default_rng(1)
    x = np.clip(rng.normal(size=inst.n), inst.l, inst.u)
    y = rng.normal(size=inst.m)
    y[inst.m_eq:] = np.abs(y[inst.m_eq:])
    h = G.handle(inst)
    try:
        got = pdqp.pdqp_kkt(h, x, y)
    finally:
        pdqp.pdqp_destroy(h)
    ref = R.kkt_parts(R.problem_from_instance(inst), x, y)
    for k, key in enumerate(("r_primal", "r_dual", "r_gap", "rel_kkt", "primal_obj", "dual_obj")):
        assert got[k] == pytest.approx(ref[key], rel=1e-12, abs=1e-13), key


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_small_portfolio_end_state(pdqp, precision):
    inst = qpgen.portfolio_qp(n=2000, r=16)
    st, info, x, y = G.solve(inst, precision=precision)
    assert st == pdqp.PDQP_OK
    p = R.problem_from_instance(inst)
    parts = R.kkt_parts(p, x, y)
    ref = R.solve(inst, R.Options())
    assert parts["rel_kkt"] <= 1.0001e-6, parts
    obj = ref.kkt["primal_obj"]
    assert abs(parts["primal_obj"] - obj) <= 1e-6 * (1 + abs(obj))
    assert abs(x.sum() - 1.0) <= 1e-5 and np.all(x >= 0) and np.all(x <= 0.05)


def test_full_portfolio_relkkt(pdqp):
    """n = 1e5 assets, rank-64 factor, two dense rows: the oracle's relKKT of the
    returned point."""
    inst = qpgen.portfolio_qp()
    st, info, x, y = G.solve(inst, precision=1)
    assert st == pdqp.PDQP_OK
    parts = R.kkt_parts(R.problem_from_instance(inst), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6, parts
    print(f"portfolio n=1e5: {info.iterations} iterations, {info.seconds * 1e3:.1f} ms, relKKT {parts['rel_kkt']:.2e}")
