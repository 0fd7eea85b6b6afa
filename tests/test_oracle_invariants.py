"""Invariants of the oracle that its pins on end states cannot see.

* R10's stop test is relative, so Lanczos is scale-invariant: on c M it takes
  the steps it takes on M and returns c times the value.
* The start point is projected (x onto X, y onto Y) before the first
  iteration: a start outside X or Y gives the iterates of its projection.
* relKKT is measured on the original problem (R6): every check's recorded
  relKKT equals that of the traced iterate, unscaled, on the original data."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R


@pytest.mark.parametrize("c", [1e-4, 1e6])
def test_lanczos_is_scale_invariant(c):
    rng = np.random.default_rng(5)
    B = rng.standard_normal((60, 40))
    M = B.T @ B
    R.lanczos_max_eig(lambda v: M @ v, 40, tol=1e-6, name="M")
    steps, val = R.NORM_STEPS["M"], R.lanczos_max_eig(lambda v: M @ v, 40, tol=1e-6, name="M")
    val_c = R.lanczos_max_eig(lambda v: (c * M) @ v, 40, tol=1e-6, name="cM")
    assert R.NORM_STEPS["cM"] == steps
    assert val_c == pytest.approx(c * val, rel=1e-12)


def test_start_point_is_projected():
    inst = qpgen.tiny_qp(61, n=6, m=4, m_eq=2, bounds="box")
    rng = np.random.default_rng(6)
    x0 = rng.uniform(-30, 30, inst.n)                    # far outside the box
    y0 = rng.uniform(-3, 3, inst.m)                      # inequality entries of both signs
    xp = np.clip(x0, inst.l, inst.u)
    yp = y0.copy()
    yp[inst.m_eq:] = np.maximum(yp[inst.m_eq:], 0.0)
    o = R.Options(max_iter=20, eps=0.0, check_period=8)
    a = R.solve(inst, o, x0=x0, y0=y0, trace_at=range(1, 21))
    b = R.solve(inst, o, x0=xp, y0=yp, trace_at=range(1, 21))
    for t in range(1, 21):
        for key in ("x", "y", "xbar", "ybar"):
            np.testing.assert_array_equal(a.trace[t][key], b.trace[t][key])


def test_checks_measure_the_original_problem():
    inst = qpgen.tiny_qp(62, n=8, m=5, m_eq=2, bounds="mixed")
    p = R.problem_from_instance(inst)
    r = R.solve(inst, R.Options(eps=1e-9, check_period=16), trace_at=range(16, 2000, 16))
    D = r.D1, r.D2
    assert np.max(np.abs(D[0] - 1)) > 1e-3 or np.max(np.abs(D[1] - 1)) > 1e-3     # scaling is active
    for c in r.checks:
        st = r.trace.get(c["total"])
        if st is None:
            continue
        assert c["kkt_cur"] == pytest.approx(R.rel_kkt(p, st["x"], st["y"]), rel=1e-12)
        assert c["kkt_avg"] == pytest.approx(R.rel_kkt(p, st["xbar"], st["ybar"]), rel=1e-12)
