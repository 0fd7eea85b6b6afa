"""Theorem 1's claim on the oracle: with the theory step schedule and restarts
at a fixed frequency K, the method converges linearly -- relKKT at the restart
points falls by at least a constant factor per restart, not at a slowing
(sublinear) rate."""
import pytest

import qpgen
from oracle import rapdhg as R


@pytest.mark.parametrize("K", [128, 256])
def test_fixed_frequency_restarts_converge_linearly(K):
    inst = qpgen.tiny_qp(91, n=6, m=4, m_eq=1, bounds="box", q_rank=3)
    r = R.solve(inst, R.Options(step_rule="theory", restart_rule="fixed", fixed_K=K, eps=1e-11,
                                max_iter=200_000, check_period=K))
    assert r.status == "optimal"
    at_restarts = [c["kkt_avg"] for c in r.checks if c["restart"]]
    assert len(at_restarts) >= 8
    ratios = [b / a for a, b in zip(at_restarts, at_restarts[1:])]
    assert max(ratios) <= 0.5, ratios           # a constant factor every restart
