"""Pins of the oracle's restart bookkeeping and of its l2 scaling pass.

* Section 6's rule, replayed from the oracle's own check records: the restart
  at every check follows conditions (i)-(iii) from the recorded relKKT of the
  current and average iterate, the anchor relKKT (which a restart resets to
  the candidate's) and the previous check's candidate in the same epoch
  (none at an epoch's first check).
* Algorithm 1's outer loop: a restart is a fresh start from the candidate.
  With Theorem 1's schedule (no primal-weight updates), fixed-frequency
  restarts and plain PDHG (theta = 1, so the extrapolation reads x_prev), the
  iterates after a restart equal those of a new solve started at the point
  restarted to.
* The l2 pass worked by hand: for Q = 0 and A = [3 4], K = [[0, A'], [A, 0]]
  has row 2-norms (3, 4, 5), so one pass from d = 1 gives D2 = (1/sqrt 3,
  1/2) and D1 = 1/sqrt 5 (an l1 pass would give 1/sqrt 7)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R

BETA_SUFF, BETA_NEC, BETA_ART = 0.2, 0.8, 0.36


# (seed, check period, bounds): the last three restart at a check whose previous
# candidate comes from the epoch before, where a stale value would change (ii)
@pytest.mark.parametrize("seed,period,bounds", [(91, 16, "mixed"), (92, 16, "mixed"), (93, 16, "mixed"),
                                                (88, 32, "mixed"), (90, 8, "mixed"), (88, 8, "lower")])
def test_restart_decisions_replay_from_the_records(seed, period, bounds):
    inst = qpgen.tiny_qp(seed, n=6, m=4, m_eq=1, bounds=bounds, q_rank=3)
    r = R.solve(inst, R.Options(eps=1e-9, check_period=period, max_iter=20000))
    assert r.status == "optimal"
    recs = r.checks
    assert sum(c["restart"] for c in recs) >= 3
    prev_cand = None
    anchor = None
    for c in recs[:-1]:                                   # the last check terminates
        cand = c["kkt_cur"] if c["kkt_cur"] < c["kkt_avg"] else c["kkt_avg"]
        if anchor is not None:
            assert c["anchor_kkt"] == anchor              # reset to the last restart's candidate
        a = c["anchor_kkt"]
        want = (cand <= BETA_SUFF * a
                or (prev_cand is not None and cand <= BETA_NEC * a and cand > prev_cand)
                or c["k"] >= BETA_ART * c["total"])
        assert bool(c["restart"]) == want, c
        if c["restart"]:
            prev_cand, anchor = None, cand
        else:
            prev_cand = cand


def test_restart_is_a_fresh_start_from_the_candidate():
    inst = qpgen.tiny_qp(94, n=5, m=3, m_eq=1, bounds="box")
    K = 8
    base = dict(step_rule="theory", restart_rule="fixed", fixed_K=K, accelerate=False, scaling=False,
                norm_A=3.0, norm_Q=4.0, eps=0.0, check_period=K)
    first = R.solve(inst, R.Options(max_iter=K, **base), trace_at=(K,))
    xc, yc = first.trace[K]["xbar"], first.trace[K]["ybar"]     # fixed restarts go to the average
    both = R.solve(inst, R.Options(max_iter=2 * K, **base), trace_at=range(K + 1, 2 * K + 1))
    fresh = R.solve(inst, R.Options(max_iter=K, **base), x0=xc, y0=yc, trace_at=range(1, K + 1))
    for j in range(1, K + 1):
        for key in ("x", "y", "xbar", "ybar"):
            np.testing.assert_allclose(both.trace[K + j][key], fresh.trace[j][key], rtol=1e-13, atol=1e-15)


def test_l2_pass_worked_by_hand():
    p = R.Problem(sp.csr_matrix((2, 2)), sp.csr_matrix(np.array([[3.0, 4.0]])), np.zeros(2), np.zeros(1),
                  np.zeros(2), np.ones(2), 0)
    D1, D2 = R.scaling_factors(p, ruiz_iters=0, l2=True, pock_chambolle=False)
    np.testing.assert_allclose(D2, [1 / math.sqrt(3), 0.5], rtol=1e-15)
    np.testing.assert_allclose(D1, [1 / math.sqrt(5)], rtol=1e-15)
