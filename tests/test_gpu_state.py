"""Checkpoint and resume through the C ABI (pdqp_get_state / pdqp_set_state).

A solve stopped by the iteration limit, saved, loaded into a fresh handle of
the same problem and continued must follow the uninterrupted solve bit for
bit: the iterates, the averages, the restart decisions of Section 6 (anchor
relKKT, previous candidate, epoch counters, primal weight) and the step sizes
tabulated for the check period it stopped in.  Stops both in the middle of a
check period and exactly at a check; float64 and mixed precision; a batch whose
instances stop at different checks.  In float64 the resumed iterate also meets
the oracle's trace to the parity bar."""
import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


@pytest.fixture(scope="module")
def cfg0():
    return qpgen.random_sparse_qp()


@pytest.fixture(scope="module")
def cfg0_trace(cfg0):
    return R.solve(cfg0, R.Options(max_iter=600, eps=0.0), trace_at=(600,))


def _iterates(pdqp, h, inst):
    out = [np.zeros(inst.n), np.zeros(inst.m), np.zeros(inst.n), np.zeros(inst.m)]
    pdqp.pdqp_get_iterates(h, *out)
    return out


def _solve(pdqp, h, n, m, **opts):
    x, y = np.zeros(n), np.zeros(m)
    st, info = pdqp.pdqp_solve(h, pdqp.pdqp_default_options(**opts), x_out=x, y_out=y)
    return st, info, x, y


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("stop", [300, 320])      # mid-period (300 = 4 * 64 + 44) and at a check
def test_resume_follows_the_uninterrupted_solve(pdqp, cfg0, cfg0_trace, precision, stop):
    inst = cfg0
    common = dict(eps=0.0, precision=precision, norm_A=cfg0_trace.norm_A, norm_Q=cfg0_trace.norm_Q)
    ha, hb, hc = G.handle(inst), G.handle(inst), G.handle(inst)
    try:
        st_a, info_a, _, _ = _solve(pdqp, ha, inst.n, inst.m, max_iter=600, **common)
        want = _iterates(pdqp, ha, inst)
        st_b, info_b, _, _ = _solve(pdqp, hb, inst.n, inst.m, max_iter=stop, **common)
        assert st_b == pdqp.PDQP_ITER_LIMIT and info_b.iterations == stop
        blob = pdqp.pdqp_get_state(hb)
        pdqp.pdqp_set_state(hc, blob)
        st_c, info_c, _, _ = _solve(pdqp, hc, inst.n, inst.m, max_iter=600, **common)
        got = _iterates(pdqp, hc, inst)
    finally:
        for h in (ha, hb, hc):
            pdqp.pdqp_destroy(h)
    assert st_c == st_a == pdqp.PDQP_ITER_LIMIT
    assert info_c.iterations == info_a.iterations == 600
    assert info_c.restarts == info_a.restarts and info_c.omega == info_a.omega
    for k, (g, w) in enumerate(zip(got, want)):
        np.testing.assert_array_equal(g, w, err_msg=f"field {k}")
    if precision == 0:
        for key, g in zip(("x", "y", "xbar", "ybar"), got):
            assert G.rel_err(g, cfg0_trace.trace[600][key]) <= ITER_TOL, key


def test_resume_to_optimality_returns_the_same_answer(pdqp, cfg0):
    inst = cfg0
    ha, hb, hc = G.handle(inst), G.handle(inst), G.handle(inst)
    try:
        st_a, info_a, xa, ya = _solve(pdqp, ha, inst.n, inst.m)
        assert st_a == pdqp.PDQP_OK
        stop = info_a.iterations // 2 + 7
        st_b, _, _, _ = _solve(pdqp, hb, inst.n, inst.m, max_iter=stop)
        assert st_b == pdqp.PDQP_ITER_LIMIT
        pdqp.pdqp_set_state(hc, pdqp.pdqp_get_state(hb))
        st_c, info_c, xc, yc = _solve(pdqp, hc, inst.n, inst.m)
    finally:
        for h in (ha, hb, hc):
            pdqp.pdqp_destroy(h)
    assert st_c == pdqp.PDQP_OK
    assert info_c.iterations == info_a.iterations and info_c.rel_kkt == info_a.rel_kkt
    np.testing.assert_array_equal(xc, xa)
    np.testing.assert_array_equal(yc, ya)


@pytest.mark.parametrize("back", [20, 64])      # stop mid-period, or at a check
def test_batch_resume_with_instances_stopping_at_different_checks(pdqp, back):
    """Instances the iteration limit stopped follow the uninterrupted solve;
    one that met the tolerance at the stop (the check forced by max_iter)
    keeps that answer, and the others that had finished before stay put."""
    from paper_2311_07710_gb300 import pdqp as P
    insts = qpgen.mpc_batch(6, seed=qpgen.SEED_BASE + 77)
    N, M = sum(i.n for i in insts), sum(i.m for i in insts)
    xo = np.cumsum([0] + [i.n for i in insts])
    yo = np.cumsum([0] + [i.m for i in insts])
    mk = lambda: P.batch_from_instances(insts)
    ha, hb, hc = mk(), mk(), mk()
    try:
        st_a, _, xa, ya = _solve(P, ha, N, M, precision=1)
        infos_a = P.pdqp_batch_info(ha)
        its = sorted(i.iterations for i in infos_a)
        assert its[0] < its[-1]                       # the instances stop at different checks
        stop = its[len(its) // 2] - back              # some finished, the rest stopped by the limit
        _, _, xb, yb = _solve(P, hb, N, M, precision=1, max_iter=stop)
        infos_b = P.pdqp_batch_info(hb)
        P.pdqp_set_state(hc, P.pdqp_get_state(hb))
        st_c, _, xc, yc = _solve(P, hc, N, M, precision=1)
        infos_c = P.pdqp_batch_info(hc)
    finally:
        for h in (ha, hb, hc):
            P.pdqp_destroy(h)
    assert st_c == st_a == P.PDQP_OK
    resumed = 0
    for i in range(len(insts)):
        sx, sy = slice(xo[i], xo[i + 1]), slice(yo[i], yo[i + 1])
        if infos_b[i].status == P.PDQP_ITER_LIMIT:
            resumed += 1
            assert infos_c[i].iterations == infos_a[i].iterations, i
            np.testing.assert_array_equal(xc[sx], xa[sx])
            np.testing.assert_array_equal(yc[sy], ya[sy])
        else:
            assert infos_b[i].status == P.PDQP_OK
            assert infos_c[i].iterations == infos_b[i].iterations, i
            np.testing.assert_array_equal(xc[sx], xb[sx])
            np.testing.assert_array_equal(yc[sy], yb[sy])
    assert resumed >= 2


def test_state_calls_reject_what_does_not_fit(pdqp, cfg0):
    other = qpgen.tiny_qp(8, n=30, m=20, m_eq=5, bounds="mixed")
    h, g, k = G.handle(cfg0), G.handle(other), G.handle(cfg0)
    try:
        with pytest.raises(pdqp.PdqpError):
            pdqp.pdqp_get_state(h)                    # no solve yet
        _solve(pdqp, h, cfg0.n, cfg0.m, max_iter=100)
        blob = pdqp.pdqp_get_state(h)
        with pytest.raises(pdqp.PdqpError):
            pdqp.pdqp_set_state(g, blob)              # another problem
        with pytest.raises(pdqp.PdqpError):
            pdqp.pdqp_set_state(k, blob[: len(blob) // 2])   # truncated
        bad = bytearray(blob)
        bad[0] ^= 0xFF
        with pytest.raises(pdqp.PdqpError):
            pdqp.pdqp_set_state(k, bytes(bad))        # not a state
        pdqp.pdqp_set_state(k, blob)
        with pytest.raises(pdqp.PdqpError):
            _solve(pdqp, k, cfg0.n, cfg0.m, check_period=32)     # other check period
        pdqp.pdqp_set_state(k, blob)
        with pytest.raises(pdqp.PdqpError):
            _solve(pdqp, k, cfg0.n, cfg0.m, max_iter=50)         # max_iter not beyond the state
        pdqp.pdqp_set_state(k, blob)
        st, info, _, _ = _solve(pdqp, k, cfg0.n, cfg0.m)        # loaded again: resumes
        assert st == pdqp.PDQP_OK and info.iterations > 100
    finally:
        for x in (h, g, k):
            pdqp.pdqp_destroy(x)
