"""Infeasibility certificates on the GPU (optional detection, not in the
paper) against the oracle: in float64, with the oracle's spectral norms, the
same status at the same iteration and the same certificate to 1e-10; in mixed
precision the status, with the certificate checked against its defining
inequalities (support function by brute force); feasible solves unchanged;
a batch mixing feasible and infeasible instances ends each one as its
standalone solve does, bit for bit; so does a family handle (the certificate
passes on its replicated matrix, whose scaled values are copied from its
one-member template) against a batch of its members."""
import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G
from tests.test_oracle_infeasibility import (DUAL_INFEASIBLE, FEASIBLE, PRIMAL_INFEASIBLE, _check_farkas,
                                             _check_ray)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


def _gpu(pdqp, inst, **opts):
    return G.solve(inst, detect_infeasibility=1, max_iter=5000, **opts)


CASES = [(n, i, "primal") for n, i in sorted(PRIMAL_INFEASIBLE.items())] + \
        [(n, i, "dual") for n, i in sorted(DUAL_INFEASIBLE.items())]


@pytest.mark.parametrize("name,inst,kind", CASES, ids=[c[0] for c in CASES])
def test_fp64_certificate_matches_the_oracle(pdqp, name, inst, kind):
    ref = R.solve(inst, R.Options(detect_infeasibility=True, max_iter=5000))
    st, info, x, y = _gpu(pdqp, inst, norm_A=ref.norm_A, norm_Q=ref.norm_Q)
    want = pdqp.PDQP_PRIMAL_INFEASIBLE if kind == "primal" else pdqp.PDQP_DUAL_INFEASIBLE
    assert ref.status == ("primal_infeasible" if kind == "primal" else "dual_infeasible")
    assert st == want and info.status == want
    assert info.iterations == ref.iterations
    assert G.rel_err(x, ref.x) <= 1e-10 and G.rel_err(y, ref.y) <= 1e-10
    (_check_farkas(inst, y) if kind == "primal" else _check_ray(inst, x))


@pytest.mark.parametrize("name,inst,kind", CASES, ids=[c[0] for c in CASES])
def test_mixed_certificate_is_valid(pdqp, name, inst, kind):
    st, info, x, y = _gpu(pdqp, inst, precision=pdqp.PDQP_PREC_MIXED)
    if kind == "primal":
        assert st == pdqp.PDQP_PRIMAL_INFEASIBLE
        assert np.all(x == 0)
        _check_farkas(inst, y)
    else:
        assert st == pdqp.PDQP_DUAL_INFEASIBLE
        assert np.all(y == 0)
        _check_ray(inst, x)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("k", range(len(FEASIBLE)))
def test_detection_leaves_feasible_solves_alone(pdqp, k, precision):
    inst = FEASIBLE[k]
    a = G.solve(inst, precision=precision)
    b = _gpu(pdqp, inst, precision=precision)
    assert a[0] == b[0] == pdqp.PDQP_OK
    assert a[1].iterations == b[1].iterations
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batch_ends_each_instance_as_alone(pdqp, precision):
    insts = [FEASIBLE[0], PRIMAL_INFEASIBLE["box_lp"], DUAL_INFEASIBLE["ray_no_rows"], FEASIBLE[3],
             PRIMAL_INFEASIBLE["mixed"], qpgen.random_sparse_qp()]
    h = pdqp.batch_from_instances(insts)
    try:
        N, M = sum(i.n for i in insts), sum(i.m for i in insts)
        x, y = np.zeros(N), np.zeros(M)
        st, info = pdqp.pdqp_solve(h, pdqp.pdqp_default_options(precision=precision, detect_infeasibility=1,
                                                                max_iter=5000), x_out=x, y_out=y)
        infos = pdqp.pdqp_batch_info(h)
    finally:
        pdqp.pdqp_destroy(h)
    assert st == pdqp.PDQP_DUAL_INFEASIBLE        # the largest status of the batch
    ox = oy = 0
    for k, inst in enumerate(insts):
        s1, i1, x1, y1 = _gpu(pdqp, inst, precision=precision)
        assert infos[k].status == s1 and infos[k].iterations == i1.iterations, k
        np.testing.assert_array_equal(x[ox:ox + inst.n], x1)
        np.testing.assert_array_equal(y[oy:oy + inst.m], y1)
        ox += inst.n
        oy += inst.m
    assert [i.status for i in infos] == [pdqp.PDQP_OK, pdqp.PDQP_PRIMAL_INFEASIBLE, pdqp.PDQP_DUAL_INFEASIBLE,
                                        pdqp.PDQP_OK, pdqp.PDQP_PRIMAL_INFEASIBLE, pdqp.PDQP_OK]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_family_handle_with_certificates_reproduces_batch(pdqp, precision):
    fam = qpgen.family_qp(n=300, m=150)
    C, B = fam.params(0, 5)
    B[2, 0] = 1e4              # an equality row that no point of the box [-10, 10] meets
    insts = [qpgen.QPInstance("member", fam.base.n, fam.base.m, fam.base.m_eq, fam.base.Q, fam.base.A, C[k], B[k],
                              fam.base.l, fam.base.u) for k in range(5)]
    N, M = 5 * fam.base.n, 5 * fam.base.m
    o = pdqp.pdqp_default_options(precision=precision, detect_infeasibility=1, max_iter=5000)
    out = []
    for make in (lambda: pdqp.batch_from_instances(insts), lambda: pdqp.family_from_base(fam.base, C, B)):
        h = make()
        try:
            x, y = np.zeros(N), np.zeros(M)
            st, _ = pdqp.pdqp_solve(h, o, x_out=x, y_out=y)
            out.append((st, [(i.status, i.iterations) for i in pdqp.pdqp_batch_info(h)], x, y))
        finally:
            pdqp.pdqp_destroy(h)
    assert out[0][0] == out[1][0] == pdqp.PDQP_PRIMAL_INFEASIBLE
    assert [s for s, _ in out[1][1]] == [pdqp.PDQP_OK, pdqp.PDQP_OK, pdqp.PDQP_PRIMAL_INFEASIBLE, pdqp.PDQP_OK,
                                         pdqp.PDQP_OK]
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_array_equal(out[0][3], out[1][3])


def test_graph_replay_matches_direct_launches(pdqp):
    for inst in (PRIMAL_INFEASIBLE["eq_scaled"], DUAL_INFEASIBLE["ray_lp"], FEASIBLE[1]):
        a = _gpu(pdqp, inst, no_graphs=0)
        b = _gpu(pdqp, inst, no_graphs=1)
        assert a[0] == b[0] and a[1].iterations == b[1].iterations
        np.testing.assert_array_equal(a[2], b[2])
        np.testing.assert_array_equal(a[3], b[3])


def test_options_are_validated(pdqp):
    inst = FEASIBLE[2]
    for bad in (dict(detect_infeasibility=2), dict(detect_infeasibility=1, eps_infeasible=0.0),
                dict(detect_infeasibility=1, eps_infeasible=1.5)):
        with pytest.raises(pdqp.PdqpError) as e:
            G.solve(inst, **bad)
        assert e.value.status == pdqp.PDQP_ERR_INVALID
