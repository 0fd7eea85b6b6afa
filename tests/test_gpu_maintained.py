"""Maintained products (options.maintained_products, float64): the iteration
carries A x, A x_bar, Q x_bar, A'y and A'y_bar with the iterates (the
updates of Algorithm 1 are linear, Section 2), so a check gathers x once for
A x and once for Q x and the next iteration starts from those products.

In exact arithmetic the iterates are those of the direct products; the
rounding differs, so they are held to the float64 path's bar against the
oracle (relative 1e-10 over the first 200 iterations, through restarts and
every restart and step variant), solves to the oracle's end-state bar, and a
batch, a family handle and graph replay reproduce the standalone solves bit
for bit.  What the option cannot run is refused with PDQP_ERR_INVALID."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R
from tests import gpu_util as G
from tests.test_oracle_infeasibility import DUAL_INFEASIBLE, PRIMAL_INFEASIBLE, _check_farkas, _check_ray

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
CHECKPOINTS = (1, 2, 3, 10, 63, 64, 65, 100, 128, 129, 150, 192, 199, 200)
MP = dict(maintained_products=1)


@pytest.fixture(scope="module")
def pdqp():
    return G.lib()


@pytest.fixture(scope="module")
def cfg0():
    return qpgen.random_sparse_qp()


@pytest.fixture(scope="module")
def cfg0_oracle(cfg0):
    return R.solve(cfg0, R.Options(max_iter=200, eps=0.0), trace_at=CHECKPOINTS)


@pytest.mark.parametrize("t", CHECKPOINTS)
def test_iterates_match_oracle(pdqp, cfg0, cfg0_oracle, t):
    ref = cfg0_oracle.trace[t]
    got = G.state_after(cfg0, t, norm_A=cfg0_oracle.norm_A, norm_Q=cfg0_oracle.norm_Q, **MP)
    for key in ("x", "y", "xbar", "ybar"):
        assert G.rel_err(got[key], ref[key]) <= ITER_TOL, (t, key, G.rel_err(got[key], ref[key]))


def test_restart_decisions_match_over_600_iterations(pdqp, cfg0):
    ref = R.solve(cfg0, R.Options(max_iter=600, eps=0.0), trace_at=(600,))
    got = G.state_after(cfg0, 600, norm_A=ref.norm_A, norm_Q=ref.norm_Q, **MP)
    for key in ("x", "y", "xbar", "ybar"):
        assert G.rel_err(got[key], ref.trace[600][key]) <= 1e-9, key


@pytest.mark.parametrize("variant", ["halving", "fixed", "none_pdhg", "theory", "noscale", "warm", "eq_only"])
def test_variant_iterates_match_oracle(pdqp, variant):
    """Every restart and step variant, from zero and from a given start, at
    partial chunks (t not a multiple of the check period) and across restarts."""
    from paper_2311_07710_gb300 import pdqp as P
    inst = qpgen.tiny_qp(5, n=37, m=29, m_eq=29 if variant == "eq_only" else 9, bounds="mixed", density=0.3)
    ro = dict(halving=R.Options(restart_rule="halving"), fixed=R.Options(restart_rule="fixed", fixed_K=64),
              none_pdhg=R.Options(restart_rule="none", accelerate=False),
              theory=R.Options(step_rule="theory", restart_rule="fixed", fixed_K=64),
              noscale=R.Options(scaling=False), warm=R.Options(), eq_only=R.Options())[variant]
    go = dict(halving=dict(restart_rule=1), fixed=dict(restart_rule=2, fixed_K=64),
              none_pdhg=dict(restart_rule=3, accelerate=0), theory=dict(step_rule=1, restart_rule=2, fixed_K=64),
              noscale=dict(scaling=0), warm={}, eq_only={})[variant]
    ro.max_iter, ro.eps, ro.check_period = 300, 0.0, 32
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-1, 1, inst.n) if variant == "warm" else None
    y0 = rng.uniform(-1, 1, inst.m) if variant == "warm" else None
    ref = R.solve(inst, ro, x0=x0, y0=y0, trace_at=(1, 33, 100, 300))
    for t in (1, 33, 100, 300):
        h = G.handle(inst)
        try:
            o = P.pdqp_default_options(max_iter=t, eps=0.0, check_period=32, norm_A=ref.norm_A,
                                       norm_Q=ref.norm_Q, **go, **MP)
            P.pdqp_solve(h, o, x0=x0, y0=y0)
            out = [np.zeros(inst.n), np.zeros(inst.m), np.zeros(inst.n), np.zeros(inst.m)]
            P.pdqp_get_iterates(h, *out)
        finally:
            P.pdqp_destroy(h)
        for key, v in zip(("x", "y", "xbar", "ybar"), out):
            assert G.rel_err(v, ref.trace[t][key]) <= ITER_TOL, (variant, t, key, G.rel_err(v, ref.trace[t][key]))


def test_solves_to_oracle_end_state(pdqp, cfg0):
    """To 1e-6 from zero: relKKT recomputed by the oracle on the returned point,
    the objective of the oracle's solve, the iteration count of the direct
    products' solve (the decisions are the same up to rounding)."""
    ref = R.solve(cfg0, R.Options())
    st, info, x, y = G.solve(cfg0, **MP)
    st0, info0, _, _ = G.solve(cfg0)
    assert st == st0 == pdqp.PDQP_OK
    parts = R.kkt_parts(R.problem_from_instance(cfg0), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6
    assert info.rel_kkt == pytest.approx(parts["rel_kkt"], rel=1e-6, abs=1e-12)
    assert abs(parts["primal_obj"] - ref.kkt["primal_obj"]) <= 1e-6 * (1 + abs(ref.kkt["primal_obj"]))
    assert abs(info.iterations - info0.iterations) <= 64
    assert info.spmv_threads == 256


def test_check_values_match_direct_products(pdqp, cfg0):
    """The relKKT a check forms from the maintained products equals the
    oracle's relKKT of the same iterate (original problem, direct products)."""
    from paper_2311_07710_gb300 import pdqp as P
    p = R.problem_from_instance(cfg0)
    for t in (64, 192):
        h = G.handle(cfg0)
        try:
            # the iteration limit ends the solve at that check with its candidate
            st, info = P.pdqp_solve(h, P.pdqp_default_options(max_iter=t, eps=0.0, **MP))
            out = [np.zeros(cfg0.n), np.zeros(cfg0.m), np.zeros(cfg0.n), np.zeros(cfg0.m)]
            P.pdqp_get_iterates(h, *out)
        finally:
            P.pdqp_destroy(h)
        assert st == pdqp.PDQP_ITER_LIMIT
        cur = R.kkt_parts(p, out[0], out[1])["rel_kkt"]
        avg = R.kkt_parts(p, out[2], out[3])["rel_kkt"]
        assert info.rel_kkt == pytest.approx(min(cur, avg), rel=1e-8), t


def test_device_buffers_and_graphs_reproduce_direct_launches(pdqp, cfg0):
    a = G.solve(cfg0, **MP)
    b = G.solve(cfg0, no_graphs=1, **MP)
    c = G.solve(cfg0, device=True, **MP)
    for other in (b, c):
        assert other[0] == a[0] and other[1].iterations == a[1].iterations
        np.testing.assert_array_equal(other[2], a[2])
        np.testing.assert_array_equal(other[3], a[3])


def _solve_batch(pdqp, insts, **opts):
    h = pdqp.batch_from_instances(insts)
    try:
        N, M = sum(i.n for i in insts), sum(i.m for i in insts)
        x, y = np.zeros(N), np.zeros(M)
        st, _ = pdqp.pdqp_solve(h, pdqp.pdqp_default_options(**opts), x_out=x, y_out=y)
        infos = pdqp.pdqp_batch_info(h)
    finally:
        pdqp.pdqp_destroy(h)
    xs, ys, ox, oy = [], [], 0, 0
    for i in insts:
        xs.append(x[ox:ox + i.n]); ys.append(y[oy:oy + i.m])
        ox += i.n; oy += i.m
    return st, infos, xs, ys


def test_batch_reproduces_standalone_solves(pdqp):
    """Instances of uneven sizes (one without rows) that stop at different
    checks, so that later chunks run compacted over the running row blocks."""
    insts = [qpgen.tiny_qp(40 + k, n=5 + 7 * k, m=3 + 5 * k, m_eq=k, bounds=("box", "mixed", "lower")[k % 3],
                           density=0.5) for k in range(6)]
    insts += [qpgen.diagonal_box_qp(99, 17), qpgen.random_sparse_qp()]
    insts += [qpgen.mpc_qp(7 + k, T=10 + 9 * k) for k in range(3)]
    st, infos, xs, ys = _solve_batch(pdqp, insts, **MP)
    assert st == pdqp.PDQP_OK
    assert len({i.iterations for i in infos}) > 2
    for k, inst in enumerate(insts):
        s1, info1, x1, y1 = G.solve(inst, **MP)
        assert infos[k].status == s1 and infos[k].iterations == info1.iterations, k
        np.testing.assert_array_equal(xs[k], x1)
        np.testing.assert_array_equal(ys[k], y1)
        parts = R.kkt_parts(R.problem_from_instance(inst), xs[k], ys[k])
        assert parts["rel_kkt"] <= 1.0001e-6, k


def test_family_handle_reproduces_batch(pdqp):
    """A family handle runs the row-block kernels with maintained products and
    gives the batch handle's results bit for bit, from a given start."""
    fam = qpgen.family_qp(n=300, m=150)
    C, B = fam.params(0, 5)
    insts = [qpgen.QPInstance("member", fam.base.n, fam.base.m, fam.base.m_eq, fam.base.Q, fam.base.A, C[k], B[k],
                              fam.base.l, fam.base.u) for k in range(5)]
    N, M = 5 * fam.base.n, 5 * fam.base.m
    rng = np.random.default_rng(1)
    x0, y0 = 0.1 * rng.standard_normal(N), 0.1 * rng.standard_normal(M)
    out = []
    for make in (lambda: pdqp.batch_from_instances(insts), lambda: pdqp.family_from_base(fam.base, C, B)):
        h = make()
        try:
            x, y = np.zeros(N), np.zeros(M)
            st, info = pdqp.pdqp_solve(h, pdqp.pdqp_default_options(**MP), x0=x0, y0=y0, x_out=x, y_out=y)
            out.append((st, [(i.status, i.iterations) for i in pdqp.pdqp_batch_info(h)], x, y, info.spmv_threads))
        finally:
            pdqp.pdqp_destroy(h)
    assert out[0][0] == out[1][0] == pdqp.PDQP_OK
    assert out[1][4] == 256
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_array_equal(out[0][3], out[1][3])


CERT_CASES = [(n, i, "primal") for n, i in sorted(PRIMAL_INFEASIBLE.items())] + \
             [(n, i, "dual") for n, i in sorted(DUAL_INFEASIBLE.items())]


@pytest.mark.parametrize("name,inst,kind", CERT_CASES, ids=[c[0] for c in CERT_CASES])
def test_certificates_match_the_oracle(pdqp, name, inst, kind):
    """Certificates come from the iterates: the oracle's certificate, at its
    iteration, within the float64 path's bar."""
    ref = R.solve(inst, R.Options(detect_infeasibility=True, max_iter=5000))
    st, info, x, y = G.solve(inst, detect_infeasibility=1, max_iter=5000, norm_A=ref.norm_A, norm_Q=ref.norm_Q,
                             **MP)
    want = pdqp.PDQP_PRIMAL_INFEASIBLE if kind == "primal" else pdqp.PDQP_DUAL_INFEASIBLE
    assert st == want and info.iterations == ref.iterations
    assert G.rel_err(x, ref.x) <= 1e-10 and G.rel_err(y, ref.y) <= 1e-10
    (_check_farkas(inst, y) if kind == "primal" else _check_ray(inst, x))


def test_refusals(pdqp, cfg0):
    from paper_2311_07710_gb300 import pdqp as P

    def refused(inst, **opts):
        h = G.handle(inst)
        try:
            with pytest.raises(P.PdqpError) as e:
                P.pdqp_solve(h, P.pdqp_default_options(**opts))
            assert e.value.status == P.PDQP_ERR_INVALID
        finally:
            P.pdqp_destroy(h)

    refused(cfg0, precision=1, **MP)                  # float32 products
    refused(cfg0, spmv_threads=512, **MP)
    refused(cfg0, spmv_threads=2, **MP)
    refused(cfg0, maintained_products=2)
    refused(qpgen.portfolio_qp(n=500, r=4), **MP)     # low-rank term
    n, m = 30, 3000
    A = sp.random(m, n, density=0.05, random_state=5, format="csr")
    A = sp.csr_matrix(A + sp.csr_matrix((np.ones(m), (np.arange(m), np.zeros(m, int))), shape=(m, n)))
    A.sort_indices()
    rng = np.random.default_rng(5)
    long_col = qpgen.QPInstance("long_column", n, m, 0, sp.identity(n, format="csr"), A, rng.standard_normal(n),
                                A @ rng.uniform(-0.5, 0.5, n) - 1.0, -5 * np.ones(n), 5 * np.ones(n))
    refused(long_col, **MP)                           # row 0 of P holds 3000 nonzeros of A'
    # no resumable state after such a solve, and none to resume from
    h = G.handle(cfg0)
    try:
        P.pdqp_solve(h, P.pdqp_default_options(max_iter=100, **MP))
        with pytest.raises(P.PdqpError) as e:
            P.pdqp_get_state(h)
        assert e.value.status == P.PDQP_ERR_INVALID
        P.pdqp_solve(h, P.pdqp_default_options(max_iter=100))
        state = P.pdqp_get_state(h)
        P.pdqp_set_state(h, state)
        with pytest.raises(P.PdqpError) as e:
            P.pdqp_solve(h, P.pdqp_default_options(max_iter=200, **MP))
        assert e.value.status == P.PDQP_ERR_INVALID
    finally:
        P.pdqp_destroy(h)


def test_large_sparse_end_state(pdqp):
    """n = 1e5 of the large random sparse family: to 1e-6 with the direct
    products' iteration count, relKKT recomputed by the oracle."""
    inst = qpgen.large_sparse_qp(n=100_000)
    st, info, x, y = G.solve(inst, **MP)
    st0, info0, _, _ = G.solve(inst)
    assert st == st0 == pdqp.PDQP_OK
    assert abs(info.iterations - info0.iterations) <= 64
    parts = R.kkt_parts(R.problem_from_instance(inst), x, y)
    assert parts["rel_kkt"] <= 1.0001e-6
    assert abs(info.primal_obj - info0.primal_obj) <= 1e-5 * (1 + abs(info0.primal_obj))
