"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-worked
fractions, closed forms, a brute-force active-set enumeration, the KKT
conditions checked term by term, textbook special cases (accelerated gradient
for unconstrained QPs, constant-step PDHG for LPs) and the invariants Lemma 1
and Lemma 2 state for the step schedule.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R
from tests.qp_truth import active_set_solve, kkt_certificate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(v):
    if isinstance(v, str):
        if v in ("inf", "-inf"):
            return float(v)
        return float(Fraction(v))
    return float(v)


def _problem(d, l=None, u=None):
    Q = np.array(d["Q"], float)
    A = np.array(d["A"], float)
    n = Q.shape[0]
    l = np.array([_frac(v) for v in (l if l is not None else d["l"])])
    u = np.array([_frac(v) for v in (u if u is not None else d["u"])])
    return R.Problem(sp.csr_matrix(Q), sp.csr_matrix(A), np.array(d["c"], float),
                     np.array(d["b"], float), l, u, int(d["m_eq"]))


# --------------------------------------------------------------------------- golden
def test_hand_worked_first_three_iterations():
    """Algorithm 1 with Theorem 1's schedule, three iterations in exact fractions."""
    g = json.load(open(os.path.join(GOLDEN, "hand_three_iterations.json")))
    p = _problem(g["problem"])
    s = g["settings"]
    opts = R.Options(step_rule="theory", restart_rule="fixed", fixed_K=s["K"], scaling=False,
                     norm_Q=s["norm_Q"], norm_A=s["norm_A"], max_iter=3, check_period=1000, eps=0.0)
    res = R.solve(p, opts, trace_at=(1, 2, 3))
    for it, want in g["iterates"].items():
        got = res.trace[int(it)]
        for key in ("x", "y", "xbar", "ybar"):
            assert got[key][0] == pytest.approx(_frac(want[key]), rel=1e-14, abs=1e-15), (it, key)


def test_hand_worked_relkkt():
    g = json.load(open(os.path.join(GOLDEN, "hand_relkkt.json")))
    for case in g["cases"]:
        p = _problem(g["problem"], case["l"], case["u"])
        x = np.array([_frac(v) for v in case["x"]])
        y = np.array([_frac(v) for v in case["y"]])
        parts = R.kkt_parts(p, x, y)
        for key in ("r_primal", "r_dual", "r_gap", "rel_kkt", "primal_obj", "dual_obj"):
            assert parts[key] == pytest.approx(_frac(case[key]), rel=1e-13, abs=1e-14), key


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_diagonal_box_qp_closed_form(seed):
    """Diagonal Q, no rows: x* = clip(-c/q, l, u) exactly."""
    inst = qpgen.diagonal_box_qp(seed, 40)
    q = inst.Q.diagonal()
    want = np.clip(-inst.c / q, inst.l, inst.u)
    res = R.solve(inst, R.Options(eps=1e-10))
    assert res.status == "optimal"
    np.testing.assert_allclose(res.x, want, atol=1e-8)


def test_unconstrained_quadratic_is_accelerated_gradient():
    """m = 0, free bounds: the minimiser of 1/2 x'Qx + c'x is -Q^{-1} c."""
    inst = qpgen.tiny_qp(7, n=10, m=1, m_eq=0, bounds="free")
    p = R.problem_from_instance(inst)
    p = R.Problem(p.Q, sp.csr_matrix((0, 10)), p.c, np.zeros(0), p.l, p.u, 0)
    want = np.linalg.solve(p.Q.toarray(), -p.c)
    res = R.solve(p, R.Options(eps=1e-10))
    assert res.status == "optimal"
    np.testing.assert_allclose(res.x, want, rtol=1e-7, atol=1e-7)


def test_equality_qp_kkt_linear_system():
    """Free variables and equality rows only: [[Q, -A'], [A, 0]] [x; y] = [-c; b]."""
    inst = qpgen.tiny_qp(11, n=8, m=3, m_eq=3, bounds="free")
    Q, A = inst.Q.toarray(), inst.A.toarray()
    K = np.block([[Q, -A.T], [A, np.zeros((3, 3))]])
    sol = np.linalg.solve(K, np.concatenate([-inst.c, inst.b]))
    res = R.solve(inst, R.Options(eps=1e-10))
    assert res.status == "optimal"
    np.testing.assert_allclose(res.x, sol[:8], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(res.y, sol[8:], rtol=1e-6, atol=1e-7)


def test_tiny_lp_vertex():
    """Q = 0: min -x1 - x2 s.t. x1 + 2 x2 <= 4, 3 x1 + x2 <= 6, x >= 0 has the
    unique vertex solution (8/5, 6/5), objective -14/5."""
    A = sp.csr_matrix(np.array([[-1.0, -2.0], [-3.0, -1.0]]))
    p = R.Problem(sp.csr_matrix((2, 2)), A, np.array([-1.0, -1.0]), np.array([-4.0, -6.0]),
                  np.zeros(2), np.full(2, np.inf), 0)
    res = R.solve(p, R.Options(eps=1e-10))
    assert res.status == "optimal"
    np.testing.assert_allclose(res.x, [1.6, 1.2], atol=1e-8)
    assert res.kkt["primal_obj"] == pytest.approx(-2.8, abs=1e-8)


# --------------------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed,n,m,m_eq,bounds", [
    (21, 4, 3, 1, "box"), (22, 5, 4, 2, "mixed"), (23, 6, 3, 0, "lower"),
    (24, 5, 2, 1, "upper"), (25, 6, 4, 2, "mixed"), (26, 4, 4, 0, "box"),
])
def test_brute_force_active_set(seed, n, m, m_eq, bounds):
    inst = qpgen.tiny_qp(seed, n=n, m=m, m_eq=m_eq, bounds=bounds)
    truth = active_set_solve(inst.Q.toarray(), inst.A.toarray(), inst.b, inst.c, inst.l, inst.u, m_eq)
    assert truth is not None
    res = R.solve(inst, R.Options(eps=1e-10))
    assert res.status == "optimal"
    np.testing.assert_allclose(res.x, truth[0], atol=1e-6)
    assert res.kkt["primal_obj"] == pytest.approx(truth[2], rel=1e-8, abs=1e-8)
    assert kkt_certificate(inst.Q.toarray(), inst.A.toarray(), inst.b, inst.c, inst.l, inst.u,
                           m_eq, res.x, res.y, tol=1e-6)


def test_singular_Q_brute_force():
    """Rank-deficient Q (mixed LP/QP directions)."""
    inst = qpgen.tiny_qp(31, n=6, m=3, m_eq=1, bounds="box", q_rank=2)
    truth = active_set_solve(inst.Q.toarray(), inst.A.toarray(), inst.b, inst.c, inst.l, inst.u, 1)
    res = R.solve(inst, R.Options(eps=1e-10))
    assert res.status == "optimal"
    assert res.kkt["primal_obj"] == pytest.approx(truth[2], rel=1e-8, abs=1e-8)


def test_config0_kkt_certificate():
    """The oracle's answer on the n=1000 workload satisfies the KKT conditions."""
    inst = qpgen.random_sparse_qp()
    res = R.solve(inst, R.Options(eps=1e-8))
    assert res.status == "optimal"
    assert res.kkt["rel_kkt"] <= 1e-8
    assert kkt_certificate(inst.Q.toarray(), inst.A.toarray(), inst.b, inst.c, inst.l, inst.u,
                           inst.m_eq, res.x, res.y, tol=1e-5)


# --------------------------------------------------------------------------- step schedule
def test_theory_schedule_satisfies_lemma1_conditions():
    """Lemma 2(i): the eq. (param-choice) schedule satisfies eq. (param) with
    theta_{k+1} = eta_k/eta_{k+1} = tau_k/tau_{k+1}."""
    nQ, nA, K = 3.0, 2.0, 50
    for k in range(K - 1):
        b0, t0 = R.beta_theta(k, True)
        b1, t1 = R.beta_theta(k + 1, True)
        e0, s0 = R.theory_steps(k, K, nQ, nA)
        e1, s1 = R.theory_steps(k + 1, K, nQ, nA)
        if k == 0:
            assert b0 == 1.0
        assert b1 - 1.0 == pytest.approx(b0 * t1, rel=1e-15)
        assert t1 == pytest.approx(e0 / e1, rel=1e-14)
        assert t1 == pytest.approx(s0 / s1, rel=1e-14)
        assert 1.0 / e0 - nQ / b0 - 4.0 * nA ** 2 * s0 >= -1e-12


def test_pdqp_step_rule_special_cases():
    """||A|| = 0: the rule reduces to accelerated gradient, primal step
    0.99 beta_k/||Q||; ||Q|| = 0: constant PDHG step with tau*sigma*||A||^2 = 0.99^2."""
    omega = 1.7
    eta = 0.0
    for k in range(30):
        eta = R.pdqp_eta(k, eta, 4.0, 0.0, omega)
        beta, _ = R.beta_theta(k, True)
        assert eta / omega == pytest.approx(0.99 * beta / 4.0, rel=1e-14)
    eta = 0.0
    for k in range(30):
        eta = R.pdqp_eta(k, eta, 0.0, 2.5, omega)
        assert (eta / omega) * (eta * omega) * 2.5 ** 2 == pytest.approx(0.99 ** 2, rel=1e-14)


def test_pdqp_step_rule_respects_lemma1_bound():
    """1/tau_p - ||Q||/beta_k - ||A||^2 sigma_d >= 0 (Lemma 1's last condition in
    the form its proof uses) and the growth cap theta_{k+1} <= eta_k/eta_{k+1}."""
    for nQ, nA, omega in [(1.0, 1.0, 1.0), (5.0, 0.3, 0.2), (0.2, 3.0, 7.0)]:
        eta = 0.0
        prev = None
        for k in range(200):
            eta = R.pdqp_eta(k, eta, nQ, nA, omega)
            beta, theta = R.beta_theta(k, True)
            tau_p, sigma_d = eta / omega, eta * omega
            assert 1.0 / tau_p - nQ / beta - nA ** 2 * sigma_d >= -1e-12
            if prev is not None:
                assert theta <= prev / eta * (1 + 1e-14)
            prev = eta


# --------------------------------------------------------------------------- Section 6 rules
def test_restart_conditions():
    o = R.Options()
    cur, avg = ("xc", "yc", 0.3), ("xa", "ya", 0.5)
    # candidate = current (strictly smaller)
    assert R.get_restart_candidate(cur, avg)[2] == 0.3
    assert R.get_restart_candidate(("a", "b", 0.5), avg)[0] == "xa"      # tie -> average
    # (i) sufficient decay
    assert R.restart_decision(o, ("x", "y", 0.19), avg, 1.0, None, 10, 1000)[3]
    # (ii) necessary decay + no local progress
    assert R.restart_decision(o, ("x", "y", 0.7), ("x", "y", 0.9), 1.0, 0.6, 10, 1000)[3]
    assert not R.restart_decision(o, ("x", "y", 0.7), ("x", "y", 0.9), 1.0, 0.75, 10, 1000)[3]
    assert not R.restart_decision(o, ("x", "y", 0.7), ("x", "y", 0.9), 1.0, None, 10, 1000)[3]
    assert not R.restart_decision(o, ("x", "y", 0.85), ("x", "y", 0.9), 1.0, 0.6, 10, 1000)[3]
    # (iii) long inner loop: t >= 0.36 k
    assert R.restart_decision(o, ("x", "y", 0.9), ("x", "y", 0.95), 1.0, None, 360, 1000)[3]
    assert not R.restart_decision(o, ("x", "y", 0.9), ("x", "y", 0.95), 1.0, None, 359, 1000)[3]
    # halving restarts to the average
    oh = R.Options(restart_rule="halving")
    r = R.restart_decision(oh, ("x", "y", 0.1), ("xa", "ya", 0.5), 1.0, None, 5, 1000)
    assert r[0] == "xa" and r[3]
    assert not R.restart_decision(oh, ("x", "y", 0.1), ("xa", "ya", 0.51), 1.0, None, 5, 1000)[3]


def test_primal_weight_rules():
    c, b = np.array([3.0, 4.0]), np.array([0.0, 2.0])
    assert R.initialize_primal_weight(c, b, 1e-10) == pytest.approx(2.5)
    assert R.initialize_primal_weight(c, np.zeros(2), 1e-10) == 1.0
    z_old = (np.zeros(2), np.zeros(1))
    z_new = (np.array([3.0, 4.0]), np.array([40.0]))     # dx = 5, dy = 40
    w = R.primal_weight_update(z_new, z_old, 2.0, 0.2, 1e-10)
    assert w == pytest.approx(8.0 ** 0.2 * 2.0 ** 0.8, rel=1e-14)
    assert R.primal_weight_update((np.zeros(2), z_new[1]), z_old, 2.0, 0.2, 1e-10) == 2.0


# --------------------------------------------------------------------------- preprocessing / norms
def test_lanczos_norms_match_dense_linear_algebra():
    """On a 12-variable problem Lanczos reaches an invariant subspace within 12
    steps, so the Ritz value is the exact top eigenvalue."""
    inst = qpgen.tiny_qp(41, n=12, m=7, m_eq=2, bounds="box")
    p = R.problem_from_instance(inst)
    assert R.norm_A(p, tol=0.0) == pytest.approx(np.linalg.norm(p.A.toarray(), 2), rel=1e-10)
    assert R.norm_Q(p, tol=0.0) == pytest.approx(np.linalg.eigvalsh(p.Q.toarray()).max(), rel=1e-10)


def test_lanczos_on_the_n1000_workload():
    """Against a dense eigen-solve of the scaled n=1000 operators, at the default
    tolerance: Ritz values are lower bounds of the top eigenvalue and the
    default stopping rule leaves them within 1e-5 of it."""
    inst = qpgen.random_sparse_qp()
    p = R.problem_from_instance(inst)
    D1, D2 = R.scaling_factors(p)
    ps = R.scale_problem(p, D1, D2)
    A, Q = ps.A.toarray(), ps.Q.toarray()
    truth_A, truth_Q = np.linalg.norm(A, 2), np.linalg.eigvalsh(Q).max()
    nA, nQ = R.norm_A(ps), R.norm_Q(ps)
    assert nA == pytest.approx(truth_A, rel=1e-5) and nA <= truth_A * (1 + 1e-12)
    assert nQ == pytest.approx(truth_Q, rel=1e-5) and nQ <= truth_Q * (1 + 1e-12)
    assert R.NORM_STEPS["A"] < 100 and R.NORM_STEPS["Q"] < 100


def test_ruiz_equilibrates_and_scaling_is_symmetric():
    inst = qpgen.tiny_qp(51, n=9, m=5, m_eq=2, bounds="box")
    p = R.problem_from_instance(inst)
    p.A = sp.csr_matrix(p.A.toarray() * np.array([1e3, 1, 1e-2, 5, 1])[:, None])
    D1, D2 = R.scaling_factors(p, ruiz_iters=60, l2=False, pock_chambolle=False)
    ps = R.scale_problem(p, D1, D2)
    K = np.block([[ps.Q.toarray(), ps.A.toarray().T], [ps.A.toarray(), np.zeros((5, 5))]])
    np.testing.assert_allclose(np.abs(K).max(axis=1), 1.0, atol=1e-6)
    # scaled data equal D K D built densely
    Kd = np.block([[p.Q.toarray(), p.A.toarray().T], [p.A.toarray(), np.zeros((5, 5))]])
    d = np.concatenate([D2, D1])
    np.testing.assert_allclose(K, d[:, None] * Kd * d[None, :], rtol=1e-13, atol=1e-300)


def test_pock_chambolle_pass_normalises_l1_rows():
    """A lone alpha=1 Pock-Chambolle pass on K leaves each row's scaled l1 sum
    sum_j |K_ij| d_i d_j with d_i = 1/sqrt(l1_i): for a diagonal K, exactly 1."""
    n = 4
    q = np.array([4.0, 9.0, 0.25, 16.0])
    p = R.Problem(sp.csr_matrix(np.diag(q)), sp.csr_matrix((0, n)), np.ones(n), np.zeros(0),
                  -np.ones(n), np.ones(n), 0)
    D1, D2 = R.scaling_factors(p, ruiz_iters=0, l2=False, pock_chambolle=True)
    np.testing.assert_allclose(D2, 1.0 / np.sqrt(q), rtol=1e-15)


def test_scaling_does_not_change_the_answer():
    inst = qpgen.tiny_qp(61, n=8, m=5, m_eq=2, bounds="mixed")
    a = R.solve(inst, R.Options(eps=1e-10, scaling=True))
    b = R.solve(inst, R.Options(eps=1e-10, scaling=False))
    np.testing.assert_allclose(a.x, b.x, atol=1e-6)
    assert a.kkt["primal_obj"] == pytest.approx(b.kkt["primal_obj"], rel=1e-8)


# --------------------------------------------------------------------------- variants
def test_plain_pdhg_variant_matches_textbook_step():
    """accelerate=False: beta = theta = 1 turns Algorithm 1 into PDHG with
    x_tilde = 2 x^k - x^{k-1} and constant steps; compare two steps by hand."""
    inst = qpgen.tiny_qp(71, n=5, m=3, m_eq=1, bounds="box")
    p = R.problem_from_instance(inst)
    opts = R.Options(accelerate=False, scaling=False, norm_A=2.0, norm_Q=3.0, max_iter=2,
                     check_period=1000, eps=0.0)
    res = R.solve(p, opts, trace_at=(1, 2))
    omega = np.linalg.norm(p.c) / np.linalg.norm(p.b)
    eta = 1.98 / (3.0 / omega + math.sqrt(4 * 4.0 + (3.0 / omega) ** 2))
    tp, sd = eta / omega, eta * omega
    A, Q = p.A.toarray(), p.Q.toarray()
    x_prev = x = np.clip(np.zeros(5), p.l, p.u)
    y = np.zeros(3)
    for it in (1, 2):
        xt = 2 * x - x_prev
        y = y - sd * (A @ xt - p.b)
        y[1:] = np.maximum(y[1:], 0)
        x_prev, x = x, np.clip(x - tp * (Q @ x + p.c - A.T @ y), p.l, p.u)
        np.testing.assert_allclose(res.trace[it]["x"], x, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(res.trace[it]["y"], y, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(res.trace[it]["xbar"], x, rtol=1e-14, atol=1e-15)


def test_iterates_stay_feasible_for_projections():
    inst = qpgen.tiny_qp(81, n=7, m=4, m_eq=2, bounds="mixed")
    res = R.solve(inst, R.Options(max_iter=150, eps=0.0, check_period=32), trace_at=range(1, 151))
    for t, st in res.trace.items():
        assert np.all(st["x"] >= inst.l - 1e-12) and np.all(st["x"] <= inst.u + 1e-12)
        assert np.all(st["y"][2:] >= 0.0)


def test_restart_variants_converge_and_rapdhg_beats_pdhg():
    """All restart schemes reach the brute-force optimum; with acceleration and
    restarts the method needs fewer iterations than plain PDHG (Tables 1-2)."""
    inst = qpgen.tiny_qp(91, n=6, m=4, m_eq=1, bounds="box", q_rank=3)
    truth = active_set_solve(inst.Q.toarray(), inst.A.toarray(), inst.b, inst.c, inst.l, inst.u, 1)
    iters = {}
    for name, o in {
        "rapdhg": R.Options(eps=1e-8),
        "halving": R.Options(eps=1e-8, restart_rule="halving"),
        "fixed": R.Options(eps=1e-8, restart_rule="fixed", fixed_K=128),
        "pdhg": R.Options(eps=1e-8, restart_rule="none", accelerate=False, max_iter=400000),
    }.items():
        res = R.solve(inst, o)
        assert res.status == "optimal", name
        assert res.kkt["primal_obj"] == pytest.approx(truth[2], rel=1e-6, abs=1e-6), name
        iters[name] = res.iterations
    assert iters["rapdhg"] < iters["pdhg"]


def test_relkkt_when_the_dual_objective_exceeds_the_primal():
    """Worked by hand: min 1/2 x^2 s.t. x >= 1 (no bounds) at x = 1/2, y = 3.
    Primal violation 1 - 1/2 over 1 + max(|Ax|, |b|) = 2: 1/4.  Reduced cost
    Qx - A'y = -5/2 with Lambda = {0}: dual residual 5/2 over 1 + max(1/2, 3, 0):
    5/8.  Objectives p = 1/8, d = -1/8 + 3 = 23/8: gap |p - d| / (1 + 23/8) =
    22/31, the largest, so relKKT = 22/31 (the gap is an absolute value)."""
    p = R.Problem(sp.csr_matrix(np.array([[1.0]])), sp.csr_matrix(np.array([[1.0]])), np.zeros(1),
                  np.array([1.0]), np.array([-np.inf]), np.array([np.inf]), 0)
    k = R.kkt_parts(p, np.array([0.5]), np.array([3.0]))
    assert k["r_primal"] == pytest.approx(1 / 4, abs=1e-15)
    assert k["r_dual"] == pytest.approx(5 / 8, abs=1e-15)
    assert (k["primal_obj"], k["dual_obj"]) == (pytest.approx(1 / 8, abs=1e-15), pytest.approx(23 / 8, abs=1e-15))
    assert k["r_gap"] == pytest.approx(22 / 31, abs=1e-15)
    assert k["rel_kkt"] == pytest.approx(22 / 31, abs=1e-15)
