"""Planted mistakes: each mutation edits a copy of the oracle's source on the
CPU (a dropped term, a wrong sign or index, a transposed operand) and at least
one pin of the oracle must then fail."""
import json
import os
import sys
import types
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from tests.qp_truth import active_set_solve

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "rapdhg.py")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MUTATIONS = {
    "dual_sign": ("proj_Y(y - sigma_d * (ps.A @ x_tilde - ps.b), m_eq)",
                  "proj_Y(y + sigma_d * (ps.A @ x_tilde - ps.b), m_eq)"),
    "drop_ATy": ("ps.Qmul(x_md) + ps.c - ps.A.T @ y_new", "ps.Qmul(x_md) + ps.c"),
    "ATy_uses_old_y": ("ps.Qmul(x_md) + ps.c - ps.A.T @ y_new", "ps.Qmul(x_md) + ps.c - ps.A.T @ y"),
    "xmd_from_x": ("x_md = (1.0 - 1.0 / beta) * xbar + x / beta", "x_md = x"),
    "no_extrapolation": ("x_tilde = x + theta * (x - x_prev)", "x_tilde = x"),
    "theta_index": ("return (k + 2) / 2.0, k / (k + 1.0)", "return (k + 2) / 2.0, (k + 1) / (k + 2.0)"),
    "beta_index": ("return (k + 2) / 2.0, k / (k + 1.0)", "return (k + 1) / 2.0 + 0.5 * (k == 0), k / (k + 1.0)"),
    "ybar_weight": ("ybar = (1.0 - 1.0 / beta) * ybar + y_new / beta", "ybar = (1.0 - 1.0 / beta) * ybar + y / beta"),
    "no_dual_projection": ("out[m_eq:] = np.maximum(out[m_eq:], 0.0)", "pass"),
    "eq_rows_projected": ("out[m_eq:] = np.maximum(out[m_eq:], 0.0)", "out[:] = np.maximum(out, 0.0)"),
    "primal_viol_sign": ("np.maximum(p.b[p.m_eq:] - Ax[p.m_eq:], 0.0)", "np.maximum(Ax[p.m_eq:] - p.b[p.m_eq:], 0.0)"),
    "gap_drops_bound_term": ("dual_obj = -0.5 * xQx + float(p.b @ y) + bound_term",
                             "dual_obj = -0.5 * xQx + float(p.b @ y)"),
    "dual_denominator": ("max(inf(Qx), inf(ATy), inf(p.c))", "max(inf(Qx), inf(ATy))"),
    "transposed_A_in_kkt": ("ATy = p.A.T @ y", "ATy = p.A.T @ (y[::-1])"),
    "theory_dual_step": ("(k + 1) / (2.0 * K * normA)", "(k + 1) / (2.0 * (normQ + K * normA))"),
    "scale_c_wrong": ("return Problem(Qs, As, D2 * p.c, D1 * p.b, p.l / D2, p.u / D2, p.m_eq, F)",
                      "return Problem(Qs, As, p.c / D2, D1 * p.b, p.l / D2, p.u / D2, p.m_eq, F)"),
    "scale_bounds_wrong": ("return Problem(Qs, As, D2 * p.c, D1 * p.b, p.l / D2, p.u / D2, p.m_eq, F)",
                           "return Problem(Qs, As, D2 * p.c, D1 * p.b, p.l * D2, p.u * D2, p.m_eq, F)"),
    "lanczos_sign": ("w = w - alpha * v - beta_prev * v_prev", "w = w - alpha * v + beta_prev * v_prev"),
    "unscale_wrong": ("unscale = lambda xs, ys: (D2 * xs, D1 * ys)", "unscale = lambda xs, ys: (xs / D2, ys / D1)"),
}


def _load(mutation):
    src = open(ORACLE_SRC).read()
    old, new = MUTATIONS[mutation]
    assert src.count(old) >= 1, f"mutation anchor not found: {mutation}"
    src = src.replace(old, new)
    name = "oracle_mutant_" + mutation
    mod = types.ModuleType(name)
    sys.modules[name] = mod          # dataclasses look their module up here
    exec(compile(src, name, "exec"), mod.__dict__)
    return mod


def _pins_pass(R):
    """A subset of the oracle pins, re-run against module R."""
    try:
        g = json.load(open(os.path.join(GOLDEN, "hand_three_iterations.json")))
        d = g["problem"]
        p = R.Problem(sp.csr_matrix(np.array(d["Q"], float)), sp.csr_matrix(np.array(d["A"], float)),
                      np.array(d["c"], float), np.array(d["b"], float), np.array(d["l"], float),
                      np.array(d["u"], float), d["m_eq"])
        o = R.Options(step_rule="theory", restart_rule="fixed", fixed_K=4, scaling=False, norm_Q=2,
                      norm_A=1, max_iter=3, check_period=1000, eps=0.0)
        res = R.solve(p, o, trace_at=(1, 2, 3))
        for it, want in g["iterates"].items():
            for key in ("x", "y", "xbar", "ybar"):
                if abs(res.trace[int(it)][key][0] - float(Fraction(want[key]))) > 1e-12:
                    return False
        g = json.load(open(os.path.join(GOLDEN, "hand_relkkt.json")))
        d = g["problem"]
        for case in g["cases"]:
            p = R.Problem(sp.csr_matrix(np.array(d["Q"], float)), sp.csr_matrix(np.array(d["A"], float)),
                          np.array(d["c"], float), np.array(d["b"], float),
                          np.array([float(Fraction(v)) if v not in ("inf", "-inf") else float(v) for v in case["l"]]),
                          np.array([float(Fraction(v)) if v not in ("inf", "-inf") else float(v) for v in case["u"]]),
                          d["m_eq"])
            parts = R.kkt_parts(p, np.array([float(Fraction(str(v))) for v in case["x"]]),
                                np.array([float(Fraction(str(v))) for v in case["y"]]))
            for key in ("r_primal", "r_dual", "r_gap", "primal_obj", "dual_obj"):
                if abs(parts[key] - float(Fraction(case[key]))) > 1e-12:
                    return False
        inst = qpgen.tiny_qp(41, n=12, m=7, m_eq=2, bounds="box")
        p = R.problem_from_instance(inst)
        if abs(R.norm_A(p, tol=0.0) - np.linalg.norm(p.A.toarray(), 2)) > 1e-9:
            return False
        if abs(R.norm_Q(p, tol=0.0) - np.linalg.eigvalsh(p.Q.toarray()).max()) > 1e-9:
            return False
        for seed, n, m, m_eq, bounds in [(21, 4, 3, 1, "box"), (22, 5, 4, 2, "mixed")]:
            inst = qpgen.tiny_qp(seed, n=n, m=m, m_eq=m_eq, bounds=bounds)
            inst.A = sp.csr_matrix(inst.A.toarray() * np.linspace(0.5, 3.0, m)[:, None])
            truth = active_set_solve(inst.Q.toarray(), inst.A.toarray(), inst.b * np.linspace(0.5, 3.0, m),
                                     inst.c, inst.l, inst.u, m_eq)
            inst.b = inst.b * np.linspace(0.5, 3.0, m)
            res = R.solve(inst, R.Options(eps=1e-9, max_iter=20000))
            if res.status != "optimal" or np.max(np.abs(res.x - truth[0])) > 1e-5:
                return False
        return True
    except (FloatingPointError, ValueError, ZeroDivisionError, OverflowError, IndexError, np.linalg.LinAlgError):
        return False


def test_unmutated_oracle_passes_the_subset():
    import oracle.rapdhg as R
    assert _pins_pass(R)


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_planted_mistake_is_caught(mutation):
    with np.errstate(all="ignore"):
        assert not _pins_pass(_load(mutation))
