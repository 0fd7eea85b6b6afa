"""More planted mistakes, each run against the complete oracle pin files: the
oracle, the generators and the tests are copied to a scratch directory, the
mistake is planted in the copy of the oracle, and the pin files run there in
a subprocess (the repository's own oracle is never edited).  Every mistake
must fail at least one pin.  Not planted: replacing the step-growth cap
min((1 + 1/k) eta_{k-1}, bound_k) by bound_k, an equivalent change (within an
epoch the min always picks the bound, since bound_k / bound_{k-1} <=
(k+2)/(k+1) < (k+1)/k)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_fixed_point.py", "tests/test_oracle_theorem1.py",
             "tests/test_oracle_infeasibility.py", "tests/test_oracle_lowrank.py",
             "tests/test_oracle_lanczos_start.py", "tests/test_oracle_classes.py",
             "tests/test_oracle_restart_bookkeeping.py", "tests/test_oracle_invariants.py"]

MUTATIONS = {
    "primal_weight_inverted": ("math.exp(theta * math.log(dy / dx) + (1.0 - theta) * math.log(omega))",
                               "math.exp(theta * math.log(dx / dy) + (1.0 - theta) * math.log(omega))"),
    "primal_weight_theta_swapped": ("math.exp(theta * math.log(dy / dx) + (1.0 - theta) * math.log(omega))",
                                    "math.exp((1.0 - theta) * math.log(dy / dx) + theta * math.log(omega))"),
    "initial_weight_inverted": ("return nc / nb if (nc > eps_zero and nb > eps_zero) else 1.0",
                                "return nb / nc if (nc > eps_zero and nb > eps_zero) else 1.0"),
    "first_step_halved": ("return 1.98 / (q + math.sqrt(4.0 * normA ** 2 + q ** 2))",
                          "return 0.99 / (q + math.sqrt(4.0 * normA ** 2 + q ** 2))"),
    "condition_ii_reversed": ("and cand > prev_cand_kkt)", "and cand < prev_cand_kkt)"),
    "artificial_restart_constant": ("or k >= opts.beta_art * total)", "or k >= opts.beta_nec * total)"),
    "halving_factor": ("return ax, ay, akkt, akkt <= 0.5 * anchor_kkt",
                       "return ax, ay, akkt, akkt <= 0.8 * anchor_kkt"),
    "xbar_from_old_x": ("xbar = (1.0 - 1.0 / beta) * xbar + x_new / beta",
                        "xbar = (1.0 - 1.0 / beta) * xbar + x / beta"),
    "steps_swapped": ("tau_p, sigma_d = eta / omega, eta * omega", "tau_p, sigma_d = eta * omega, eta / omega"),
    "l2_pass_is_l1": ("nu = np.sqrt(np.asarray(absK.multiply(absK).sum(axis=1)).ravel())",
                      "nu = np.asarray(absK.sum(axis=1)).ravel()"),
    "anchor_relkkt_not_reset": ("anchor_x, anchor_y, anchor_kkt = x.copy(), y.copy(), cand_kkt",
                                "anchor_x, anchor_y = x.copy(), y.copy()"),
    "previous_candidate_kept": ("        anchor_x, anchor_y, anchor_kkt = x.copy(), y.copy(), cand_kkt\n        prev_cand_kkt = None",
                                "        anchor_x, anchor_y, anchor_kkt = x.copy(), y.copy(), cand_kkt"),
    "restart_keeps_x_prev": ("        x_prev, xbar, ybar = x.copy(), x.copy(), y.copy()\n        anchor_x",
                             "        xbar, ybar = x.copy(), y.copy()\n        anchor_x"),
    "lanczos_absolute_tolerance": (
        "if abs(theta - theta_prev) <= tol * abs(theta) or beta <= 1e-12 * abs(theta):",
        "if abs(theta - theta_prev) <= tol or beta <= 1e-12 * abs(theta):"),
    "x0_not_projected": ("x = proj_X(np.zeros(n) if x0 is None else np.asarray(x0, np.float64) / D2, ps.l, ps.u)",
                         "x = np.zeros(n) if x0 is None else np.asarray(x0, np.float64) / D2"),
    "y0_not_projected": ("y = proj_Y(np.zeros(m) if y0 is None else np.asarray(y0, np.float64) / D1, m_eq)",
                         "y = np.zeros(m) if y0 is None else np.asarray(y0, np.float64) / D1"),
    "relkkt_on_scaled_problem": ("kkt_cur = rel_kkt(p, *unscale(x, y))", "kkt_cur = rel_kkt(ps, x, y)"),
    "no_check_at_max_iter": ("if total % opts.check_period != 0 and total != opts.max_iter:",
                             "if total % opts.check_period != 0:"),
    "termination_strict": ("if cand_kkt <= opts.eps:", "if cand_kkt < opts.eps:"),
    "certificate_average_first": ("    for xs, ys in iterates:\n", "    for xs, ys in reversed(iterates):\n"),
    "primal_rays_tested_first": (
        "    for d, rho in rays:\n        v = dual_ray_value(p, rho, eps)\n        if v > 0:\n"
        "            return \"primal_infeasible\", np.zeros(p.n), rho / v\n"
        "    for d, rho in rays:\n        v = primal_ray_value(p, d, eps)\n        if v > 0:\n"
        "            return \"dual_infeasible\", d / v, np.zeros(p.m)\n",
        "    for d, rho in rays:\n        v = primal_ray_value(p, d, eps)\n        if v > 0:\n"
        "            return \"dual_infeasible\", d / v, np.zeros(p.m)\n"
        "    for d, rho in rays:\n        v = dual_ray_value(p, rho, eps)\n        if v > 0:\n"
        "            return \"primal_infeasible\", np.zeros(p.n), rho / v\n"),
    "gap_without_abs": ("r_gap = abs(primal_obj - dual_obj) / (1.0 + max(abs(primal_obj), abs(dual_obj)))",
                        "r_gap = (primal_obj - dual_obj) / (1.0 + max(abs(primal_obj), abs(dual_obj)))"),
}


def _scratch(tmp_path):
    for d in ("oracle", "qpgen", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=shutil.ignore_patterns("__pycache__"))
    return tmp_path


def _run_pins(where):
    env = {**os.environ, "PYTHONDONTWRITEBYTECODE": "1"}
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_FILES],
                          cwd=where, env=env, capture_output=True, text=True, timeout=900)


def test_unmutated_copy_passes(tmp_path):
    r = _run_pins(_scratch(tmp_path))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    where = _scratch(tmp_path)
    src_path = where / "oracle" / "rapdhg.py"
    src = src_path.read_text()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    src_path.write_text(src.replace(old, new))
    r = _run_pins(where)
    assert r.returncode != 0, f"{name} passed every pin"
