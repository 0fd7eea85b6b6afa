"""Plain FP64 CPU oracle for restarted accelerated PDHG (rAPDHG) on convex QP.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
CPU-baseline / reference leg may import this module; the product path never
does and shares no code with it.

It restates, slowly and in float64, what the paper (Lu & Yang, "A Practical
and Optimal First-Order Method for Large-Scale Convex Quadratic Programming")
defines:

* Algorithm 1 (rAPDHG): the inner accelerated-PDHG loop (Section 2, Lemma 1
  restates the same update) with x_md, the extrapolated primal point, the
  projected dual step, the primal step and the running averages.
* Theorem 1 / eq. (param-choice): beta_k = (k+2)/2, theta_k = k/(k+1) and the
  theory step sizes eta_k, tau_k for fixed-frequency restarts.
* Section 5: the relative KKT error (r_primal, r_dual, r_gap, relKKT), the
  termination rule eq. (terminate), the diagonal preconditioning (10 Ruiz
  steps, l2 scaling, Pock-Chambolle on [[Q, A'], [A, 0]]) and the halving /
  fixed-frequency / no-restart schemes.
* Section 6: PDQP's restart candidate, its three restart conditions, its
  adaptive step size eta^{n,k} and the primal-weight initialisation and
  update.

Problem form (extension of eq. (1) allowed by its footnote):
    min 1/2 x'Qx + c'x  s.t.  A_E x = b_E,  A_I x >= b_I,  l <= x <= u
with Lagrangian L(x,y) = 1/2 x'Qx + c'x - y'(Ax - b), x in X = [l,u],
y in Y = R^{m_eq} x R_+^{m-m_eq}.  Substituting A' = -A, b' = -b into eq. (2)
and Algorithm 1 gives the signs used below.

Readings of the paper where it is silent or ambiguous (each is also listed in
the design notes of the repository):
  R1 problem form as above; bounds enter as a projection onto X in the primal step.
  R2 signs from A' = -A, b' = -b.
  R3 PDQP's primal step is eta/omega, its dual step eta*omega (the only
     assignment under which the Section 6 step rule equals the Lemma 1 bound
     1/eta_p - ||Q||/beta_k - ||A||^2 tau_d >= 0 with a 0.99 margin).
  R4 beta_k = (k+2)/2, theta_k = k/(k+1) also in the practical solver; the
     inner counter k restarts at 0 in every epoch.  Without acceleration
     beta_k = theta_k = 1 and eta stays at its k = 0 value.
  R5 relKKT for equalities and bounds: primal violation |A_E x - b_E| and
     [b_I - A_I x]_+; reduced cost lambda = proj_Lambda(Qx + c - A'y); dual
     residual Qx + c - A'y - lambda; dual objective
     -1/2 x'Qx + b'y + sum_j (l_j lambda_j^+ - u_j lambda_j^-).
  R6 relKKT is measured on the original (unscaled) problem.
  R7 relKKT is evaluated every `check_period` iterations (and at max_iter);
     condition (ii) compares with the candidate of the previous check of
     the same epoch and is false at the first check of an epoch.
  R8 condition (iii): t = iterations of the current epoch, k = total iterations.
  R9 eps_zero = 1e-10.
  R10 ||A||_2, ||Q||_2 by the Lanczos method (largest Ritz value) from the
      sign vector s/sqrt(n), s_j = -1 where the top bit of SplitMix64's
      finaliser (Steele, Lea & Flood 2014) of the index j is set, else +1; the
      paper does not say how the norms are obtained.  (Not the all-ones
      vector: it is an eigenvector of Laplacian-like operators -- of Q = L + cI
      for its smallest eigenvalue, of A'A in its null space when every row of
      A sums to zero -- where Lanczos stops at once at the wrong value.)
  R11 scaling passes divide every index j of the symmetric K by
      sqrt(norm of row j of the current scaled K) (inf-norm for Ruiz, 2-norm
      for the l2 pass, 1-norm for Pock-Chambolle with alpha = 1); zero
      norms leave the index unscaled; l, u are divided by D2.
  R12 the step rule, primal weight and restart distances live in the scaled
      space the iteration runs in.
  R13 candidate ties pick the average (strict '<' in GetRestartCandidate).
  R14 a low-rank term F F' of Q is applied as F(F'x) and is left out of the
      scaling norms (D2 still scales F).
  R15 fixed-frequency restarts (restart_rule "fixed") are taken at the first
      check with k >= K: restarts happen only at checks.
  R18 (not in the paper; optional) infeasibility certificates: at every
      check after the termination and iteration-limit tests, the current and
      the average iterate's displacement from the epoch's anchor, projected
      onto the recession cones of X and Y and unscaled, are tested as a
      Farkas ray y (primal infeasible) and as an unbounded direction d (dual
      infeasible), each to eps_infeasible relative to its own objective term.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------------------
# Problem data
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """Data of one QP.  Q is a sparse symmetric matrix; F (optional) adds F F'."""
    Q: sp.csr_matrix
    A: sp.csr_matrix
    c: np.ndarray
    b: np.ndarray
    l: np.ndarray
    u: np.ndarray
    m_eq: int
    F: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return self.Q.shape[0]

    @property
    def m(self) -> int:
        return self.A.shape[0]

    def Qmul(self, v: np.ndarray) -> np.ndarray:
        out = self.Q @ v
        if self.F is not None:
            out = out + self.F @ (self.F.T @ v)
        return out


def problem_from_instance(inst) -> Problem:
    F = None if inst.F is None else np.asarray(inst.F, dtype=np.float64)
    return Problem(sp.csr_matrix(inst.Q, dtype=np.float64), sp.csr_matrix(inst.A, dtype=np.float64),
                   np.asarray(inst.c, np.float64), np.asarray(inst.b, np.float64),
                   np.asarray(inst.l, np.float64), np.asarray(inst.u, np.float64), int(inst.m_eq), F)


# ---------------------------------------------------------------------------
# Projections onto X = [l, u] and Y = R^{m_eq} x R_+^{m - m_eq}
# ---------------------------------------------------------------------------
def proj_X(x, l, u):
    return np.minimum(np.maximum(x, l), u)


def proj_Y(y, m_eq):
    out = y.copy()
    out[m_eq:] = np.maximum(out[m_eq:], 0.0)
    return out


# ---------------------------------------------------------------------------
# Relative KKT error (Section 5 "Progress metric", generalised per R5)
# ---------------------------------------------------------------------------
def kkt_parts(p: Problem, x: np.ndarray, y: np.ndarray) -> Dict[str, float]:
    """Relative primal residual, dual residual and gap of (x, y) on problem p."""
    Ax = p.A @ x
    Qx = p.Qmul(x)
    ATy = p.A.T @ y
    # primal violation: equality rows |Ax - b|, inequality rows [b - Ax]_+
    viol = Ax - p.b
    viol[p.m_eq:] = np.maximum(p.b[p.m_eq:] - Ax[p.m_eq:], 0.0)
    viol = np.abs(viol)
    inf = lambda v: float(np.max(np.abs(v))) if v.size else 0.0
    r_primal = inf(viol) / (1.0 + max(inf(Ax), inf(p.b)))
    # reduced cost lambda = proj_Lambda(g), Lambda_j set by which bounds are finite
    g = Qx + p.c - ATy
    lo_fin = np.isfinite(p.l)
    up_fin = np.isfinite(p.u)
    lam = np.where(lo_fin & up_fin, g,
                   np.where(lo_fin, np.maximum(g, 0.0),
                            np.where(up_fin, np.minimum(g, 0.0), 0.0)))
    r_dual = inf(g - lam) / (1.0 + max(inf(Qx), inf(ATy), inf(p.c)))
    xQx = float(x @ Qx)
    primal_obj = 0.5 * xQx + float(p.c @ x)
    lam_pos = np.maximum(lam, 0.0)
    lam_neg = np.maximum(-lam, 0.0)
    # lambda_j^+ > 0 only where l_j is finite and lambda_j^- > 0 only where u_j is
    # finite, so 0 * inf never enters the sum
    bound_term = float(np.sum(np.where(lam_pos > 0, p.l, 0.0) * lam_pos)
                       - np.sum(np.where(lam_neg > 0, p.u, 0.0) * lam_neg))
    dual_obj = -0.5 * xQx + float(p.b @ y) + bound_term
    r_gap = abs(primal_obj - dual_obj) / (1.0 + max(abs(primal_obj), abs(dual_obj)))
    return dict(r_primal=r_primal, r_dual=r_dual, r_gap=r_gap,
                rel_kkt=max(r_primal, r_dual, r_gap),
                primal_obj=primal_obj, dual_obj=dual_obj)


def rel_kkt(p: Problem, x, y) -> float:
    return kkt_parts(p, x, y)["rel_kkt"]


# ---------------------------------------------------------------------------
# Diagonal preconditioning (Section 5 "Preprocessing", R11)
# ---------------------------------------------------------------------------
def _kkt_matrix(p: Problem) -> sp.csr_matrix:
    """K = [[Q, A'], [A, 0]] (sparse part of Q only, R14)."""
    return sp.bmat([[p.Q, p.A.T], [p.A, None]], format="csr")


def scaling_factors(p: Problem, ruiz_iters: int = 10, l2: bool = True,
                    pock_chambolle: bool = True):
    """Return (D1, D2) with K_scaled = D K D, D = diag(D2, D1)."""
    K = _kkt_matrix(p)
    d = np.ones(p.n + p.m)

    def one_pass(norm):
        nonlocal d
        Ks = sp.diags(d) @ K @ sp.diags(d)
        absK = abs(Ks)
        if norm == "inf":
            nu = np.asarray(absK.max(axis=1).todense()).ravel()
        elif norm == "l2":
            nu = np.sqrt(np.asarray(absK.multiply(absK).sum(axis=1)).ravel())
        else:  # "l1"
            nu = np.asarray(absK.sum(axis=1)).ravel()
        nu = np.where(nu > 0, nu, 1.0)
        d = d / np.sqrt(nu)

    for _ in range(ruiz_iters):
        one_pass("inf")
    if l2:
        one_pass("l2")
    if pock_chambolle:
        one_pass("l1")
    return d[p.n:].copy(), d[:p.n].copy()


def scale_problem(p: Problem, D1: np.ndarray, D2: np.ndarray) -> Problem:
    """Q~ = D2 Q D2, A~ = D1 A D2, c~ = D2 c, b~ = D1 b, l~ = l/D2, u~ = u/D2."""
    Qs = sp.csr_matrix(sp.diags(D2) @ p.Q @ sp.diags(D2))
    As = sp.csr_matrix(sp.diags(D1) @ p.A @ sp.diags(D2))
    F = None if p.F is None else p.F * D2[:, None]
    return Problem(Qs, As, D2 * p.c, D1 * p.b, p.l / D2, p.u / D2, p.m_eq, F)


# ---------------------------------------------------------------------------
# Spectral norms (R10)
# ---------------------------------------------------------------------------
NORM_STEPS = {}   # Lanczos steps taken by the latest call for each operator name


def lanczos_start(dim: int) -> np.ndarray:
    """R10's start vector: s_j / sqrt(dim), s_j = -1 where the top bit of the
    SplitMix64 finaliser of j (Steele, Lea & Flood 2014; uint64 arithmetic,
    which numpy wraps mod 2^64) is set, else +1."""
    z = np.arange(dim, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) == 1, -1.0, 1.0) / math.sqrt(dim)


def lanczos_max_eig(apply_sym, dim: int, max_iter: int = 500, tol: float = 1e-6, name: str = "") -> float:
    """Largest eigenvalue of a symmetric PSD operator: the largest Ritz value of
    the Lanczos tridiagonal T_k (plain three-term recurrence, no
    reorthogonalisation) started from lanczos_start (R10).  Stops when that
    value changes by at most tol relative, when beta_k <= 1e-12 theta_k (an
    invariant subspace: the value is exact), or after max_iter steps."""
    if dim == 0:
        return 0.0
    v = lanczos_start(dim)
    v_prev = np.zeros(dim)
    beta_prev = 0.0
    alphas, betas = [], []
    theta_prev = 0.0
    theta = 0.0
    for step in range(1, max_iter + 1):
        NORM_STEPS[name] = step
        w = apply_sym(v)
        alpha = float(v @ w)
        w = w - alpha * v - beta_prev * v_prev
        beta = float(np.linalg.norm(w))
        alphas.append(alpha)
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        theta = float(np.linalg.eigvalsh(T)[-1])
        if abs(theta - theta_prev) <= tol * abs(theta) or beta <= 1e-12 * abs(theta):
            break
        betas.append(beta)
        v_prev, v = v, w / beta
        beta_prev = beta
        theta_prev = theta
    return theta


def norm_A(p: Problem, **kw) -> float:
    if p.m == 0:
        return 0.0
    return math.sqrt(max(lanczos_max_eig(lambda v: p.A.T @ (p.A @ v), p.n, name="A", **kw), 0.0))


def norm_Q(p: Problem, **kw) -> float:
    return max(lanczos_max_eig(p.Qmul, p.n, name="Q", **kw), 0.0)


# ---------------------------------------------------------------------------
# Step-size schedules
# ---------------------------------------------------------------------------
def pdqp_eta(k: int, eta_prev: float, normQ: float, normA: float, omega: float) -> float:
    """Section 6 adaptive step size eta^{n,k}."""
    q = normQ / omega
    if k == 0:
        return 1.98 / (q + math.sqrt(4.0 * normA ** 2 + q ** 2))
    bound = 0.99 * (k + 2) / (q + math.sqrt(normA ** 2 * (k + 2) ** 2 + q ** 2))
    return min((1.0 + 1.0 / k) * eta_prev, bound)


def theory_steps(k: int, K: int, normQ: float, normA: float):
    """Theorem 1 / eq. (param-choice): (primal eta_k, dual tau_k)."""
    return (k + 1) / (2.0 * (normQ + K * normA)), (k + 1) / (2.0 * K * normA)


def beta_theta(k: int, accelerate: bool):
    """Theorem 1: beta_k = (k+2)/2, theta_k = k/(k+1); plain PDHG: 1, 1 (R4)."""
    if not accelerate:
        return 1.0, 1.0
    return (k + 2) / 2.0, k / (k + 1.0)



# ---------------------------------------------------------------------------
# Section 6 rules: restart candidate, restart conditions, primal weight
# ---------------------------------------------------------------------------
def get_restart_candidate(cur, avg):
    """GetRestartCandidate: the current iterate if its relKKT is strictly
    smaller, else the average (R13).  cur/avg = (x, y, relKKT)."""
    return cur if cur[2] < avg[2] else avg


def restart_decision(opts, cur, avg, anchor_kkt, prev_cand_kkt, k, total):
    """Returns (x_c, y_c, relKKT_c, restart?) for the rule in opts.restart_rule.
    pdqp: Section 6 conditions (i)-(iii) (R7, R8); halving: Section 5 adaptive
    scheme relKKT(z_bar) <= relKKT(z^{n,0}) / 2; fixed: after fixed_K inner
    iterations (Algorithm 1), both restarting from the average; none: never."""
    cx, cy, cand = get_restart_candidate(cur, avg)
    if opts.restart_rule == "pdqp":
        restart = (cand <= opts.beta_suff * anchor_kkt
                   or (cand <= opts.beta_nec * anchor_kkt and prev_cand_kkt is not None
                       and cand > prev_cand_kkt)
                   or k >= opts.beta_art * total)
        return cx, cy, cand, restart
    ax, ay, akkt = avg
    if opts.restart_rule == "halving":
        return ax, ay, akkt, akkt <= 0.5 * anchor_kkt
    if opts.restart_rule == "fixed":
        return ax, ay, akkt, k >= opts.fixed_K
    return cx, cy, cand, False


def initialize_primal_weight(c, b, eps_zero):
    """InitializePrimalWeight: ||c||_2 / ||b||_2 if both exceed eps_zero, else 1."""
    nc, nb = float(np.linalg.norm(c)), float(np.linalg.norm(b))
    return nc / nb if (nc > eps_zero and nb > eps_zero) else 1.0


def primal_weight_update(z_new, z_old, omega, theta, eps_zero):
    """PrimalWeightUpdate: exp(theta log(dy/dx) + (1-theta) log omega) with
    dx = ||x^{n,0} - x^{n-1,0}||_2, dy likewise; unchanged if either is tiny."""
    dx = float(np.linalg.norm(z_new[0] - z_old[0]))
    dy = float(np.linalg.norm(z_new[1] - z_old[1]))
    if dx > eps_zero and dy > eps_zero:
        return math.exp(theta * math.log(dy / dx) + (1.0 - theta) * math.log(omega))
    return omega

# ---------------------------------------------------------------------------
# Infeasibility certificates (R18; not in the paper)
# ---------------------------------------------------------------------------
def recession_project(d, l, u):
    """Projection onto the recession cone of X = [l, u]: {0} where both bounds
    are finite, [0, inf) where only l is, (-inf, 0] where only u is, R else."""
    lo, up = np.isfinite(l), np.isfinite(u)
    return np.where(lo & up, 0.0, np.where(lo, np.maximum(d, 0.0), np.where(up, np.minimum(d, 0.0), d)))


def _inf_norm(v) -> float:
    return float(np.max(np.abs(v))) if v.size else 0.0


def dual_ray_value(p: Problem, rho: np.ndarray, eps: float) -> float:
    """Farkas test for primal infeasibility.  For rho with rho_I >= 0 and every
    feasible x, b'rho <= rho'Ax <= sigma_X(A'rho) (sigma_X the support function
    of the box); so b'rho - sigma_X(A'rho) > 0 proves that no x is feasible.
    With lam = proj_Lambda(-A'rho), b'rho + l'lam+ - u'lam- is that value on the
    part of -A'rho inside Lambda (where sigma_X is finite) and |-A'rho - lam|_inf
    is what leaves it.  Returns the value when it is positive and the residual
    is at most eps times it, else 0."""
    g = -(p.A.T @ rho)
    lo, up = np.isfinite(p.l), np.isfinite(p.u)
    lam = np.where(lo & up, g, np.where(lo, np.maximum(g, 0.0), np.where(up, np.minimum(g, 0.0), 0.0)))
    lam_pos, lam_neg = np.maximum(lam, 0.0), np.maximum(-lam, 0.0)
    value = float(p.b @ rho) + float(np.sum(np.where(lam_pos > 0, p.l, 0.0) * lam_pos)
                                     - np.sum(np.where(lam_neg > 0, p.u, 0.0) * lam_neg))
    return value if (value > 0 and _inf_norm(g - lam) <= eps * value) else 0.0


def primal_ray_value(p: Problem, d: np.ndarray, eps: float) -> float:
    """Test of d (in the recession cone of X) as a direction of unbounded
    descent: c'd < 0, Qd = 0, A_E d = 0, A_I d >= 0, the last three to eps
    times |c'd|.  Returns |c'd| when d passes, else 0."""
    cd = float(p.c @ d)
    if not cd < 0:
        return 0.0
    Ad = p.A @ d
    viol = np.abs(Ad)
    viol[p.m_eq:] = np.maximum(-Ad[p.m_eq:], 0.0)
    worst = max(_inf_norm(viol), _inf_norm(p.Qmul(d)))
    return -cd if worst <= eps * (-cd) else 0.0


def find_certificate(p: Problem, ps: Problem, D1, D2, iterates, anchor, eps: float):
    """R18: the rays of the current and the average iterate (in that order),
    tested for primal infeasibility first.  Returns (status, x, y) with the
    normalised certificate -- y with b'y - sigma_X(A'y) = 1, or d with c'd = -1
    -- or None."""
    rays = []
    for xs, ys in iterates:
        d = D2 * recession_project(xs - anchor[0], ps.l, ps.u)
        rho = D1 * proj_Y(ys - anchor[1], p.m_eq)
        rays.append((d, rho))
    for d, rho in rays:
        v = dual_ray_value(p, rho, eps)
        if v > 0:
            return "primal_infeasible", np.zeros(p.n), rho / v
    for d, rho in rays:
        v = primal_ray_value(p, d, eps)
        if v > 0:
            return "dual_infeasible", d / v, np.zeros(p.m)
    return None


# ---------------------------------------------------------------------------
# Solver
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Options:
    eps: float = 1e-6
    max_iter: int = 200_000
    check_period: int = 64
    restart_rule: str = "pdqp"        # "pdqp" | "halving" | "fixed" | "none"
    step_rule: str = "adaptive"       # "adaptive" | "theory"
    accelerate: bool = True
    scaling: bool = True
    ruiz_iters: int = 10
    l2_scaling: bool = True
    pock_chambolle: bool = True
    fixed_K: int = 64
    beta_suff: float = 0.2
    beta_nec: float = 0.8
    beta_art: float = 0.36
    pw_theta: float = 0.2
    eps_zero: float = 1e-10
    norm_A: float = 0.0               # <= 0: Lanczos estimate (R10)
    norm_Q: float = 0.0
    norm_iters: int = 500
    norm_tol: float = 1e-6
    detect_infeasibility: bool = False   # R18
    eps_infeasible: float = 1e-8


@dataclasses.dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    status: str                       # "optimal" | "iteration_limit" | "primal_infeasible" | "dual_infeasible"
    iterations: int
    restarts: int
    kkt: Dict[str, float]
    omega: float
    norm_A: float
    norm_Q: float
    D1: np.ndarray
    D2: np.ndarray
    trace: Dict[int, Dict[str, np.ndarray]]
    checks: List[Dict[str, float]]


def solve(inst_or_problem, opts: Optional[Options] = None, x0=None, y0=None,
          trace_at=()) -> Result:
    """rAPDHG (Algorithm 1 with the Section 6 rules).  `trace_at` lists total
    iteration counts at which the raw iterate state (after that iteration's
    update, before any relKKT check) is recorded in original coordinates."""
    opts = opts or Options()
    p = inst_or_problem if isinstance(inst_or_problem, Problem) else problem_from_instance(inst_or_problem)
    n, m, m_eq = p.n, p.m, p.m_eq

    # -- preprocessing (Section 5) --
    if opts.scaling:
        D1, D2 = scaling_factors(p, opts.ruiz_iters, opts.l2_scaling, opts.pock_chambolle)
    else:
        D1, D2 = np.ones(m), np.ones(n)
    ps = scale_problem(p, D1, D2)
    nA = opts.norm_A if opts.norm_A > 0 else norm_A(ps, max_iter=opts.norm_iters, tol=opts.norm_tol)
    nQ = opts.norm_Q if opts.norm_Q > 0 else norm_Q(ps, max_iter=opts.norm_iters, tol=opts.norm_tol)

    unscale = lambda xs, ys: (D2 * xs, D1 * ys)

    # -- initial point (x^{0,0}, y^{0,0}); zeros by default (Section 5 "Algorithms") --
    x = proj_X(np.zeros(n) if x0 is None else np.asarray(x0, np.float64) / D2, ps.l, ps.u)
    y = proj_Y(np.zeros(m) if y0 is None else np.asarray(y0, np.float64) / D1, m_eq)

    # -- primal weight initialisation (Section 6) --
    omega = initialize_primal_weight(ps.c, ps.b, opts.eps_zero)

    x_prev, xbar, ybar = x.copy(), x.copy(), y.copy()
    anchor_x, anchor_y = x.copy(), y.copy()
    anchor_kkt = rel_kkt(p, *unscale(x, y))
    prev_cand_kkt = None
    k = 0            # inner iteration counter of the current epoch
    total = 0        # total iterations
    restarts = 0
    eta = 0.0
    trace: Dict[int, Dict[str, np.ndarray]] = {}
    checks: List[Dict[str, float]] = []
    trace_at = set(int(t) for t in trace_at)

    def finish(xs, ys, status):
        xo, yo = unscale(xs, ys)
        return Result(xo, yo, status, total, restarts, kkt_parts(p, xo, yo), omega, nA, nQ,
                      D1, D2, trace, checks)

    if anchor_kkt <= opts.eps:
        return finish(x, y, "optimal")

    while True:
        # ---- step sizes for inner iteration k ----
        beta, theta = beta_theta(k, opts.accelerate)
        if opts.step_rule == "theory":
            tau_p, sigma_d = theory_steps(k, opts.fixed_K, nQ, nA)
        else:
            eta = pdqp_eta(k if opts.accelerate else 0, eta, nQ, nA, omega)
            tau_p, sigma_d = eta / omega, eta * omega

        # ---- one inner iteration of Algorithm 1 ----
        x_md = (1.0 - 1.0 / beta) * xbar + x / beta
        x_tilde = x + theta * (x - x_prev)
        y_new = proj_Y(y - sigma_d * (ps.A @ x_tilde - ps.b), m_eq)
        x_new = proj_X(x - tau_p * (ps.Qmul(x_md) + ps.c - ps.A.T @ y_new), ps.l, ps.u)
        xbar = (1.0 - 1.0 / beta) * xbar + x_new / beta
        ybar = (1.0 - 1.0 / beta) * ybar + y_new / beta
        x_prev, x, y = x, x_new, y_new
        k += 1
        total += 1

        if total in trace_at:
            xo, yo = unscale(x, y)
            xbo, ybo = unscale(xbar, ybar)
            trace[total] = dict(x=xo, y=yo, xbar=xbo, ybar=ybo, k=k, omega=omega,
                                tau_p=tau_p, sigma_d=sigma_d)

        # ---- relKKT check (R7) ----
        if total % opts.check_period != 0 and total != opts.max_iter:
            continue
        kkt_cur = rel_kkt(p, *unscale(x, y))
        kkt_avg = rel_kkt(p, *unscale(xbar, ybar))
        cx, cy, cand_kkt = get_restart_candidate((x, y, kkt_cur), (xbar, ybar, kkt_avg))
        rec = dict(total=total, k=k, kkt_cur=kkt_cur, kkt_avg=kkt_avg, anchor_kkt=anchor_kkt,
                   omega=omega, restart=0)
        checks.append(rec)
        if cand_kkt <= opts.eps:
            return finish(cx, cy, "optimal")
        if total >= opts.max_iter:
            return finish(cx, cy, "iteration_limit")
        if opts.detect_infeasibility:
            cert = find_certificate(p, ps, D1, D2, ((x, y), (xbar, ybar)), (anchor_x, anchor_y),
                                    opts.eps_infeasible)
            if cert is not None:
                rec["infeasible"] = cert[0]
                return Result(cert[1], cert[2], cert[0], total, restarts, kkt_parts(p, cert[1], cert[2]),
                              omega, nA, nQ, D1, D2, trace, checks)

        cx, cy, cand_kkt, restart = restart_decision(
            opts, (x, y, kkt_cur), (xbar, ybar, kkt_avg), anchor_kkt, prev_cand_kkt, k, total)

        if not restart:
            prev_cand_kkt = cand_kkt
            continue
        # ---- restart the outer loop from the candidate ----
        rec["restart"] = 1
        restarts += 1
        if opts.step_rule == "adaptive":
            omega = primal_weight_update((cx, cy), (anchor_x, anchor_y), omega,
                                         opts.pw_theta, opts.eps_zero)
        x, y = cx.copy(), cy.copy()
        x_prev, xbar, ybar = x.copy(), x.copy(), y.copy()
        anchor_x, anchor_y, anchor_kkt = x.copy(), y.copy(), cand_kkt
        prev_cand_kkt = None
        k = 0
