"""The maintained-products scheme (options.maintained_products) restated in
numpy and held to the oracle's direct iteration (Algorithm 1, Section 2;
Theorem 1's beta_k, theta_k): the products of each new primal iterate are
formed once (A x^{k+1}, Q x^{k+1}; A'y^{k+1} from the new dual iterate), the
extrapolated and averaged points' products follow by the linear updates

    A x_tilde^k  = A x^k + theta_k (A x^k - A x^{k-1})
    Q x_md^k     = (1 - 1/beta_k) Q x_bar^k + Q x^k / beta_k
    M z_bar^{k+1} = (1 - 1/beta_k) M z_bar^k + M z^{k+1} / beta_k   (M z = A x, Q x, A'y)

and the epoch's first iteration (k = 0, after a restart to the average)
starts them from the products of the restart point.  Agreement to 1e-12 over
200 iterations with restarts pins the indices the kernels use; the planted
index mistakes below each fail it."""
import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R

TOL = 1e-12


def _maintained(ps, x, y, omega, nA, nQ, iters, K, accelerate=True, pw_theta=0.2, eps_zero=1e-10,
                theta_shift=0, beta_prev=False):
    """Fixed-length restarts to the average every K iterations (the fixed rule:
    its decisions need no relKKT).  theta_shift / beta_prev plant mistakes:
    theta_{k+shift} in the extrapolation, 1/beta_{k-1} in the averages."""
    A, AT = ps.A, ps.A.T.tocsr()
    Ax, Qx, ATy = A @ x, ps.Qmul(x), AT @ y
    Ax_prev = Ax.copy()
    Axb, Qxb, ATyb = Ax.copy(), Qx.copy(), ATy.copy()
    xbar, ybar = x.copy(), y.copy()
    anchor = (x.copy(), y.copy())
    k, eta = 0, 0.0
    for _ in range(iters):
        beta, _theta = R.beta_theta(k, accelerate)
        theta = R.beta_theta(max(k + theta_shift, 0), accelerate)[1]
        ib = 1.0 / (R.beta_theta(k - 1, accelerate)[0] if (beta_prev and k > 0) else beta)
        eta = R.pdqp_eta(k if accelerate else 0, eta, nQ, nA, omega)
        tau, sigma = eta / omega, eta * omega
        Axt = Ax + theta * (Ax - Ax_prev)
        y_new = R.proj_Y(y - sigma * (Axt - ps.b), ps.m_eq)
        ATy_new = AT @ y_new
        Qmd = (1.0 - 1.0 / beta) * Qxb + Qx / beta
        x_new = R.proj_X(x - tau * (Qmd + ps.c - ATy_new), ps.l, ps.u)
        Ax_new, Qx_new = A @ x_new, ps.Qmul(x_new)
        xbar = (1.0 - ib) * xbar + ib * x_new
        ybar = (1.0 - ib) * ybar + ib * y_new
        Axb = (1.0 - ib) * Axb + ib * Ax_new
        Qxb = (1.0 - ib) * Qxb + ib * Qx_new
        ATyb = (1.0 - ib) * ATyb + ib * ATy_new
        Ax_prev, x, y = Ax, x_new, y_new
        Ax, Qx, ATy = Ax_new, Qx_new, ATy_new
        k += 1
        if k >= K:   # restart to the average: its products are the averaged ones
            omega = R.primal_weight_update((xbar, ybar), anchor, omega, pw_theta, eps_zero)
            x, y = xbar.copy(), ybar.copy()
            Ax, Qx, ATy = Axb.copy(), Qxb.copy(), ATyb.copy()
            Ax_prev = Ax.copy()
            anchor = (x.copy(), y.copy())
            k = 0
    return dict(x=x, y=y, xbar=xbar, ybar=ybar, Axb=Axb, Qxb=Qxb, ATyb=ATyb)


def _case(accelerate=True, seed=5):
    inst = qpgen.tiny_qp(seed, n=37, m=29, m_eq=9, bounds="mixed", density=0.3)
    o = R.Options(scaling=False, restart_rule="fixed", fixed_K=32, check_period=32, max_iter=200, eps=0.0,
                  accelerate=accelerate)
    ref = R.solve(inst, o, trace_at=(200,))
    p = R.problem_from_instance(inst)
    x = R.proj_X(np.zeros(p.n), p.l, p.u)
    y = R.proj_Y(np.zeros(p.m), p.m_eq)
    omega = R.initialize_primal_weight(p.c, p.b, o.eps_zero)
    return p, x, y, omega, ref


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


@pytest.mark.parametrize("accelerate", [True, False], ids=["rapdhg", "pdhg"])
def test_scheme_matches_direct_iteration(accelerate):
    p, x, y, omega, ref = _case(accelerate)
    assert sum(c["restart"] for c in ref.checks) >= 5
    got = _maintained(p, x, y, omega, ref.norm_A, ref.norm_Q, 200, 32, accelerate=accelerate)
    for key in ("x", "y", "xbar", "ybar"):
        assert _rel(got[key], ref.trace[200][key]) <= TOL, key
    # the maintained averages are the products of the averaged iterates
    assert _rel(got["Axb"], p.A @ got["xbar"]) <= TOL
    assert _rel(got["Qxb"], p.Qmul(got["xbar"])) <= TOL
    assert _rel(got["ATyb"], p.A.T @ got["ybar"]) <= TOL


@pytest.mark.parametrize("plant", ["theta_next", "theta_prev", "beta_prev"])
def test_planted_index_mistakes_fail(plant):
    p, x, y, omega, ref = _case()
    kw = dict(theta_next=dict(theta_shift=1), theta_prev=dict(theta_shift=-1), beta_prev=dict(beta_prev=True))[plant]
    got = _maintained(p, x, y, omega, ref.norm_A, ref.norm_Q, 200, 32, **kw)
    assert max(_rel(got[k], ref.trace[200][k]) for k in ("x", "y", "xbar", "ybar")) > 1e-6, plant
