"""Ground truth for tiny QPs, independent of the oracle's iteration.

* `active_set_solve`: brute-force enumeration of active sets.  For every
  assignment of each variable to {at l, at u, free} (finite bounds only) and
  each inequality row to {active, inactive} it solves the equality-constrained
  KKT system with numpy's dense solver and keeps the points satisfying every
  KKT condition of the QP (primal feasibility, multiplier signs, stationarity).
  For a convex QP any such point is a global optimum.
* `kkt_certificate`: the KKT conditions (eq. (KKT) of Section 3, with bounds
  and equality rows) checked term by term, not through relKKT.
"""
import itertools

import numpy as np


def active_set_solve(Q, A, b, c, l, u, m_eq, tol=1e-9):
    Q = np.asarray(Q, float)
    A = np.asarray(A, float).reshape(-1, Q.shape[0])
    n, m = Q.shape[0], A.shape[0]
    var_choices = []
    for j in range(n):
        ch = ["free"]
        if np.isfinite(l[j]):
            ch.append("l")
        if np.isfinite(u[j]):
            ch.append("u")
        var_choices.append(ch)
    row_choices = [["act"] if i < m_eq else ["act", "ina"] for i in range(m)]
    best = None
    for vs in itertools.product(*var_choices):
        fixed = np.array([v != "free" for v in vs])
        xB = np.array([l[j] if v == "l" else (u[j] if v == "u" else 0.0) for j, v in enumerate(vs)])
        F = np.nonzero(~fixed)[0]
        for rs in itertools.product(*row_choices):
            act = np.array([r == "act" for r in rs], dtype=bool)
            Aa = A[act]
            ba = b[act]
            na = Aa.shape[0]
            nf = F.size
            # unknowns: x_F (nf), y_act (na):  Q_FF x_F - A_aF' y = -c_F - Q_FB x_B
            #                                   A_aF x_F = b_a - A_aB x_B
            K = np.zeros((nf + na, nf + na))
            rhs = np.zeros(nf + na)
            K[:nf, :nf] = Q[np.ix_(F, F)]
            K[:nf, nf:] = -Aa[:, F].T
            K[nf:, :nf] = Aa[:, F]
            rhs[:nf] = -c[F] - Q[np.ix_(F, np.nonzero(fixed)[0])] @ xB[fixed]
            rhs[nf:] = ba - Aa[:, fixed] @ xB[fixed]
            try:
                sol = np.linalg.solve(K, rhs)
            except np.linalg.LinAlgError:
                sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
                if np.linalg.norm(K @ sol - rhs) > 1e-9 * (1 + np.linalg.norm(rhs)):
                    continue
            x = xB.copy()
            x[F] = sol[:nf]
            y = np.zeros(m)
            y[act] = sol[nf:]
            if not kkt_certificate(Q, A, b, c, l, u, m_eq, x, y, tol=tol):
                continue
            obj = 0.5 * x @ Q @ x + c @ x
            if best is None or obj < best[2] - 1e-12:
                best = (x, y, obj)
    return best


def kkt_certificate(Q, A, b, c, l, u, m_eq, x, y, tol=1e-7):
    """True iff (x, y) satisfies the QP's KKT conditions to absolute tolerance tol."""
    Q = np.asarray(Q, float)
    A = np.asarray(A, float).reshape(-1, Q.shape[0])
    scale = 1.0 + np.max(np.abs(np.concatenate([b, c, [0.0]])))
    t = tol * scale
    Ax = A @ x
    if np.any(x < l - t) or np.any(x > u + t):
        return False
    if m_eq and np.max(np.abs(Ax[:m_eq] - b[:m_eq])) > t:
        return False
    if np.any(Ax[m_eq:] < b[m_eq:] - t):
        return False
    if np.any(y[m_eq:] < -t):
        return False
    # complementary slackness on inequality rows
    if np.any(np.abs(y[m_eq:] * (Ax[m_eq:] - b[m_eq:])) > t * scale):
        return False
    g = Q @ x + c - A.T @ y     # = multipliers of the bounds
    at_l = np.abs(x - l) <= t
    at_u = np.abs(x - u) <= t
    interior = ~(at_l | at_u)
    if np.any(np.abs(g[interior]) > t):
        return False
    if np.any(g[at_l & ~at_u] < -t):
        return False
    if np.any(g[at_u & ~at_l] > t):
        return False
    return True
