"""Pins of the oracle's low-rank term (R14: Q_total = Q + F F' applied as
F(F'x), F left out of the scaling norms, D2 scaling F's rows): solves through
that route reach the optimum of the dense Q + F F' -- its closed form for an
unconstrained problem, brute-force active-set enumeration for a small
portfolio -- with and without scaling; dropping the term or scaling F the
wrong way is caught."""
import sys
import types

import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import rapdhg as R
from tests.qp_truth import active_set_solve
from tests.test_oracle_mutations import ORACLE_SRC


def _unconstrained(seed=3, n=9, r=2):
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.5, 2.0, n)
    F = 0.5 * rng.standard_normal((n, r))
    c = rng.standard_normal(n)
    inst = qpgen.QPInstance("lowrank_free", n, 0, 0, sp.csr_matrix(sp.diags(d)), sp.csr_matrix((0, n)), c,
                            np.zeros(0), np.full(n, -np.inf), np.full(n, np.inf), F=F)
    return inst, np.linalg.solve(np.diag(d) + F @ F.T, -c)


def _portfolio(seed=4, n=7, r=3):
    """min 1/2 x'(D + F F')x - 0.1 mu'x s.t. sum x = 1, mu'x >= 0.05, 0 <= x <= 0.4."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.01, 0.1, n)
    F = 0.3 * rng.standard_normal((n, r))
    mu = rng.normal(0.05, 0.02, n)
    A = np.vstack([np.ones(n), mu])
    inst = qpgen.QPInstance("lowrank_portfolio", n, 2, 1, sp.csr_matrix(sp.diags(d)), sp.csr_matrix(A),
                            -0.1 * mu, np.array([1.0, 0.05]), np.zeros(n), np.full(n, 0.4), F=F)
    truth = active_set_solve(np.diag(d) + F @ F.T, A, inst.b, inst.c, inst.l, inst.u, 1)
    return inst, truth[0]


@pytest.mark.parametrize("scaling", [False, True], ids=["unscaled", "scaled"])
def test_unconstrained_lowrank_closed_form(scaling):
    inst, xstar = _unconstrained()
    r = R.solve(inst, R.Options(eps=1e-10, scaling=scaling))
    assert r.status == "optimal"
    np.testing.assert_allclose(r.x, xstar, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("scaling", [False, True], ids=["unscaled", "scaled"])
def test_portfolio_lowrank_brute_force(scaling):
    inst, xstar = _portfolio()
    r = R.solve(inst, R.Options(eps=1e-10, scaling=scaling, max_iter=400_000))
    assert r.status == "optimal"
    np.testing.assert_allclose(r.x, xstar, atol=1e-6)


MUTATIONS = {
    "drop_lowrank_term": ("out = out + self.F @ (self.F.T @ v)", "pass"),
    "F_scaled_inversely": ("F = None if p.F is None else p.F * D2[:, None]",
                           "F = None if p.F is None else p.F / D2[:, None]"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_lowrank_mistakes_are_caught(name):
    src = open(ORACLE_SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1
    mod = types.ModuleType("oracle_lowrank_mutant_" + name)
    sys.modules[mod.__name__] = mod
    exec(compile(src.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    inst, xstar = _unconstrained()
    r = mod.solve(inst, mod.Options(eps=1e-10, scaling=True, max_iter=20_000))
    assert not (r.status == "optimal" and np.allclose(r.x, xstar, rtol=1e-7, atol=1e-8))
