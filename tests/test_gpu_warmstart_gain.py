"""What the learned warm start gains: a network trained by the library's own
kernels on solutions the solver produced for a parameterised family (the
configuration-0 pattern at n = 400, m = 200 with c = c_bar + 0.1 N(0,1),
b = b_bar + 0.1 N(0,1)) cuts the iterations of held-out solves, beats the
mean-solution start, and leaves the answers where the cold start puts them:
every solve still ends at relKKT <= 1e-6 by the solver's own test."""
import numpy as np
import pytest

import qpgen
from oracle import rapdhg as R
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


def solve_family(pd, base, C, B, X0=None, Y0=None, precision=1, chunk=2048):
    Xs, Ys, infos = [], [], []
    for s0 in range(0, C.shape[0], chunk):
        c, b = C[s0:s0 + chunk], B[s0:s0 + chunk]
        h = pd.family_from_base(base, c, b)
        try:
            x, y = np.zeros(c.size), np.zeros(b.size)
            x0 = None if X0 is None else np.ascontiguousarray(X0[s0:s0 + chunk]).ravel()
            y0 = None if Y0 is None else np.ascontiguousarray(Y0[s0:s0 + chunk]).ravel()
            pd.pdqp_solve(h, pd.pdqp_default_options(precision=precision), x0=x0, y0=y0, x_out=x, y_out=y)
            infos += pd.pdqp_batch_info(h)
        finally:
            pd.pdqp_destroy(h)
        Xs.append(x.reshape(c.shape))
        Ys.append(y.reshape(b.shape))
    return np.vstack(Xs), np.vstack(Ys), infos


def test_learned_warm_start_saves_iterations():
    pd = lib()
    fam = qpgen.family_qp(n=400, m=200)
    n, m = fam.base.n, fam.base.m
    Ctr, Btr = fam.params(0, 8192)
    Cte, Bte = fam.params(1_000_000, 256)
    X, Y, info_tr = solve_family(pd, fam.base, Ctr, Btr)
    assert all(i.status == pd.PDQP_OK for i in info_tr)

    proj, layers = qpgen.warmstart_params(7, n + m, 512, 512, 3)
    w = pd.pdqp_ws_create(n, m, 512, 512, 3, 512)
    try:
        pd.pdqp_ws_set_params(w, -1, proj)
        for j, (W, b) in enumerate(layers):
            pd.pdqp_ws_set_params(w, j, W, b)
        pd.pdqp_ws_fit(w, Ctr, Btr, X, Y)
        losses = pd.pdqp_ws_train(w, Ctr, Btr, X, Y, epochs=30, batch=256, lr=1e-3, seed=1)
        assert losses[-1] < 0.5 * losses[0]
        X0 = np.zeros((256, n))
        Y0 = np.zeros((256, m))
        pd.pdqp_ws_infer(w, Cte, Bte, X0, Y0)
    finally:
        pd.pdqp_ws_destroy(w)

    Xc, Yc, cold = solve_family(pd, fam.base, Cte, Bte)
    Xw, Yw, warm = solve_family(pd, fam.base, Cte, Bte, X0, Y0)
    Xm = np.broadcast_to(X.mean(axis=0), X0.shape).copy()
    Ym = np.broadcast_to(Y.mean(axis=0), Y0.shape).copy()
    _, _, mean = solve_family(pd, fam.base, Cte, Bte, Xm, Ym)

    # the prediction is closer to the solutions than the mean solution is
    err = lambda P, Q: np.linalg.norm(P - Q) / np.linalg.norm(Q)
    assert err(np.hstack([X0, Y0]), np.hstack([Xc, Yc])) < 0.8 * err(np.hstack([Xm, Ym]), np.hstack([Xc, Yc]))
    # every solve ends where the solver's own test says it must
    for infos in (cold, warm, mean):
        assert all(i.status == pd.PDQP_OK and i.rel_kkt <= 1e-6 for i in infos)
    it = {k: np.mean([i.iterations for i in v]) for k, v in (("cold", cold), ("warm", warm), ("mean", mean))}
    assert it["warm"] <= 0.85 * it["cold"], it
    assert it["warm"] < it["mean"], it
    # the answers agree with the cold start to the tolerance (objective within 1e-6)
    for k in range(0, 256, 51):
        inst = qpgen.QPInstance("member", n, m, fam.base.m_eq, fam.base.Q, fam.base.A, Cte[k], Bte[k],
                                fam.base.l, fam.base.u)
        p = R.problem_from_instance(inst)
        pc = R.kkt_parts(p, Xc[k], Yc[k])["primal_obj"]
        pw = R.kkt_parts(p, Xw[k], Yw[k])["primal_obj"]
        assert abs(pc - pw) <= 4e-6 * (1 + abs(pc)), k
