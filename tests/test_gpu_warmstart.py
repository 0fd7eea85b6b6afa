"""The warm-start network's CUDA forward, backward, Adam, normalisation and
inference against the CPU oracle (oracle/warmstart.py) on the same bf16
parameters and data.

The oracle rounds to bf16 / float32 where the device stores those types and
sums in float64, so the remaining differences are the float32 summation order
of the tensor-core products (relative ~1e-6) and the rare bf16 rounding it
flips (one bf16 ulp, 2^-8, in a few elements).  A pre-activation within that
summation error of zero could take the other side of the ReLU on the device,
which switches a whole unit of one sample on or off and moves every gradient
below it by up to a few percent; the tests therefore set the hidden biases so
that every pre-activation of the test batch is at least 10% of its unit's
range away from zero (a quarter of the units always off, the rest always on).
Tolerances: relative Frobenius error 1e-3 and largest element error 1e-2 of
the largest element for gradients, 1e-5 relative for losses."""
import numpy as np
import pytest

import qpgen
from oracle import warmstart as WS
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


def separate_units(layers, proj, U, margin=0.1):
    """Hidden biases that keep every pre-activation of the batch U at least
    margin * (its unit's range) away from zero: units 0, 4, 8, ... always off,
    the others always on."""
    rb = WS.bf16_round
    h = rb(U @ rb(proj.astype(np.float64)).T)
    out = []
    for W, _ in layers[:-1]:
        z = h @ rb(W.astype(np.float64)).T
        lo, hi = z.min(axis=0), z.max(axis=0)
        pad = margin * np.maximum(hi - lo, 1e-3) + margin
        off = (np.arange(W.shape[0]) % 4) == 0
        b = np.where(off, -hi - pad, -lo + pad).astype(np.float32)
        out.append((W, b))
        h = rb(np.maximum(z + b, 0.0))
    out.append(layers[-1])
    return out


def make_net(pd, n, m, d, width, depth, maxb, seed, out_scale=1.0, separate_on=None):
    """separate_on: (C, B, norm) of the batch whose ReLU decisions must be unambiguous."""
    proj, layers = qpgen.warmstart_params(seed, n + m, d, width, depth)
    W, b = layers[-1]
    layers[-1] = ((W * out_scale).astype(np.float32), b)
    if separate_on is not None:
        C, B, norm = separate_on
        layers = separate_units(layers, proj, WS.prep_input(C, B, norm), margin=0.1)
    w = pd.pdqp_ws_create(n, m, d, width, depth, maxb)
    pd.pdqp_ws_set_params(w, -1, proj)
    for j, (Wj, bj) in enumerate(layers):
        pd.pdqp_ws_set_params(w, j, Wj, bj)
    return w, proj.astype(np.float64), [(Wj.astype(np.float64), bj.astype(np.float64)) for Wj, bj in layers]


def data(seed, count, n, m):
    rng = np.random.default_rng(seed)
    C = 1.0 + 0.3 * rng.standard_normal((count, n))
    B = -2.0 + 0.5 * rng.standard_normal((count, m))
    V = np.hstack([C, B])
    X = V[:, :n] * 0.7 + 0.2 * rng.standard_normal((count, n))
    Y = np.tanh(V[:, V.shape[1] - m:]) + 0.1 * rng.standard_normal((count, m))
    return C, B, X, Y


def set_norm(pd, w, norm):
    pd.pdqp_ws_set_normalization(w, norm["in_mean"], norm["in_scale"], norm["out_mean"], norm["out_std"],
                                 norm["out_inv"])


def read(pd, w, layer, what, shape):
    W = np.zeros(shape, np.float32)
    b = np.zeros(shape[0], np.float32)
    pd.pdqp_ws_get_params(w, layer, what, W, b)
    return W.astype(np.float64), b.astype(np.float64)


def close_grad(got, want, what):
    fro = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
    big = np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)
    assert fro <= 1e-3 and big <= 1e-2, (what, fro, big)


@pytest.mark.parametrize("n,m,d,width,depth,count,maxb", [
    (37, 23, 64, 96, 3, 48, 64),        # F = 60: padded leading dimensions, single tiles
    (200, 100, 128, 256, 3, 160, 160),  # several tiles in every product, ragged batch
    (300, 0, 64, 128, 1, 40, 40),       # no rows (m = 0), one hidden layer
])
def test_gradients_match_oracle(n, m, d, width, depth, count, maxb):
    pd = lib()
    C, B, X, Y = data(n * 3 + m, count, n, m)
    norm = WS.fit_normalization(C, B, X, Y)
    w, proj, layers = make_net(pd, n, m, d, width, depth, maxb, seed=n + m, out_scale=30.0,
                               separate_on=(C, B, norm))
    try:
        set_norm(pd, w, norm)
        loss = pd.pdqp_ws_grad(w, C, B, X, Y)
        U = WS.prep_input(C, B, norm)
        T = WS.prep_target(X, Y, norm)
        want_loss, grads = WS.loss_and_grads(layers, proj, U, T, mimic=True)
        assert abs(loss - want_loss) <= 1e-5 * want_loss
        for j, (gW, gb) in enumerate(grads):
            W, b = read(pd, w, j, 1, gW.shape)
            close_grad(W, gW, f"dW{j}")
            close_grad(b, gb, f"db{j}")
    finally:
        pd.pdqp_ws_destroy(w)


def test_fit_matches_oracle():
    pd = lib()
    n, m = 50, 30
    w, _, _ = make_net(pd, n, m, 32, 32, 1, 32, seed=1)
    try:
        C, B, X, Y = data(2, 300, n, m)
        X[:, 3] = 5.0                                   # a constant target feature
        pd.pdqp_ws_fit(w, C, B, X, Y)
        got = pd.pdqp_ws_get_normalization(w, n + m)
        want = WS.fit_normalization(C, B, X, Y)
        for k in want:
            np.testing.assert_allclose(got[k], want[k], rtol=2e-7, atol=0, err_msg=k)
        assert got["out_std"][3] == 1.0
    finally:
        pd.pdqp_ws_destroy(w)


def test_one_adam_step_matches_oracle():
    pd = lib()
    n, m, d, width, depth, batch = 60, 20, 64, 64, 2, 32
    C, B, X, Y = data(8, batch, n, m)
    norm = WS.fit_normalization(C, B, X, Y)
    w, proj, layers = make_net(pd, n, m, d, width, depth, batch, seed=7, out_scale=30.0, separate_on=(C, B, norm))
    try:
        set_norm(pd, w, norm)
        lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
        losses = pd.pdqp_ws_train(w, C, B, X, Y, epochs=1, batch=batch, lr=lr, beta1=b1, beta2=b2, eps=eps, seed=3)
        U = WS.prep_input(C, B, norm)
        T = WS.prep_target(X, Y, norm)
        want_loss, grads = WS.loss_and_grads(layers, proj, U, T, mimic=True)
        assert abs(losses[0] - want_loss) <= 1e-5 * want_loss
        for j, (W0, b0) in enumerate(layers):
            gW, gb = read(pd, w, j, 1, W0.shape)
            close_grad(gW, grads[j][0], f"dW{j}")
            W1, b1v = read(pd, w, j, 0, W0.shape)
            mW, mb = read(pd, w, j, 2, W0.shape)
            vW, vb = read(pd, w, j, 3, W0.shape)
            for p0, g, p1, mm, vv in ((W0, gW, W1, mW, vW), (b0, gb, b1v, mb, vb)):
                want_p, want_m, want_v = WS.adam_step(p0, g, 0.0, 0.0, 1, lr, b1, b2, eps)
                np.testing.assert_allclose(p1, want_p, rtol=0, atol=2e-7 * np.abs(p0).max() + 1e-3 * lr)
                np.testing.assert_allclose(mm, want_m, rtol=1e-6, atol=1e-30)
                # (1 - beta2) in float32 is 0.0009999871: relative 1.3e-5
                np.testing.assert_allclose(vv, want_v, rtol=5e-5, atol=1e-36)
    finally:
        pd.pdqp_ws_destroy(w)


def test_training_follows_oracle_visit_order():
    # two minibatches per epoch: the weights after the epoch depend on which
    # samples went into which step, so they pin the visit order as well
    pd = lib()
    n, m, d, width, depth, batch = 24, 16, 32, 32, 2, 16
    C, B, X, Y = data(10, 3 * batch + 5, n, m)     # 3 steps per epoch, 5 samples dropped
    norm = WS.fit_normalization(C, B, X, Y)
    w, proj, layers = make_net(pd, n, m, d, width, depth, 2 * batch, seed=9, out_scale=10.0,
                               separate_on=(C, B, norm))
    try:
        set_norm(pd, w, norm)
        losses = pd.pdqp_ws_train(w, C, B, X, Y, epochs=3, batch=batch, lr=3e-3, seed=21)
        want_layers, want_losses = WS.train(layers, proj, C, B, X, Y, norm, epochs=3, batch=batch, lr=3e-3,
                                            seed=21, mimic=True)
        np.testing.assert_allclose(losses, want_losses, rtol=1e-3)
        for j, (Ww, bw) in enumerate(want_layers):
            W, b = read(pd, w, j, 0, Ww.shape)
            dW = W - layers[j][0]
            dWw = Ww - layers[j][0]
            assert np.linalg.norm(dW - dWw) <= 2e-2 * np.linalg.norm(dWw), j
    finally:
        pd.pdqp_ws_destroy(w)


@pytest.mark.parametrize("count", [5, 130])
def test_infer_matches_oracle(count):
    pd = lib()
    n, m, d, width, depth = 90, 45, 64, 128, 3
    w, proj, layers = make_net(pd, n, m, d, width, depth, 64, seed=11, out_scale=30.0)
    try:
        C, B, X, Y = data(12, count, n, m)
        norm = WS.fit_normalization(C, B, X, Y)
        set_norm(pd, w, norm)
        X0 = np.zeros((count, n))
        Y0 = np.zeros((count, m))
        pd.pdqp_ws_infer(w, C, B, X0, Y0)               # count > max_batch runs in chunks
        _, O = WS.forward(layers, proj, WS.prep_input(C, B, norm), mimic=True)
        x0, y0 = WS.prediction(O, norm, n)
        scale = norm["out_std"].astype(np.float64) * (1.0 + np.abs(O))
        assert np.all(np.abs(np.hstack([X0, Y0]) - np.hstack([x0, y0])) <= 3e-2 * scale)
        assert np.linalg.norm(np.hstack([X0, Y0]) - np.hstack([x0, y0])) <= 3e-3 * np.linalg.norm(np.hstack([x0, y0]))
        # device arrays give the same answer
        import torch
        X0d = torch.zeros((count, n), dtype=torch.float64, device="cuda")
        Y0d = torch.zeros((count, m), dtype=torch.float64, device="cuda")
        pd.pdqp_ws_infer(w, torch.from_numpy(C).cuda(), torch.from_numpy(B).cuda(), X0d, Y0d)
        np.testing.assert_array_equal(X0d.cpu().numpy(), X0)
        np.testing.assert_array_equal(Y0d.cpu().numpy(), Y0)
    finally:
        pd.pdqp_ws_destroy(w)


def test_invalid_calls_are_rejected():
    pd = lib()
    with pytest.raises(pd.PdqpError):
        pd.pdqp_ws_create(10, 5, 12, 16, 1, 16)      # d not a multiple of 8
    with pytest.raises(pd.PdqpError):
        pd.pdqp_ws_create(10, 5, 16, 16, 0, 16)      # depth 0
    w = pd.pdqp_ws_create(10, 5, 16, 16, 1, 16)
    try:
        C, B, X, Y = data(1, 16, 10, 5)
        with pytest.raises(pd.PdqpError):             # no normalisation / projection yet
            pd.pdqp_ws_grad(w, C, B, X, Y)
        pd.pdqp_ws_fit(w, C, B, X, Y)
        with pytest.raises(pd.PdqpError):
            pd.pdqp_ws_grad(w, C, B, X, Y)            # projection still missing
        proj, layers = qpgen.warmstart_params(0, 15, 16, 16, 1)
        pd.pdqp_ws_set_params(w, -1, proj)
        pd.pdqp_ws_grad(w, C, B, X, Y)
        with pytest.raises(pd.PdqpError):
            pd.pdqp_ws_train(w, C, B, X, Y, epochs=1, batch=12)   # batch not a multiple of 8
        with pytest.raises(pd.PdqpError):
            pd.pdqp_ws_train(w, C[:8], B[:8], X[:8], Y[:8], epochs=1, batch=16)   # count < batch
        with pytest.raises(pd.PdqpError):
            pd.pdqp_ws_set_params(w, 2, layers[0][0])            # layer out of range
    finally:
        pd.pdqp_ws_destroy(w)
