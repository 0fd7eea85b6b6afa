"""Pins of the warm-start network oracle against facts that do not depend on
it: finite differences of the loss, the closed form of Adam under a constant
gradient, torch's bfloat16 conversion, the invariants of the normalisation and
of the visit order."""
import numpy as np
import pytest

import qpgen
from oracle import warmstart as ws


def tiny_net(seed=3, F=7, d=6, width=5, depth=2):
    proj, layers = qpgen.warmstart_params(seed, F, d, width, depth)
    # a larger output layer than the generator's so the loss depends visibly on it
    W, b = layers[-1]
    layers[-1] = (W * 10.0, b + 0.1)
    layers = [(W.astype(np.float64), b.astype(np.float64) + 0.05) for W, b in layers]
    return proj.astype(np.float64), layers


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-20, 20, 5000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -(1.0 + 2 ** -8), 65504.0, 1e-38]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ws.bf16_round(a), ref)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert ws.bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert ws.bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6


def _flat_loss(layers, proj, U, T):
    loss, _ = ws.loss_and_grads(layers, proj, U, T, mimic=False)
    return loss


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_gradients_match_finite_differences(depth):
    proj, layers = tiny_net(depth=depth)
    rng = np.random.default_rng(depth)
    S, F = 5, proj.shape[1]
    U = rng.standard_normal((S, F))
    T = rng.standard_normal((S, F))
    _, grads = ws.loss_and_grads(layers, proj, U, T, mimic=False)
    h = 1e-6
    for li, (W, b) in enumerate(layers):
        for which, P in ((0, W), (1, b)):
            G = grads[li][which]
            it = np.nditer(P, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = P[idx]
                P[idx] = old + h
                lp = _flat_loss(layers, proj, U, T)
                P[idx] = old - h
                lm = _flat_loss(layers, proj, U, T)
                P[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(G[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (li, which, idx, G[idx], fd)


def test_mimic_stays_within_bf16_error():
    proj, layers = tiny_net()
    rng = np.random.default_rng(9)
    U = rng.standard_normal((16, proj.shape[1]))
    T = rng.standard_normal((16, proj.shape[1]))
    l64, g64 = ws.loss_and_grads(layers, proj, U, T, mimic=False)
    lbf, gbf = ws.loss_and_grads(layers, proj, ws.bf16_round(U), T, mimic=True)
    assert abs(lbf - l64) <= 0.05 * l64
    for (a, b), (c, d) in zip(g64, gbf):
        assert np.linalg.norm(a - c) <= 0.05 * np.linalg.norm(a)
        assert np.linalg.norm(b - d) <= 0.05 * np.linalg.norm(b)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g the bias-corrected moments are exactly g and g^2,
    # so every step moves p by lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        p, m, v = ws.adam_step(p, g, m, v, t, lr, 0.9, 0.999, eps)
        np.testing.assert_allclose(p, -t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_adam_first_step_is_sign_descent():
    rng = np.random.default_rng(1)
    g = rng.standard_normal(50)
    p, _, _ = ws.adam_step(np.ones(50), g, np.zeros(50), np.zeros(50), 1, 0.1, 0.9, 0.999, 0.0)
    np.testing.assert_allclose(p, 1.0 - 0.1 * np.sign(g), rtol=0, atol=1e-14)


@pytest.mark.parametrize("count", [1, 2, 7, 64, 1000, 4096, 10007])
def test_visit_order_is_a_permutation(count):
    for e in range(3):
        order = ws.affine_permutation(count, e, 11)
        assert sorted(order.tolist()) == list(range(count))


def test_splitmix64_reference_values():
    # SplitMix64 from state 0: the first outputs of the published generator
    # (each call adds the golden gamma to the state, then mixes)
    assert ws._mix64(0) == 0xE220A8397B1DCDAF
    assert ws._mix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_normalization_invariants():
    rng = np.random.default_rng(2)
    C = 3.0 + 0.1 * rng.standard_normal((200, 6))
    B = -1.0 + 2.0 * rng.standard_normal((200, 4))
    X = np.hstack([rng.standard_normal((200, 5)), np.full((200, 1), 7.0)])   # a constant column
    Y = rng.standard_normal((200, 4))
    norm = ws.fit_normalization(C, B, X, Y)
    U = ws.prep_input(C, B, norm, mimic=False)
    T = ws.prep_target(X, Y, norm, mimic=False)
    np.testing.assert_allclose(U.mean(0), 0.0, atol=1e-5)
    np.testing.assert_allclose(U.std(0), 1.0, rtol=1e-5)
    np.testing.assert_allclose(T[:, :5].std(0), 1.0, rtol=1e-5)
    assert norm["out_std"][5] == 1.0 and np.all(np.abs(T[:, 5]) < 1e-5)
    x0, y0 = ws.prediction(T, norm, 6)
    np.testing.assert_allclose(np.hstack([x0, y0]), np.hstack([X, Y]), rtol=1e-5, atol=1e-5)


def test_training_fits_a_linear_family():
    # targets linear in the inputs: the network must cut the loss well below
    # that of predicting the mean (normalised loss 1)
    rng = np.random.default_rng(4)
    S, n, m = 256, 12, 4
    C = rng.standard_normal((S, n))
    B = rng.standard_normal((S, m))
    M = rng.standard_normal((n + m, n + m)) / 4
    V = np.hstack([C, B]) @ M
    X, Y = V[:, :n], V[:, n:]
    proj, layers = qpgen.warmstart_params(5, n + m, 32, 32, 2)
    norm = ws.fit_normalization(C, B, X, Y)
    _, losses = ws.train(layers, proj.astype(np.float64), C, B, X, Y, norm, epochs=60, batch=32, lr=3e-3,
                         seed=1, mimic=False)
    assert losses[0] > 0.5
    assert losses[-1] < 0.15 * losses[0]
