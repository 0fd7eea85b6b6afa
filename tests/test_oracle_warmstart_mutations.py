"""Planted mistakes in the warm-start oracle: each edits a copy of its source
on the CPU and at least one pin (finite differences, Adam's closed form, the
normalisation invariants) must then fail."""
import os
import sys
import types

import numpy as np
import pytest

import qpgen

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "warmstart.py")

MUTATIONS = {
    "no_relu_mask": ("dZ = rf(np.where(H[j] > 0.0, dH, 0.0))", "dZ = rf(dH)"),
    "mask_from_wrong_layer": ("dZ = rf(np.where(H[j] > 0.0, dH, 0.0))",
                              "dZ = rf(np.where(H[j - 1][:, :dH.shape[1]] > 0.0, dH, 0.0))"),
    "wrong_sample_pairing": ("gW = dZb.T @ H[j]", "gW = dZb.T @ H[j][::-1]"),
    "bias_grad_mean": ("gb = dZ.sum(axis=0)", "gb = dZ.mean(axis=0)"),
    "loss_scale": ("else (2.0 / (S * F)) * R", "else (1.0 / (S * F)) * R"),
    "input_grad_transposed_use": ("dH = dZb @ rb(W)", "dH = dZb @ rb(W)[:, ::-1]"),
    "adam_no_bias_correction": ("mhat = m / (1.0 - beta1 ** t)", "mhat = m"),
    "adam_second_moment_abs": ("(1.0 - beta2) * g * g", "(1.0 - beta2) * np.abs(g)"),
    "adam_sign": ("return p - lr * mhat", "return p + lr * mhat"),
    "norm_scale_is_std": ("in_scale=(1.0 / si).astype(np.float32)", "in_scale=si.astype(np.float32)"),
    "out_inv_is_std": ("out_inv=(1.0 / so).astype(np.float32)", "out_inv=so.astype(np.float32)"),
}


def _load(mutation):
    src = open(SRC).read()
    old, new = MUTATIONS[mutation]
    assert src.count(old) >= 1, f"mutation anchor not found: {mutation}"
    name = "warmstart_mutant_" + mutation
    mod = types.ModuleType(name)
    sys.modules[name] = mod
    exec(compile(src.replace(old, new), name, "exec"), mod.__dict__)
    return mod


def _pins_pass(W):
    try:
        proj, layers = qpgen.warmstart_params(3, 7, 6, 5, 2)
        proj = proj.astype(np.float64)
        layers = [(w.astype(np.float64) * (10.0 if i == 2 else 1.0), b.astype(np.float64) + 0.05)
                  for i, (w, b) in enumerate(layers)]
        rng = np.random.default_rng(1)
        U = rng.standard_normal((5, 7))
        T = rng.standard_normal((5, 7))
        _, grads = W.loss_and_grads(layers, proj, U, T, mimic=False)
        h = 1e-6
        for li, (Wm, b) in enumerate(layers):
            for which, P in ((0, Wm), (1, b)):
                it = np.nditer(P, flags=["multi_index"])
                for _ in it:
                    idx = it.multi_index
                    old = P[idx]
                    P[idx] = old + h
                    lp = W.loss_and_grads(layers, proj, U, T, mimic=False)[0]
                    P[idx] = old - h
                    lm = W.loss_and_grads(layers, proj, U, T, mimic=False)[0]
                    P[idx] = old
                    if abs(grads[li][which][idx] - (lp - lm) / (2 * h)) > 1e-6 * max(1.0, abs(lp - lm) / (2 * h)):
                        return False
        g = np.array([3.0, -0.5, 1e-3])
        p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
        for t in range(1, 4):
            p, m, v = W.adam_step(p, g, m, v, t, 0.01, 0.9, 0.999, 1e-8)
            if np.max(np.abs(p + t * 0.01 * g / (np.abs(g) + 1e-8))) > 1e-12:
                return False
        C = 3.0 + 0.1 * rng.standard_normal((100, 4))
        B = rng.standard_normal((100, 2))
        X = 5.0 * rng.standard_normal((100, 3))
        Y = rng.standard_normal((100, 2))
        norm = W.fit_normalization(C, B, X, Y)
        Un = W.prep_input(C, B, norm, mimic=False)
        Tn = W.prep_target(X, Y, norm, mimic=False)
        if np.max(np.abs(Un.std(0) - 1.0)) > 1e-5 or np.max(np.abs(Tn.std(0) - 1.0)) > 1e-5:
            return False
        return True
    except (ValueError, IndexError, FloatingPointError, ZeroDivisionError):
        return False


def test_unmutated_passes():
    from oracle import warmstart
    assert _pins_pass(warmstart)


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_planted_mistake_is_caught(mutation):
    with np.errstate(all="ignore"):
        assert not _pins_pass(_load(mutation))
