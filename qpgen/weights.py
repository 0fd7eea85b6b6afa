"""Seeded initial parameters of the warm-start network.

Random draws only: the fixed input projection P (d x F, N(0, 1/F) entries, so
that a unit-variance input gives unit-variance features), hidden weights with
N(0, 2/fan_in) entries (He et al. 2015), an output layer with N(0, 0.01/fan_in)
entries so that the untrained network predicts close to the mean solution, and
zero biases.  All arrays are float32, row-major, W of shape (out, in).
"""
from __future__ import annotations

import numpy as np


def warmstart_params(seed: int, features: int, d: int = 1024, width: int = 1024, depth: int = 3):
    """Returns (proj, layers): proj (d x features) and a list of (W, b) for the
    `depth` hidden layers followed by the output layer (features x width)."""
    rng = np.random.default_rng(seed)
    proj = (rng.standard_normal((d, features)) / np.sqrt(features)).astype(np.float32)
    layers = []
    fan_in = d
    for _ in range(depth):
        W = (rng.standard_normal((width, fan_in)) * np.sqrt(2.0 / fan_in)).astype(np.float32)
        layers.append((W, np.zeros(width, np.float32)))
        fan_in = width
    W = (rng.standard_normal((features, fan_in)) * np.sqrt(0.01 / fan_in)).astype(np.float32)
    layers.append((W, np.zeros(features, np.float32)))
    return proj, layers
