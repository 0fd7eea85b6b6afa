"""Helpers shared by the GPU tests: building the library, creating handles from
generated instances, and comparing against the oracle."""
import numpy as np
import pytest


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def lib():
    from paper_2311_07710_gb300 import build, pdqp
    build.build()
    require_gpu()
    return pdqp


def handle(inst, device=False):
    from paper_2311_07710_gb300 import pdqp
    h = pdqp.create_from_csr(inst.n, inst.m, inst.m_eq, inst.Q, inst.A, inst.c, inst.b, inst.l, inst.u,
                             device=device)
    if getattr(inst, "F", None) is not None:
        pdqp.pdqp_set_lowrank_Q(h, inst.F.shape[1], np.ascontiguousarray(inst.F, dtype=np.float32))
    return h


def solve(inst, device=False, x0=None, y0=None, **opts):
    """Solve through the C ABI; returns (status, info, x, y)."""
    from paper_2311_07710_gb300 import pdqp
    h = handle(inst, device)
    try:
        o = pdqp.pdqp_default_options(**opts)
        x = np.zeros(inst.n)
        y = np.zeros(inst.m)
        st, info = pdqp.pdqp_solve(h, o, x0=x0, y0=y0, x_out=x, y_out=y)
        return st, info, x, y
    finally:
        pdqp.pdqp_destroy(h)


def state_after(inst, iters, **opts):
    """Raw (x, y, xbar, ybar) after `iters` iterations (no restart at the last one)."""
    from paper_2311_07710_gb300 import pdqp
    h = handle(inst)
    try:
        o = pdqp.pdqp_default_options(max_iter=iters, eps=0.0, **opts)
        pdqp.pdqp_solve(h, o)
        out = [np.zeros(inst.n), np.zeros(inst.m), np.zeros(inst.n), np.zeros(inst.m)]
        pdqp.pdqp_get_iterates(h, *out)
        return dict(x=out[0], y=out[1], xbar=out[2], ybar=out[3])
    finally:
        pdqp.pdqp_destroy(h)


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))
