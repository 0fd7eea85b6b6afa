"""Distinct handles are independent: four host threads each create, solve and
destroy their own problem on their own stream at the same time (the binding
releases the interpreter lock inside every library call); every result is
bitwise the one a sequential solve gives, and the launch counter covers the
launches of every thread."""
import threading

import numpy as np
import pytest

import qpgen
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def test_concurrent_handles_match_sequential_solves():
    import torch
    pd = G.lib()
    insts = [qpgen.random_sparse_qp(seed=qpgen.SEED_BASE + 7400 + k, n=300 + 100 * k, m=150 + 50 * k)
             for k in range(4)]
    precisions = [0, 1, 0, 1]
    seq = [G.solve(inst, precision=p)[2:] for inst, p in zip(insts, precisions)]
    out = [None] * 4
    errors = []
    barrier = threading.Barrier(4)

    def work(k):
        try:
            stream = torch.cuda.Stream()
            barrier.wait()
            h = G.handle(insts[k])
            try:
                x, y = np.zeros(insts[k].n), np.zeros(insts[k].m)
                st, info = pd.pdqp_solve(h, pd.pdqp_default_options(precision=precisions[k]), x_out=x, y_out=y,
                                         stream=stream)
                out[k] = (x, y, st)
            finally:
                pd.pdqp_destroy(h)
        except Exception as e:   # reported below, in the main thread
            errors.append(e)

    l0 = pd.pdqp_launch_count()
    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    assert pd.pdqp_launch_count() > l0
    for k in range(4):
        x, y, st = out[k]
        assert st == pd.PDQP_OK
        np.testing.assert_array_equal(x, seq[k][0])
        np.testing.assert_array_equal(y, seq[k][1])
