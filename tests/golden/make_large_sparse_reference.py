"""Solve the n=1e6 large sparse QP once with the CPU oracle and store what the
tests and the bench need: iteration / restart / Lanczos step counts, the
spectral norms, objective values, relKKT parts and the optimal x*, y* at a
fixed sample of indices.  Calls only the oracle (and the seeded generator).

    python tests/golden/make_large_sparse_reference.py   # a few minutes of CPU
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import qpgen  # noqa: E402
from oracle import rapdhg as R  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_sparse_qp_reference.json")


def main():
    inst = qpgen.large_sparse_qp()
    t = time.time()
    res = R.solve(inst, R.Options())
    secs = time.time() - t
    rng = np.random.default_rng(7)
    xi = np.sort(rng.choice(inst.n, 64, replace=False))
    yi = np.sort(rng.choice(inst.m, 64, replace=False))
    rec = dict(
        what="CPU oracle solve of qpgen.large_sparse_qp() (n=1e6, m=5e5, seed 2311077101), default options",
        status=res.status, iterations=res.iterations, restarts=res.restarts,
        norm_steps_A=R.NORM_STEPS.get("A"), norm_steps_Q=R.NORM_STEPS.get("Q"),
        norm_A=res.norm_A, norm_Q=res.norm_Q, omega=res.omega, kkt=res.kkt,
        x_index=xi.tolist(), x_value=res.x[xi].tolist(), y_index=yi.tolist(), y_value=res.y[yi].tolist(),
        oracle_seconds=secs)
    json.dump(rec, open(OUT, "w"), indent=1)
    print(json.dumps({k: v for k, v in rec.items() if "index" not in k and "value" not in k}))


if __name__ == "__main__":
    main()
