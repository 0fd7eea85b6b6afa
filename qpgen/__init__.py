"""Seeded synthetic QP instances shared by the oracle, the tests and the bench."""
from .instances import (  # noqa: F401
    QPInstance, QPFamily, SEED_BASE, random_sparse_qp, large_sparse_qp, portfolio_qp,
    mpc_qp, mpc_batch, family_qp, tiny_qp, diagonal_box_qp,
)
from .weights import warmstart_params  # noqa: F401
from .classes import lasso_qp, huber_qp, svm_qp  # noqa: F401
