"""CPU checks of the binding's host-side behaviour (no CUDA call is made):
the defaults the C library fills are the ones include/pdqp.h documents, an
unknown option name is an error, every status code has its name."""
import pytest

from paper_2311_07710_gb300 import build, pdqp


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_defaults_are_the_documented_ones():
    o = pdqp.pdqp_default_options()
    assert (o.precision, o.step_rule, o.restart_rule) == (pdqp.PDQP_PREC_FP64, 0, 0)
    assert (o.accelerate, o.scaling, o.ruiz_iters, o.l2_scaling, o.pock_chambolle) == (1, 1, 10, 1, 1)
    assert (o.check_period, o.max_iter, o.eps, o.time_limit) == (64, 200_000, 1e-6, 3600.0)
    assert (o.beta_suff, o.beta_nec, o.beta_art, o.pw_theta, o.eps_zero) == (0.2, 0.8, 0.36, 0.2, 1e-10)
    assert (o.norm_A, o.norm_Q, o.norm_iters, o.norm_tol) == (0.0, 0.0, 500, 1e-6)
    assert (o.spmv_threads, o.no_graphs, o.detect_infeasibility, o.eps_infeasible) == (0, 0, 0, 1e-8)


def test_overrides_and_unknown_names():
    o = pdqp.pdqp_default_options(precision=pdqp.PDQP_PREC_MIXED, eps=1e-4, detect_infeasibility=1)
    assert (o.precision, o.eps, o.detect_infeasibility) == (pdqp.PDQP_PREC_MIXED, 1e-4, 1)
    with pytest.raises(AttributeError):
        pdqp.pdqp_default_options(detect_infeasibilty=1)


def test_status_names():
    names = {pdqp.PDQP_OK: "optimal", pdqp.PDQP_ERR_INVALID: "invalid input", pdqp.PDQP_ERR_CUDA: "CUDA error",
             pdqp.PDQP_ERR_OOM: "out of memory", pdqp.PDQP_ITER_LIMIT: "iteration limit",
             pdqp.PDQP_TIME_LIMIT: "time limit", pdqp.PDQP_NUMERICAL: "numerical error",
             pdqp.PDQP_DEVICE_TIMEOUT: "device timeout", pdqp.PDQP_PRIMAL_INFEASIBLE: "primal infeasible",
             pdqp.PDQP_DUAL_INFEASIBLE: "dual infeasible"}
    for code, name in names.items():
        assert pdqp.status_string(code) == name
    assert pdqp.status_string(99) == "unknown status"
